// Unpack (Sec. 3.1, 3.3), reciprocal reconstruction (Sec. 3.2, used twice by
// Sec. 3.4), the signed-bias correction and the reduction mod p (Sec. 4).
#include "ks_internal.cuh"
#include "ks_src.cuh"

namespace ks {

// ------------------------------------------------------------------ unpack
// h'_k = bits [off + kN, off + kN + width) of V (or of V_odd for odd k), and
// h_k = h'_k - 2^kb for signed inputs (kb >= 0).
// KS1: V = h(2^N), off = 0, width N.  KS2: V = P+ + P- = 2 h0(X^2) and
// V_odd = P+ - P- = 2X h1(X^2); then both even and odd coefficients sit at
// bit 1 + kN, width 2N (Sec. 3.3).
// One CTA writes 1024 consecutive output limbs, four per thread (strided by
// the block, so every store is coalesced and the four loads are independent).
constexpr int kUnpackPer = 4;
template <class Src>
__global__ void __launch_bounds__(256) unpack_kernel(Src src) {
  pdl_enter();
  int64_t local;
  const UnpackArgs &a = src.locate(blockIdx.x, local);
  const int64_t total = a.lh * a.ol;
  const int64_t base = local * (256 * kUnpackPer) + threadIdx.x;
  const bool narrow = total < ((int64_t)1 << 31);  // 32-bit index arithmetic suffices
#pragma unroll
  for (int i = 0; i < kUnpackPer; i++) {
    const int64_t idx = base + 256 * i;
    if (idx >= total) break;
    int64_t k;
    int l;
    if (narrow) {
      const uint32_t q = (uint32_t)idx / (uint32_t)a.ol;
      k = q;
      l = (int)((uint32_t)idx - q * (uint32_t)a.ol);
    } else {
      k = idx / a.ol;
      l = (int)(idx - k * a.ol);
    }
    const uint32_t *src_w = (a.V_odd != nullptr && (k & 1)) ? a.V_odd : a.V;
    const int rem = a.width - 64 * l;
    const int64_t pos = a.off + k * a.N;
    uint64_t v = 0;
    if (rem > 0) {
      v = get_bits64(src_w, a.nwords, pos + 64 * (int64_t)l);
      if (rem < 64) v &= (1ull << rem) - 1ull;
    }
    const int kb = a.kb;
    if (kb >= 0) {
      // field - 2^kb, limb l, two's complement: the field is at most 2^(kb+1)
      // (bits kb, kb + 1 lie inside it), so a limb above K's borrows exactly
      // when the field's bits [kb, 64 l) are all zero
      if (64 * l <= kb) {
        if (kb < 64 * l + 64) v -= 1ull << (kb - 64 * l);
      } else {
        const uint64_t top = get_bits64(src_w, a.nwords, pos + kb) & (64 * l - kb >= 2 ? 3ull : 1ull);
        if (top == 0) v -= 1ull;
      }
    }
    a.h[idx] = v;
  }
}

static unsigned grid_for(int64_t n, int threads) {
  int64_t b = (n + threads - 1) / threads;
  if (b < 1) b = 1;
  if (b > 152 * 32) b = 152 * 32;
  return (unsigned)b;
}

int64_t unpack_blocks(const UnpackArgs &a) {
  return (a.lh * a.ol + 256 * kUnpackPer - 1) / (256 * kUnpackPer);
}

cudaError_t launch_unpack(const UnpackArgs &a, cudaStream_t s) {
  (void)launch_k(unpack_kernel<One<UnpackArgs>>, dim3((unsigned)unpack_blocks(a)), dim3(256), 0, s, One<UnpackArgs>{a});
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_unpack_batch(const UnpackArgs *d, const int64_t *prefix, int n,
                                int64_t blocks, cudaStream_t s) {
  if (blocks == 0) return cudaSuccess;
  (void)launch_k(unpack_kernel<Many<UnpackArgs>>, dim3((unsigned)blocks), dim3(256), 0, s, Many<UnpackArgs>{d, prefix, n});
  note_launches(1);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ recover
// Sec. 3.2: from the base-X digits u_i of fwd = sum c_i X^i and w_i of
// rev = sum c_(n-1-i) X^i (fwd = sum_{i<=n} u_i X^i, rev = sum_{i<=n}
// w_(n-i) X^i), with c_i = alpha_i + X beta_i, 0 <= alpha_i < X,
// 0 <= beta_i < X - 1, run for j = 0 .. n-2:
//
//   eps_j       = [alpha_j > w_(j+1)]
//   beta_j      = w_j - alpha_(j-1) - eps_j            (mod X)
//   alpha_(j+1) = u_(j+1) - beta_j - delta_j           (mod X)
//   delta_(j+1) = (beta_j + alpha_(j+1) + delta_j - u_(j+1)) / X  in {0, 1}
//
// and finally beta_(n-1) = w_(n-1) - alpha_(n-2) (mod X).  The recurrence is
// sequential; chains of `chain` steps run in parallel.  A chain starting at s
// from the exact values c_(s-1), c_s: alpha_(s-1), alpha_s, beta_(s-1) follow
// directly, and delta_(s-1) = u_s - beta_(s-1) - alpha_s (mod X, necessarily 0
// or 1) gives delta_s = (beta_(s-1) + alpha_s + delta_(s-1) - u_s) / X.  The
// same recurrence on the reversed problem x^(n-1) h(1/x) (fwd and rev
// exchanged) runs downward, so every exact pair starts one chain each way (see
// RecoverRun).  Signed inputs arrive shifted by K = 2^kb, which the output
// subtracts.
namespace {

}  // namespace

// Digits of at most 63 bits live in one 64-bit register; digits of 64..127
// bits in a pair of 64-bit limbs (D2) with explicit carries.
__device__ __forceinline__ uint64_t load_d1(const uint32_t *V, int64_t nwords, int64_t pos, int M) {
  return get_bits64(V, nwords, pos) & ((1ull << M) - 1ull);
}
struct D2 {
  uint64_t lo, hi;
};
__device__ __forceinline__ uint64_t hi_mask(int M) {  // 64 <= M <= 127
  return (M - 64 == 64) ? ~0ull : ((1ull << (M - 64)) - 1ull);
}
__device__ __forceinline__ D2 load_d2(const uint32_t *V, int64_t nwords, int64_t pos, int M) {
  D2 r;
  r.lo = get_bits64(V, nwords, pos);
  r.hi = get_bits64(V, nwords, pos + 64) & hi_mask(M);
  return r;
}
// Seed value v as kAccSeedWords 32-bit words: the narrow seed kernel's six
// 64-bit column sums carried (mod 2^192: the top words are zero), or the wide
// seed kernel's words.
__device__ __forceinline__ void seed_value(const RecoverArgs &a, int64_t v,
                                           uint32_t (&out)[kAccSeedWords]) {
  if (a.seed_acc != nullptr) {
    const unsigned long long *acc = a.seed_acc + v * 6;
    unsigned long long col[6];
#pragma unroll
    for (int w = 0; w < 6; w++) col[w] = acc[w];
    unsigned long long carry = 0;
#pragma unroll
    for (int w = 0; w < kAccSeedWords; w++) {
      const unsigned long long x = (w < 6 ? col[w] : 0ull) + carry;
      out[w] = w < 6 ? (uint32_t)x : 0u;
      carry = x >> 32;
    }
  } else {
    const int nw = a.seed_words;
#pragma unroll
    for (int w = 0; w < kAccSeedWords; w++) out[w] = w < nw ? a.seeds[v * nw + w] : 0u;
  }
}
// (a - b - c) mod 2^M, c in {0, 1}
__device__ __forceinline__ D2 sub_d2(D2 a, D2 b, uint64_t c, int M) {
  D2 r;
  const uint64_t t = a.lo - b.lo;
  const uint64_t bw1 = a.lo < b.lo;
  r.lo = t - c;
  const uint64_t bw2 = t < c;
  r.hi = (a.hi - b.hi - bw1 - bw2) & hi_mask(M);
  return r;
}
// floor((a + b + c) / 2^M) for a, b < 2^M, c in {0, 1}
__device__ __forceinline__ uint64_t carry_d2(D2 a, D2 b, uint64_t c, int M) {
  const uint64_t s1 = a.lo + b.lo;
  const uint64_t c1 = s1 < a.lo;
  const uint64_t s2 = s1 + c;
  const uint64_t c2 = s2 < s1;
  const uint64_t hs = a.hi + b.hi + c1 + c2;  // < 2^(M-63) <= 2^64
  return (hs >> (M - 64)) & 1ull;
}
__device__ __forceinline__ bool gt_d2(D2 a, D2 b) {
  return a.hi != b.hi ? a.hi > b.hi : a.lo > b.lo;
}
// limb l of K = 2^kb (kb < 0: no shift)
__device__ __forceinline__ uint64_t k_limb(int kb, int l) {
  return (kb >= 0 && (kb >> 6) == l) ? 1ull << (kb & 63) : 0ull;
}
// out[l] = limb l of the value minus K, two's complement over ol limbs
__device__ __forceinline__ uint64_t sub_k(uint64_t v, int kb, int l, uint64_t &borrow) {
  const uint64_t k = k_limb(kb, l);
  const uint64_t d1 = v - k;
  const uint64_t b1 = v < k;
  const uint64_t d2 = d1 - borrow;
  const uint64_t b2 = d1 < borrow;
  borrow = b1 | b2;
  return d2;
}
// out limbs of alpha + 2^M beta - K, alpha, beta < 2^M (64 <= M < 128)
__device__ __forceinline__ void write_h2(uint64_t *out, int ol, D2 a, D2 be, int M, int kb) {
  uint64_t s[5] = {a.lo, a.hi, 0, 0, 0};
  const int r = M & 63;  // beta starts in limb 1
  s[1] |= be.lo << r;
  s[2] |= (r ? (be.lo >> (64 - r)) : 0ull) | (be.hi << r);
  s[3] |= r ? (be.hi >> (64 - r)) : 0ull;
  uint64_t borrow = 0;
#pragma unroll
  for (int l = 0; l < 5; l++)  // ol <= 5 here (2M + 2 bits): s stays in registers
    if (l < ol) out[l] = sub_k(s[l], kb, l, borrow);
}

__device__ __forceinline__ bool chain_index(const RecoverArgs &a, int64_t &gid, int &r) {
  r = 0;
  while (r < a.nruns && gid >= a.run[r].nchains) {
    gid -= a.run[r].nchains;
    r++;
  }
  return r < a.nruns;
}

// The strings a chain walks.  Step t of chain c reads DU(t + 1) and DW(t + 1):
//   upward from s:   DU(t) = u_(s+t) = digit s + t of fwd,
//                    DW(t) = w_(s+t) = digit n - s - t of rev;
//   downward from s: DU(t) = w_(s-t) = digit n - s + t of rev,
//                    DW(t) = u_(s-t) = digit s - t of fwd
// (the reversed problem: fwd and rev exchanged, s -> n - s), so DU walks one
// string up from pA and DW the other down from pB.  The chain's step t is the
// reversed or plain run's coefficient pA + t; the last coefficient of the run
// (pA + t = n - 1) takes beta = w - alpha_prev.  Step t outputs run coefficient
// s + t (upward) or s - 1 - t (downward).
struct ChainLane {
  const uint32_t *A, *B;
  int64_t offA, offB, pA, pB, s, len;
  bool up, seeded;
  int64_t vprev, vcur;  // seed value indices (seeded chains)
};
__device__ __forceinline__ ChainLane chain_lane(const RecoverArgs &a, const RecoverRun &R,
                                                int64_t c) {
  ChainLane L;
  chain_geom(R.n, a.chain, c, L.up, L.s, L.len, L.seeded);
  L.A = L.up ? R.Vf : R.Vr;
  L.offA = L.up ? R.off_f : R.off_r;
  L.B = L.up ? R.Vr : R.Vf;
  L.offB = L.up ? R.off_r : R.off_f;
  L.pA = L.up ? L.s : R.n - L.s;
  L.pB = L.up ? R.n - L.s : L.s;
  // pair j starts the downward chain 2j and the upward chain 2j + 1; the
  // downward chain sees the pair reversed: (c_s, c_(s-1))
  const int64_t pair = L.up ? (c - 1) >> 1 : c >> 1;
  const int64_t vp = pair * a.C + R.slot_prev, vc = pair * a.C + R.slot_cur;
  L.vprev = L.up ? vp : vc;
  L.vcur = L.up ? vc : vp;
  return L;
}
__device__ __forceinline__ int64_t lane_coeff(const ChainLane &L, int64_t t) {
  return L.up ? L.s + t : L.s - 1 - t;
}

// M <= 63, digits staged in shared memory.  A CTA of 128 threads runs cpc
// consecutive chains of one run (cpc <= 32, cpc * chain <= 2048), which
// cover the coefficients [j0, jhi) without gaps:
//  1. one bulk copy of the bit ranges of V_f and V_r holding u_j and w_j,
//     j0 <= j <= jhi (upward and downward chains read the same digits);
//  2. all threads extract each chain's DU(t), DW(t) into [t][lane] arrays;
//  3. warp 0, one lane per chain, runs the recurrence of Sec. 3.2 from shared
//     memory and stages the coefficients in [position][lane] order;
//  4. all threads write the coefficients out (minus K for signed inputs).
constexpr int kRT = 128;
constexpr int kRCmax = 32;

// 64 bits at bit `pos` of a staged word range (words outside [0, nw) read as zero)
__device__ __forceinline__ uint64_t sbits64(const uint32_t *w, int64_t nw, int64_t pos) {
  const int64_t i = pos >> 5;
  const int sh = (int)(pos & 31);
  const uint64_t w0 = (i >= 0 && i < nw) ? w[i] : 0u;
  const uint64_t w1 = (i + 1 >= 0 && i + 1 < nw) ? w[i + 1] : 0u;
  const uint64_t w2 = (i + 2 >= 0 && i + 2 < nw) ? w[i + 2] : 0u;
  const uint64_t lo = w0 | (w1 << 32);
  return sh ? ((lo >> sh) | (w2 << (64 - sh))) : lo;
}

// the most chains per CTA for this chain length (2048 / chain, at most 32)
__host__ __device__ __forceinline__ int recover_cpc(int64_t chain) {
  int64_t c = 2048 / chain;
  return (int)(c < 1 ? 1 : (c > kRCmax ? kRCmax : c));
}
// staged words of one digit string (multiple of four)
__host__ __device__ __forceinline__ int64_t staged_words(int64_t chain, int M, int cpc) {
  return (((cpc * chain + 2) * (int64_t)M + 31) / 32 + 12) & ~(int64_t)3;
}
// digits of one string, [step t in 0..chain][lane]
__host__ __device__ __forceinline__ int64_t staged_digits(int64_t chain, int cpc) {
  return (chain + 1) * cpc;
}
__host__ __device__ __forceinline__ int64_t staged_bytes(int64_t chain, int M, int cpc) {
  return 2 * staged_words(chain, M, cpc) * 4 + 2 * staged_digits(chain, cpc) * 8 +
         cpc * chain * 2 * 8;
}

template <class Src>
__global__ void __launch_bounds__(kRT) recover_staged1(Src src) {
  pdl_enter();
  extern __shared__ __align__(16) uint32_t stg[];
  __shared__ __align__(8) uint64_t bar;
  int64_t local;
  const RecoverArgs &a = src.locate(blockIdx.x, local);
  int r = 0;
  while (r + 1 < a.nruns && local >= a.rblocks[r]) {
    local -= a.rblocks[r];
    r++;
  }
  const RecoverRun &R = a.run[r];
  int *status = a.status;
  const int M = a.M, ol = a.ol, kb = a.kb;
  const uint64_t mask = (1ull << M) - 1ull;
  const int64_t n = R.n, chain = a.chain, nwords = a.nwords;
  const int cpc = a.cpc;
  const int tid = threadIdx.x;
  const int64_t c0 = local * cpc;
  const int64_t c1 = c0 + cpc < R.nchains ? c0 + cpc : R.nchains;
  const int64_t j0 = c0 * chain;                        // first coefficient of the CTA
  const int64_t jhi = c1 * chain < n ? c1 * chain : n;  // one past the last
  // digits u_j, j in [j0, jhi]; w_m, m in [n - jhi, n - j0]
  const int64_t ub0 = ((R.off_f + j0 * (int64_t)M) >> 5) & ~(int64_t)3;
  const int64_t nu = ((((R.off_f + (jhi + 1) * (int64_t)M) >> 5) + 3 - ub0) + 3) & ~(int64_t)3;
  const int64_t wb0 = ((R.off_r + (n - jhi) * (int64_t)M) >> 5) & ~(int64_t)3;
  const int64_t nw = ((((R.off_r + (n - j0 + 1) * (int64_t)M) >> 5) + 3 - wb0) + 3) &
                     ~(int64_t)3;
  const int64_t capw = staged_words(chain, M, cpc), capd = staged_digits(chain, cpc);
  if (nu > capw || nw > capw || ub0 < 0 || wb0 < 0 || (chain & (chain - 1)) != 0 || ol > 2) {
    if (tid == 0) atomicCAS(status, 0, 3);  // not for a plan from make_recover_args
    return;
  }
  uint32_t *su = stg, *sw = stg + capw;
  uint64_t *du = reinterpret_cast<uint64_t *>(stg + 2 * capw);
  uint64_t *dw = du + capd;
  uint64_t *so = dw + capd;  // so(position p, lane i): coefficient of lane i at offset p
  // 1. the part of each word range inside the array arrives by bulk copy; the rest is zero
  const int64_t cu = ub0 + nu <= nwords ? nu : (nwords > ub0 ? nwords - ub0 : 0);
  const int64_t cw = wb0 + nw <= nwords ? nw : (nwords > wb0 ? nwords - wb0 : 0);
  for (int64_t i = cu + tid; i < nu; i += kRT) su[i] = 0u;
  for (int64_t i = cw + tid; i < nw; i += kRT) sw[i] = 0u;
  if (tid == 0) {
    stage_init(&bar);
    stage_expect(&bar, (uint32_t)((cu + cw) * 4));
    if (cu > 0) stage_copy(su, R.Vf + ub0, (uint32_t)(cu * 4), &bar);
    if (cw > 0) stage_copy(sw, R.Vr + wb0, (uint32_t)(cw * 4), &bar);
  }
  // the seeds of this thread's chain, while the copies fly
  const int64_t c_me = c0 + tid;
  const bool chain_lane_me = tid < 32 && c_me < c1;
  uint32_t s0[kAccSeedWords], s1[kAccSeedWords];
  ChainLane Lm;
  if (chain_lane_me) {
    Lm = chain_lane(a, R, c_me);
    if (Lm.seeded) {
      seed_value(a, Lm.vprev, s0);
      seed_value(a, Lm.vcur, s1);
    }
  }
  __syncthreads();
  if (!__syncthreads_and(stage_wait(&bar))) {
    if (tid == 0) atomicCAS(status, 0, 1);
    stage_wait(&bar);  // once more (bounded) for the copies in flight before leaving
    return;
  }
  // 2. each chain's digits (chain and cpc are powers of two)
  const int lc = __ffsll((long long)chain) - 1, lp = __ffs(cpc) - 1;
  const int64_t pu = R.off_f - ub0 * 32, pw = R.off_r - wb0 * 32;  // staged bit offsets
  for (int q = tid; q < (int)capd; q += kRT) {
    const int t = q >> lp, i = q & (cpc - 1);
    const int64_t c = c0 + i;
    uint64_t x = 0, y = 0;
    if (c < c1) {
      bool up, seeded;
      int64_t s, len;
      chain_geom(n, chain, c, up, s, len, seeded);
      if (t <= len) {
        const int64_t j = up ? s + t : s - t;  // in [j0, jhi]
        const uint64_t uj = sbits64(su, nu, pu + j * (int64_t)M) & mask;
        const uint64_t wj = sbits64(sw, nw, pw + (n - j) * (int64_t)M) & mask;
        x = up ? uj : wj;
        y = up ? wj : uj;
      }
    }
    du[q] = x;
    dw[q] = y;
  }
  __syncthreads();
  // 3. the chains (warp 0)
  if (chain_lane_me) {
    const int ln = tid;
    const ChainLane &L = Lm;
    uint64_t a_prev, a_cur, delta;
    if (!L.seeded) {  // downward from n: the reversed problem's start at index 0
      a_prev = 0;
      a_cur = du[ln];
      delta = 0;
    } else {
      a_prev = load_d1(s0, kAccSeedWords, 0, M);
      const uint64_t b_prev = load_d1(s0, kAccSeedWords, M, M);
      a_cur = load_d1(s1, kAccSeedWords, 0, M);
      const uint64_t us = du[ln];
      const uint64_t dprev = (us - b_prev - a_cur) & mask;
      if (dprev > 1) atomicCAS(status, 0, 2);
      delta = (b_prev + a_cur + dprev - us) >> M;
    }
    uint64_t w_cur = dw[ln];
    // step t reads du(t + 1, ln) and dw(t + 1, ln): eight steps' digits are
    // loaded at once, then the eight steps run with compile-time indices.  A
    // step keeps only the recurrence on its critical path (alpha, the carries);
    // it stores (alpha_j, beta_j), and the output phase forms the coefficient.
    // delta_(j+1) = [beta_j + delta_j > u_(j+1)]: alpha_(j+1) wrapped below
    // zero exactly then.  (delta, epsilon are 0 or 1 by construction once the
    // start is consistent, which the seed check above verified.)  The run's
    // last coefficient (beta_(n-1) = w_(n-1) - alpha_(n-2)) can only be a
    // chain's final step and is taken after the loop.
    const uint64_t *pdu = du + cpc + ln, *pdw = dw + cpc + ln;
    const int len = (int)L.len;
    const int64_t last = n - 1 - L.pA;  // step of the run's last coefficient
    const int steps = last == len - 1 ? len - 1 : len;
    uint64_t *po = so + 2 * ln;
    const int pstride = 2 * cpc;  // so words between consecutive positions
    const int pos0 = L.up ? 0 : len - 1, pdir = L.up ? pstride : -pstride;
    for (int t0 = 0; t0 < steps; t0 += 8) {
      uint64_t U[8], Wn[8];
#pragma unroll
      for (int q = 0; q < 8; q++) {
        const bool in = t0 + q < (int)chain;  // rows up to chain exist
        U[q] = in ? pdu[(t0 + q) * cpc] : 0ull;
        Wn[q] = in ? pdw[(t0 + q) * cpc] : 0ull;
      }
      uint64_t *out = po + pos0 * pstride + t0 * pdir;
#pragma unroll
      for (int q = 0; q < 8; q++) {
        if (t0 + q >= steps) break;
        const uint64_t eps = a_cur > Wn[q] ? 1ull : 0ull;
        const uint64_t beta = (w_cur - a_prev - eps) & mask;
        const uint64_t a_next = (U[q] - beta - delta) & mask;
        const uint64_t dnext = beta + delta > U[q] ? 1ull : 0ull;
        out[0] = a_cur;
        out[1] = beta;
        out += pdir;
        a_prev = a_cur;
        a_cur = a_next;
        delta = dnext;
        w_cur = Wn[q];
      }
    }
    if (steps < len) {
      uint64_t *out = po + (pos0 + (int64_t)steps * (L.up ? 1 : -1)) * pstride;
      out[0] = a_cur;
      out[1] = (w_cur - a_prev) & mask;
    }
  }
  __syncthreads();
  // 4. coefficients alpha + 2^M beta out, minus K
  uint64_t *h = a.h;
  for (int q = tid; q < (int)((jhi - j0) * ol); q += kRT) {
    const int jj = ol == 2 ? q >> 1 : q;
    const int l = q - jj * ol;
    const int i = jj >> lc, p = jj & (int)(chain - 1);
    const uint64_t *v = so + 2 * (((int64_t)p << lp) + i);
    const uint64_t lo = v[0] | (v[1] << M), hi = v[1] >> (64 - M);
    uint64_t w = l == 0 ? lo : hi;
    if (kb >= 0) {
      uint64_t borrow = 0;
      const uint64_t l0 = sub_k(lo, kb, 0, borrow);
      w = l == 0 ? l0 : sub_k(hi, kb, 1, borrow);
    }
    h[(R.kbase + R.kstride * (j0 + jj)) * ol + l] = w;
  }
}

// 64 <= M <= 127, digits staged in shared memory: the scheme of the kernel
// above with two-limb digits (D2).  A CTA of 128 threads runs cpc <= 16
// consecutive chains of one run: one bulk copy of the word ranges holding
// the CTA's u_j and w_j, all threads extract each chain's digits, warp 0
// (a lane per chain) runs the recurrence from shared memory and stages
// (alpha, beta) per coefficient, and all threads write the coefficients.
constexpr int kRC2max = 16;
__host__ __device__ __forceinline__ int64_t staged2_bytes(int64_t chain, int M, int cpc) {
  // two word ranges, four digit arrays (u, w: lo, hi), (alpha, beta) per coefficient
  return 2 * staged_words(chain, M, cpc) * 4 + 4 * staged_digits(chain, cpc) * 8 +
         cpc * chain * 4 * 8;
}
template <class Src>
__global__ void __launch_bounds__(kRT) recover_staged2(Src src) {
  pdl_enter();
  extern __shared__ __align__(16) uint32_t stg[];
  __shared__ __align__(8) uint64_t bar;
  int64_t local;
  const RecoverArgs &a = src.locate(blockIdx.x, local);
  int r = 0;
  while (r + 1 < a.nruns && local >= a.rblocks[r]) {
    local -= a.rblocks[r];
    r++;
  }
  const RecoverRun &R = a.run[r];
  int *status = a.status;
  const int M = a.M, ol = a.ol, kb = a.kb;
  const uint64_t hmask = (1ull << (M - 64)) - 1ull;  // 64 <= M <= 127
  const int64_t n = R.n, chain = a.chain, nwords = a.nwords;
  const int cpc = a.cpc;
  const int tid = threadIdx.x;
  const int64_t c0 = local * cpc;
  const int64_t c1 = c0 + cpc < R.nchains ? c0 + cpc : R.nchains;
  const int64_t j0 = c0 * chain;
  const int64_t jhi = c1 * chain < n ? c1 * chain : n;
  const int64_t ub0 = ((R.off_f + j0 * (int64_t)M) >> 5) & ~(int64_t)3;
  const int64_t nu = ((((R.off_f + (jhi + 1) * (int64_t)M) >> 5) + 5 - ub0) + 3) & ~(int64_t)3;
  const int64_t wb0 = ((R.off_r + (n - jhi) * (int64_t)M) >> 5) & ~(int64_t)3;
  const int64_t nw = ((((R.off_r + (n - j0 + 1) * (int64_t)M) >> 5) + 5 - wb0) + 3) &
                     ~(int64_t)3;
  const int64_t capw = staged_words(chain, M, cpc), capd = staged_digits(chain, cpc);
  if (nu > capw || nw > capw || ub0 < 0 || wb0 < 0 || (chain & (chain - 1)) != 0 || ol > 5 ||
      M < 64 || M > 127) {
    if (tid == 0) atomicCAS(status, 0, 3);  // not for a plan from make_recover_args
    return;
  }
  uint32_t *su = stg, *sw = stg + capw;
  uint64_t *dul = reinterpret_cast<uint64_t *>(stg + 2 * capw);
  uint64_t *duh = dul + capd, *dwl = duh + capd, *dwh = dwl + capd;
  uint64_t *so = dwh + capd;  // so(position p, lane i): alpha lo, hi, beta lo, hi
  const int64_t cu = ub0 + nu <= nwords ? nu : (nwords > ub0 ? nwords - ub0 : 0);
  const int64_t cw = wb0 + nw <= nwords ? nw : (nwords > wb0 ? nwords - wb0 : 0);
  for (int64_t i = cu + tid; i < nu; i += kRT) su[i] = 0u;
  for (int64_t i = cw + tid; i < nw; i += kRT) sw[i] = 0u;
  if (tid == 0) {
    stage_init(&bar);
    stage_expect(&bar, (uint32_t)((cu + cw) * 4));
    if (cu > 0) stage_copy(su, R.Vf + ub0, (uint32_t)(cu * 4), &bar);
    if (cw > 0) stage_copy(sw, R.Vr + wb0, (uint32_t)(cw * 4), &bar);
  }
  const int64_t c_me = c0 + tid;
  const bool chain_lane_me = tid < 32 && c_me < c1;
  uint32_t s0[kAccSeedWords], s1[kAccSeedWords];
  ChainLane Lm;
  if (chain_lane_me) {
    Lm = chain_lane(a, R, c_me);
    if (Lm.seeded) {
      seed_value(a, Lm.vprev, s0);
      seed_value(a, Lm.vcur, s1);
    }
  }
  __syncthreads();
  if (!__syncthreads_and(stage_wait(&bar))) {
    if (tid == 0) atomicCAS(status, 0, 1);
    stage_wait(&bar);  // once more (bounded) for the copies in flight before leaving
    return;
  }
  // each chain's digits, [step t][chain i] (chain and cpc are powers of two)
  const int lc = __ffsll((long long)chain) - 1, lp = __ffs(cpc) - 1;
  const int64_t pu = R.off_f - ub0 * 32, pw = R.off_r - wb0 * 32;
  for (int q = tid; q < (int)capd; q += kRT) {
    const int t = q >> lp, i = q & (cpc - 1);
    const int64_t c = c0 + i;
    uint64_t xl = 0, xh = 0, yl = 0, yh = 0;
    if (c < c1) {
      bool up, seeded;
      int64_t s_, len;
      chain_geom(n, chain, c, up, s_, len, seeded);
      if (t <= len) {
        const int64_t j = up ? s_ + t : s_ - t;
        const int64_t bu = pu + j * (int64_t)M, bw = pw + (n - j) * (int64_t)M;
        const uint64_t ul = sbits64(su, nu, bu), uh = sbits64(su, nu, bu + 64) & hmask;
        const uint64_t wl = sbits64(sw, nw, bw), wh = sbits64(sw, nw, bw + 64) & hmask;
        xl = up ? ul : wl;
        xh = up ? uh : wh;
        yl = up ? wl : ul;
        yh = up ? wh : uh;
      }
    }
    dul[q] = xl;
    duh[q] = xh;
    dwl[q] = yl;
    dwh[q] = yh;
  }
  __syncthreads();
  // the chains (warp 0)
  if (chain_lane_me) {
    const int ln = tid;
    const ChainLane &L = Lm;
    const D2 zero = {0ull, 0ull};
    D2 a_prev, a_cur;
    uint64_t delta;
    if (!L.seeded) {
      a_prev = zero;
      a_cur = D2{dul[ln], duh[ln]};
      delta = 0;
    } else {
      a_prev = load_d2(s0, kAccSeedWords, 0, M);
      const D2 b_prev = load_d2(s0, kAccSeedWords, M, M);
      a_cur = load_d2(s1, kAccSeedWords, 0, M);
      const D2 us = D2{dul[ln], duh[ln]};
      const D2 dprev = sub_d2(sub_d2(us, b_prev, 0, M), a_cur, 0, M);
      if (dprev.hi != 0 || dprev.lo > 1) atomicCAS(status, 0, 2);
      delta = carry_d2(b_prev, a_cur, dprev.lo & 1ull, M);
    }
    D2 w_cur = D2{dwl[ln], dwh[ln]};
    const int len = (int)L.len;
    const int64_t last = n - 1 - L.pA;
    const int steps = last == len - 1 ? len - 1 : len;
    const int pstride = 4 * cpc;  // so words between consecutive positions
    uint64_t *po = so + 4 * ln + (L.up ? 0 : (int64_t)(len - 1) * pstride);
    const int pdir = L.up ? pstride : -pstride;
    for (int t = 0; t < steps; t++) {
      const int q = (t + 1) * cpc + ln;
      const D2 u_next = D2{dul[q], duh[q]}, w_next = D2{dwl[q], dwh[q]};
      const uint64_t eps = gt_d2(a_cur, w_next) ? 1ull : 0ull;
      const D2 beta = sub_d2(sub_d2(w_cur, a_prev, 0, M), zero, eps, M);
      const D2 a_next = sub_d2(sub_d2(u_next, beta, 0, M), zero, delta, M);
      const uint64_t dnext = carry_d2(beta, a_next, delta, M);
      po[0] = a_cur.lo;
      po[1] = a_cur.hi;
      po[2] = beta.lo;
      po[3] = beta.hi;
      po += pdir;
      a_prev = a_cur;
      a_cur = a_next;
      delta = dnext;
      w_cur = w_next;
    }
    if (steps < len) {
      const D2 beta = sub_d2(w_cur, a_prev, 0, M);
      po[0] = a_cur.lo;
      po[1] = a_cur.hi;
      po[2] = beta.lo;
      po[3] = beta.hi;
    }
  }
  __syncthreads();
  // coefficients alpha + 2^M beta out, minus K: a thread per coefficient
  uint64_t *h = a.h;
  for (int jj = tid; jj < (int)(jhi - j0); jj += kRT) {
    const int i = jj >> lc, p = jj & (int)(chain - 1);
    const uint64_t *v = so + 4 * (((int64_t)p << lp) + i);
    write_h2(h + (R.kbase + R.kstride * (j0 + jj)) * ol, ol, D2{v[0], v[1]}, D2{v[2], v[3]}, M,
             kb);
  }
}

// 64 <= M <= 127 with chains too long to stage: one thread per chain, the
// digits read from global memory, eight steps' worth at a time
template <class Src>
__global__ void __launch_bounds__(128) recover_kernel2(Src src) {
  pdl_enter();
  int64_t local;
  const RecoverArgs &a = src.locate(blockIdx.x, local);
  uint64_t *h = a.h;
  const int ol = a.ol, kb = a.kb;
  int *status = a.status;
  int64_t gid = local * 128 + threadIdx.x;
  int r;
  if (!chain_index(a, gid, r)) return;
  const RecoverRun &R = a.run[r];
  const int M = a.M;
  const int64_t n = R.n, nwords = a.nwords;
  const ChainLane L = chain_lane(a, R, gid);
  auto DU = [&](int64_t t) { return load_d2(L.A, nwords, L.offA + (L.pA + t) * (int64_t)M, M); };
  auto DW = [&](int64_t t) { return load_d2(L.B, nwords, L.offB + (L.pB - t) * (int64_t)M, M); };
  const D2 zero = {0ull, 0ull};
  D2 a_prev, a_cur;
  uint64_t delta;
  if (!L.seeded) {
    a_prev = zero;
    a_cur = DU(0);
    delta = 0;
  } else {
    uint32_t s0[kAccSeedWords], s1[kAccSeedWords];
    seed_value(a, L.vprev, s0);
    seed_value(a, L.vcur, s1);
    a_prev = load_d2(s0, kAccSeedWords, 0, M);
    const D2 b_prev = load_d2(s0, kAccSeedWords, M, M);
    a_cur = load_d2(s1, kAccSeedWords, 0, M);
    const D2 us = DU(0);
    const D2 dprev = sub_d2(sub_d2(us, b_prev, 0, M), a_cur, 0, M);
    if (dprev.hi != 0 || dprev.lo > 1) atomicCAS(status, 0, 2);
    delta = carry_d2(b_prev, a_cur, dprev.lo & 1ull, M);
  }
  D2 w_cur = DW(0);
  const int64_t last = n - 1 - L.pA;
  // the digits of eight steps are loaded together, ahead of their steps
  constexpr int kAhead2 = 8;
  for (int64_t t0 = 0; t0 < L.len; t0 += kAhead2) {
    D2 un[kAhead2], wn[kAhead2];
#pragma unroll
    for (int q = 0; q < kAhead2; q++) {
      const int64_t t = t0 + q;
      if (t < L.len && t != last) {
        wn[q] = DW(t + 1);
        un[q] = DU(t + 1);
      }
    }
#pragma unroll
    for (int q = 0; q < kAhead2; q++) {
      const int64_t t = t0 + q;
      if (t >= L.len) break;
      uint64_t *out = h + (R.kbase + R.kstride * lane_coeff(L, t)) * ol;
      if (t != last) {
        const D2 w_next = wn[q];
        const uint64_t eps = gt_d2(a_cur, w_next) ? 1ull : 0ull;
        const D2 beta = sub_d2(sub_d2(w_cur, a_prev, 0, M), zero, eps, M);
        const D2 a_next = sub_d2(sub_d2(un[q], beta, 0, M), zero, delta, M);
        const uint64_t dnext = carry_d2(beta, a_next, delta, M);
        write_h2(out, ol, a_cur, beta, M, kb);
        a_prev = a_cur;
        a_cur = a_next;
        delta = dnext;
        w_cur = w_next;
      } else {
        write_h2(out, ol, a_cur, sub_d2(w_cur, a_prev, 0, M), M, kb);
      }
    }
  }
}

// ---- wide digits (M >= 128): one warp per chain
// A digit of W = ceil(M / 32) words is spread over the warp: lane l holds
// words l, l + 32, l + 64 (row k = word / 32; KR rows, a compile-time count).
// Each multiword subtraction is a carry-lookahead over the warp: lane i
// generates a borrow (x_i < y_i) or propagates one (x_i = y_i); with G, P the
// ballots of those and A = G | P, the sum G + A + b_in carries exactly where a
// borrow runs, so bit i of (G + A + b_in) ^ A ^ G is the borrow into word i
// and bit 32 the borrow out of the row (the next row's borrow in).
// (at most 3 rows: W <= 96, M <= 3072)
constexpr int kWarpChains = 4;  // chains (warps) per CTA
constexpr unsigned kFull = 0xffffffffu;

template <int KR>
struct WD {
  uint32_t w[KR];
};
// bits [pos, pos + 32) of a word array, words outside [0, n) read as zero
__device__ __forceinline__ uint32_t bits32(const uint32_t *V, int64_t n, int64_t pos) {
  const int64_t wi = pos >> 5;
  const int sh = (int)(pos & 31);
  const uint32_t lo = (wi >= 0 && wi < n) ? __ldg(V + wi) : 0u;
  const uint32_t hi = (wi + 1 >= 0 && wi + 1 < n) ? __ldg(V + wi + 1) : 0u;
  return sh ? (lo >> sh) | (hi << (32 - sh)) : lo;
}
// the M-bit digit at bit pos of V, this lane's words
template <int KR>
__device__ __forceinline__ void wd_load(WD<KR> &x, const uint32_t *V, int64_t n, int64_t pos,
                                        int W, uint32_t topmask, int lane) {
#pragma unroll
  for (int k = 0; k < KR; k++) {
    const int i = lane + 32 * k;
    uint32_t v = i < W ? bits32(V, n, pos + 32 * i) : 0u;
    x.w[k] = i == W - 1 ? v & topmask : v;
  }
}
// d = (x - y - bin) mod 2^M; returns the borrow out (x, y < 2^M: the borrow
// out of the top row is the borrow out of bit M)
template <int KR>
__device__ __forceinline__ uint32_t wd_sub(WD<KR> &d, const WD<KR> &x, const WD<KR> &y,
                                           uint32_t bin, int W, uint32_t topmask, int lane) {
  uint32_t b = bin;
#pragma unroll
  for (int k = 0; k < KR; k++) {
    const int i = lane + 32 * k;
    const bool valid = i < W;
    const uint32_t xv = x.w[k], yv = y.w[k];
    const uint32_t G = __ballot_sync(kFull, valid && xv < yv);
    const uint32_t P = __ballot_sync(kFull, !valid || xv == yv);
    const uint64_t A = G | P;
    const uint64_t S = (uint64_t)G + A + b;
    const uint32_t v = xv - yv - (((uint32_t)(S ^ A ^ G) >> lane) & 1u);
    d.w[k] = !valid ? 0u : (i == W - 1 ? v & topmask : v);
    b = (uint32_t)(S >> 32) & 1u;
  }
  return b;
}
// the borrow out of x - y (x < y), without the difference
template <int KR>
__device__ __forceinline__ uint32_t wd_less(const WD<KR> &x, const WD<KR> &y, int W, int lane) {
  uint32_t b = 0;
#pragma unroll
  for (int k = 0; k < KR; k++) {
    const int i = lane + 32 * k;
    const bool valid = i < W;
    const uint32_t G = __ballot_sync(kFull, valid && x.w[k] < y.w[k]);
    const uint32_t P = __ballot_sync(kFull, !valid || x.w[k] == y.w[k]);
    const uint64_t A = G | P;
    b = (uint32_t)(((uint64_t)G + A + b) >> 32) & 1u;
  }
  return b;
}
// bits [bit, bit + M) of seed value v, this lane's words
template <int KR>
__device__ __forceinline__ void wd_seed(WD<KR> &x, const RecoverArgs &a, int64_t v, int bit,
                                        int W, uint32_t topmask, int lane) {
  if (a.seed_acc != nullptr) {
    uint32_t s[kAccSeedWords];
    seed_value(a, v, s);
#pragma unroll
    for (int k = 0; k < KR; k++) {
      const int i = lane + 32 * k;
      uint32_t r = 0;
      if (i < W) {
        const int pos = bit + 32 * i, wi = pos >> 5, sh = pos & 31;
        uint32_t lo = 0, hi = 0;
#pragma unroll
        for (int j = 0; j < kAccSeedWords; j++) {
          lo = j == wi ? s[j] : lo;
          hi = j == wi + 1 ? s[j] : hi;
        }
        r = sh ? (lo >> sh) | (hi << (32 - sh)) : lo;
        if (i == W - 1) r &= topmask;
      }
      x.w[k] = r;
    }
  } else {
    wd_load(x, a.seeds + v * a.seed_words, a.seed_words, bit, W, topmask, lane);
  }
}
// out limbs (ol of them) of alpha + 2^M beta - K for the steps q < nq of a
// group, from their words in this warp's shared memory (al, be: 32 KR words
// per step); step q's limbs at out + q cstep
template <int KR>
__device__ __forceinline__ void wd_write_group(uint64_t *out, int64_t cstep, int nq, int ol,
                                               const uint32_t *al, const uint32_t *be, int M,
                                               int W, int kb, int lane) {
  const int ow = 2 * ol;  // 32-bit output words
  for (int q = 0; q < nq; q++) {
    const uint32_t *A = al + q * 32 * KR, *B = be + q * 32 * KR;
    uint32_t *o = reinterpret_cast<uint32_t *>(out + q * cstep);
    // the value's words, then - K (a one-bit subtrahend) by the same lookahead
    uint32_t b = 0;
    for (int k = 0; 32 * k < ow; k++) {
      const int i = lane + 32 * k;
      uint32_t v = 0;
      if (i < ow) {
        if (i < W) v = A[i];
        const int qb = 32 * i - M;  // beta's bits [qb, qb + 32)
        if (qb > -32) {
          const int wi = qb >= 0 ? qb >> 5 : -1, sh = qb & 31;
          const uint32_t lo = (wi >= 0 && wi < W) ? B[wi] : 0u;
          const uint32_t hi = (wi + 1 >= 0 && wi + 1 < W) ? B[wi + 1] : 0u;
          v |= qb >= 0 ? (sh ? (lo >> sh) | (hi << (32 - sh)) : lo) : (hi << (32 - sh));
        }
      }
      if (kb >= 0) {
        const uint32_t kv = (i == (kb >> 5)) ? 1u << (kb & 31) : 0u;
        const bool valid = i < ow;
        const uint32_t G = __ballot_sync(kFull, valid && v < kv);
        const uint32_t P = __ballot_sync(kFull, !valid || v == kv);
        const uint64_t Aa = G | P;
        const uint64_t S = (uint64_t)G + Aa + b;
        v = v - kv - (((uint32_t)(S ^ Aa ^ G) >> lane) & 1u);
        b = (uint32_t)(S >> 32) & 1u;
      }
      if (i < ow) o[i] = v;
    }
  }
}

// M >= 128: a warp per chain, digits of KR rows of 32 words.  The digits of a
// group of kAhead steps are loaded together, ahead of their steps; the steps
// keep only the recurrence (and their alpha, beta words in shared memory), and
// the group's coefficients are written after it.
template <int KR, class Src>
__global__ void __launch_bounds__(32 * kWarpChains) recover_warp(Src src) {
  pdl_enter();
  constexpr int kAhead = KR == 1 ? 8 : 4;
  __shared__ uint32_t wbuf[kWarpChains][2 * kAhead * 32 * KR];
  int64_t local;
  const RecoverArgs &a = src.locate(blockIdx.x, local);
  const int lane = threadIdx.x & 31, wq = threadIdx.x >> 5;
  uint64_t *h = a.h;
  const int ol = a.ol, kb = a.kb;
  int *status = a.status;
  int64_t gid = local * kWarpChains + wq;
  int r;
  if (!chain_index(a, gid, r)) return;  // warp-uniform
  const RecoverRun &R = a.run[r];
  const int M = a.M;
  const int W = (M + 31) >> 5;
  const uint32_t topmask = (M & 31) ? (1u << (M & 31)) - 1u : 0xffffffffu;
  const int64_t n = R.n, nwords = a.nwords;
  const ChainLane L = chain_lane(a, R, gid);
  uint32_t *sal = wbuf[wq], *sbe = wbuf[wq] + kAhead * 32 * KR;
  WD<KR> a_prev, a_cur, w_cur, beta, a_next;
  uint32_t delta;
  if (!L.seeded) {
#pragma unroll
    for (int k = 0; k < KR; k++) a_prev.w[k] = 0;
    wd_load(a_cur, L.A, nwords, L.offA + L.pA * (int64_t)M, W, topmask, lane);
    delta = 0;
  } else {
    WD<KR> b_prev, us, t1, dp;
    wd_seed(a_prev, a, L.vprev, 0, W, topmask, lane);
    wd_seed(b_prev, a, L.vprev, M, W, topmask, lane);
    wd_seed(a_cur, a, L.vcur, 0, W, topmask, lane);
    wd_load(us, L.A, nwords, L.offA + L.pA * (int64_t)M, W, topmask, lane);
    // delta_(s-1) = u_s - beta_(s-1) - alpha_s (mod X) is 0 or 1, and the
    // two borrows of that difference add up to delta_s
    const uint32_t b1 = wd_sub(t1, us, b_prev, 0, W, topmask, lane);
    const uint32_t b2 = wd_sub(dp, t1, a_cur, 0, W, topmask, lane);
    bool ok = true;
#pragma unroll
    for (int k = 0; k < KR; k++) ok = ok && (dp.w[k] == 0 || (k == 0 && lane == 0 && dp.w[0] == 1));
    if (!__all_sync(kFull, ok) || b1 + b2 > 1) {
      if (lane == 0) atomicCAS(status, 0, 2);
    }
    delta = b1 + b2;
  }
  wd_load(w_cur, L.B, nwords, L.offB + L.pB * (int64_t)M, W, topmask, lane);
  const int64_t last = n - 1 - L.pA;
  // bit positions of step t's next digits: DU(t + 1), DW(t + 1)
  int64_t pu = L.offA + (L.pA + 1) * (int64_t)M, pw = L.offB + (L.pB - 1) * (int64_t)M;
  const int64_t cstep = (L.up ? 1 : -1) * R.kstride * ol;  // output limbs between steps
  uint64_t *out = h + (R.kbase + R.kstride * lane_coeff(L, 0)) * ol;
  for (int64_t t0 = 0; t0 < L.len; t0 += kAhead) {
    WD<KR> un[kAhead], wn[kAhead];  // DU, DW of steps t0 + 1 .. t0 + kAhead
#pragma unroll
    for (int q = 0; q < kAhead; q++) {
      if (t0 + q < L.len && t0 + q != last) {
        wd_load(wn[q], L.B, nwords, pw - (int64_t)q * M, W, topmask, lane);
        wd_load(un[q], L.A, nwords, pu + (int64_t)q * M, W, topmask, lane);
      }
    }
    pu += (int64_t)kAhead * M;
    pw -= (int64_t)kAhead * M;
    int nq = 0;
#pragma unroll
    for (int q = 0; q < kAhead; q++) {
      const int64_t t = t0 + q;
      if (t >= L.len) break;
      if (t != last) {
        const uint32_t eps = wd_less(wn[q], a_cur, W, lane);  // alpha_j > w_(j+1)
        wd_sub(beta, w_cur, a_prev, eps, W, topmask, lane);
        const uint32_t dnext = wd_sub(a_next, un[q], beta, delta, W, topmask, lane);
#pragma unroll
        for (int k = 0; k < KR; k++) {
          sal[q * 32 * KR + lane + 32 * k] = a_cur.w[k];
          sbe[q * 32 * KR + lane + 32 * k] = beta.w[k];
        }
        a_prev = a_cur;
        a_cur = a_next;
        delta = dnext;
        w_cur = wn[q];
      } else {
        wd_sub(beta, w_cur, a_prev, 0, W, topmask, lane);
#pragma unroll
        for (int k = 0; k < KR; k++) {
          sal[q * 32 * KR + lane + 32 * k] = a_cur.w[k];
          sbe[q * 32 * KR + lane + 32 * k] = beta.w[k];
        }
      }
      nq = q + 1;
    }
    __syncwarp();
    wd_write_group<KR>(out, cstep, nq, ol, sal, sbe, M, W, kb, lane);
    __syncwarp();
    out += kAhead * cstep;
  }
}

int make_recover_args(uint64_t *h, int ol, int kb, const RecoverRun *runs, int nruns,
                      int64_t nwords, int M, int64_t chain, int C,
                      const unsigned long long *seed_acc, const uint32_t *seeds,
                      int seed_words, int *status, RecoverArgs &a, int64_t &blocks) {
  a = RecoverArgs{};
  int64_t total = 0;
  for (int r = 0; r < nruns; r++) {
    a.run[r] = runs[r];
    total += runs[r].nchains;
  }
  a.nruns = nruns;
  a.nwords = nwords;
  a.M = M;
  a.chain = chain;
  a.h = h;
  a.ol = ol;
  a.kb = kb;
  a.status = status;
  a.C = C;
  a.seed_acc = seed_acc;
  a.seeds = seeds;
  a.seed_words = seed_words;
  if ((M + 31) / 32 > kMaxDigitWordsM) return -1;
  if (M <= 63) {  // staged: CTAs of cpc chains that do not straddle runs
    // fewer chains per CTA (down to 8) until there are two CTAs per SM: the
    // staging, digit extraction and output of a CTA then go faster
    int cpc = recover_cpc(chain);
    while (cpc > 8 && (total + cpc - 1) / cpc < 2 * 152) cpc >>= 1;
    a.cpc = cpc;
    blocks = 0;
    for (int r = 0; r < nruns; r++) {
      a.rblocks[r] = (runs[r].nchains + cpc - 1) / cpc;
      blocks += a.rblocks[r];
    }
    const int64_t bytes = staged_bytes(chain, M, cpc);
    if (bytes > 200 * 1024 || ol > 2) return -1;
    a.smem = (int)bytes;
    return 0;
  }
  if (M <= 127 && staged2_bytes(chain, M, 1) <= 200 * 1024) {
    // staged, two-limb digits: the same division into CTAs
    int cpc = recover_cpc(chain);
    if (cpc > kRC2max) cpc = kRC2max;
    while (cpc > 8 && (total + cpc - 1) / cpc < 2 * 152) cpc >>= 1;
    a.cpc = cpc;
    blocks = 0;
    for (int r = 0; r < nruns; r++) {
      a.rblocks[r] = (runs[r].nchains + cpc - 1) / cpc;
      blocks += a.rblocks[r];
    }
    const int64_t bytes = staged2_bytes(chain, M, cpc);
    if (bytes > 200 * 1024 || ol > 5) return -1;
    a.smem = (int)bytes;
    return 0;
  }
  if (M <= 127) {  // chains too long to stage: a thread per chain
    blocks = (total + 127) / 128;
    return 0;
  }
  blocks = (total + kWarpChains - 1) / kWarpChains;  // a warp per chain
  return 0;
}

// 1: M <= 63 (staged), 2: M <= 127 (staged, two limbs), 3-5: wider, by rows
// of 32 words (1-3), 6: M <= 127 with chains too long to stage
int recover_class(int M, int64_t chain) {
  if (M <= 63) return 1;
  if (M <= 127) return staged2_bytes(chain, M, 1) <= 200 * 1024 ? 2 : 6;
  return 2 + (((M + 31) / 32 + 31) / 32);
}

// the staged kernels' shared memory may pass the default 48 KB: opt in
// (once per device and kernel, to the largest size asked so far)
template <class Src, int D>
static cudaError_t staged_attr(int smem) {
  static int done[64] = {0};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  if (smem > 48 * 1024 && smem > done[dev]) {
    e = cudaFuncSetAttribute(D == 1 ? recover_staged1<Src> : recover_staged2<Src>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    done[dev] = smem;
  }
  return cudaSuccess;
}

template <class Src>
static cudaError_t launch_recover_class(int cls, int64_t blocks, const Src &src, int smem,
                                        cudaStream_t s) {
  if (cls == 1) {
    const cudaError_t e = staged_attr<Src, 1>(smem);
    if (e != cudaSuccess) return e;
    (void)launch_k(recover_staged1<Src>, dim3((unsigned)blocks), dim3(kRT), smem, s, src);
  } else if (cls == 2) {
    const cudaError_t e = staged_attr<Src, 2>(smem);
    if (e != cudaSuccess) return e;
    (void)launch_k(recover_staged2<Src>, dim3((unsigned)blocks), dim3(kRT), smem, s, src);
  }
  else if (cls == 3)
    (void)launch_k(recover_warp<1, Src>, dim3((unsigned)blocks), dim3(32 * kWarpChains), 0, s, src);
  else if (cls == 4)
    (void)launch_k(recover_warp<2, Src>, dim3((unsigned)blocks), dim3(32 * kWarpChains), 0, s, src);
  else if (cls == 5)
    (void)launch_k(recover_warp<3, Src>, dim3((unsigned)blocks), dim3(32 * kWarpChains), 0, s, src);
  else
    (void)launch_k(recover_kernel2<Src>, dim3((unsigned)blocks), dim3(128), 0, s, src);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_recover(const RecoverArgs &a, int64_t blocks, cudaStream_t s) {
  if (blocks == 0) return cudaSuccess;
  return launch_recover_class(recover_class(a.M, a.chain), blocks, One<RecoverArgs>{a}, a.smem, s);
}

cudaError_t launch_recover_batch(int cls, const RecoverArgs *d, const int64_t *prefix, int n,
                                 int64_t blocks, int smem, cudaStream_t s) {
  if (n == 0 || blocks == 0) return cudaSuccess;
  return launch_recover_class(cls, blocks, Many<RecoverArgs>{d, prefix, n}, smem, s);
}

// ------------------------------------------------------------------ mod p
// r = (hi * 2^64 + lo) mod p for hi < p < 2^63, by shift-and-subtract.
__device__ __forceinline__ uint64_t mod_128(uint64_t hi, uint64_t lo, uint64_t p) {
  for (int i = 0; i < 64; i++) {
    hi = (hi << 1) | (lo >> 63);
    lo <<= 1;
    if (hi >= p) hi -= p;
  }
  return hi;
}

__global__ void __launch_bounds__(256) reduce_mod_kernel(uint64_t *out, const uint64_t *h, int ol,
                                                         int64_t lh, uint64_t p) {
  pdl_enter();
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < lh;
       k += (int64_t)gridDim.x * blockDim.x) {
    uint64_t r = 0;
    for (int l = ol - 1; l >= 0; l--) r = mod_128(r, h[k * ol + l], p);
    out[k] = r;
  }
}

cudaError_t launch_reduce_mod(uint64_t *out, const uint64_t *h, int ol, int64_t lh, uint64_t p,
                              cudaStream_t s) {
  (void)launch_k(reduce_mod_kernel, dim3(grid_for(lh, 256)), dim3(256), 0, s, out, h, ol, lh, p);
  note_launches(1);
  return cudaGetLastError();
}

}  // namespace ks
