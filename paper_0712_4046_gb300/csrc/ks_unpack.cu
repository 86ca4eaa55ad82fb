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

// digit arithmetic on W 32-bit words, values in [0, 2^M)
struct Dig {
  uint32_t w[kMaxDigitWordsM];
};

__device__ __forceinline__ void dig_load(Dig &x, const uint32_t *V, int64_t nwords, int64_t pos,
                                         int M) {
  const int W = (M + 31) / 32;
  for (int i = 0; i < W; i += 2) {
    const uint64_t v = get_bits64(V, nwords, pos + 32 * (int64_t)i);
    x.w[i] = (uint32_t)v;
    if (i + 1 < W) x.w[i + 1] = (uint32_t)(v >> 32);
  }
  const int top = M - 32 * (W - 1);
  if (top < 32) x.w[W - 1] &= (1u << top) - 1u;
}
__device__ __forceinline__ void dig_load_local(Dig &x, const uint32_t *src, int nsrc, int pos,
                                               int M) {
  const int W = (M + 31) / 32;
  for (int i = 0; i < W; i += 2) {
    const uint64_t v = get_bits64(src, nsrc, pos + 32 * (int64_t)i);
    x.w[i] = (uint32_t)v;
    if (i + 1 < W) x.w[i + 1] = (uint32_t)(v >> 32);
  }
  const int top = M - 32 * (W - 1);
  if (top < 32) x.w[W - 1] &= (1u << top) - 1u;
}
__device__ __forceinline__ bool dig_gt(const Dig &a, const Dig &b, int W) {
  for (int i = W - 1; i >= 0; i--)
    if (a.w[i] != b.w[i]) return a.w[i] > b.w[i];
  return false;
}
// r = (a - b - c) mod 2^M
__device__ __forceinline__ void dig_sub(Dig &r, const Dig &a, const Dig &b, uint32_t c, int M) {
  const int W = (M + 31) / 32;
  int64_t borrow = c;
  for (int i = 0; i < W; i++) {
    const int64_t t = (int64_t)a.w[i] - b.w[i] - borrow;
    r.w[i] = (uint32_t)t;
    borrow = t < 0 ? 1 : 0;
  }
  const int top = M - 32 * (W - 1);
  if (top < 32) r.w[W - 1] &= (1u << top) - 1u;
}
// floor((a + b + c) / 2^M) for a, b < 2^M, c in {0, 1}
__device__ __forceinline__ uint32_t dig_add_carry(const Dig &a, const Dig &b, uint32_t c, int M) {
  const int W = (M + 31) / 32;
  uint64_t carry = c;
  uint32_t topw = 0;
  for (int i = 0; i < W; i++) {
    const uint64_t t = (uint64_t)a.w[i] + b.w[i] + carry;
    topw = (uint32_t)t;
    carry = t >> 32;
  }
  const int top = M - 32 * (W - 1);
  if (top == 32) return (uint32_t)carry;
  return (topw >> top) & 1u;
}
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
  for (int l = 0; l < ol; l++) out[l] = sub_k(l < 5 ? s[l] : 0ull, kb, l, borrow);
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

// 64 <= M <= 127, one thread per chain, digits read from global memory
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
  for (int64_t t = 0; t < L.len; t++) {
    uint64_t *out = h + (R.kbase + R.kstride * lane_coeff(L, t)) * ol;
    if (t != last) {
      const D2 w_next = DW(t + 1);
      const uint64_t eps = gt_d2(a_cur, w_next) ? 1ull : 0ull;
      const D2 beta = sub_d2(sub_d2(w_cur, a_prev, 0, M), zero, eps, M);
      const D2 u_next = DU(t + 1);
      const D2 a_next = sub_d2(sub_d2(u_next, beta, 0, M), zero, delta, M);
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

// out limbs of alpha + 2^M beta - K, alpha, beta < 2^M (any M)
__device__ void write_coeff(uint64_t *out, int ol, const Dig &al, const Dig &be, int M, int kb) {
  const int W = (M + 31) / 32;
  uint64_t borrow = 0;
  for (int l = 0; l < ol; l++) {
    uint64_t v = 0;
    for (int half = 0; half < 2; half++) {
      const int64_t p0 = 64 * (int64_t)l + 32 * half;  // bit position of this 32-bit chunk
      uint64_t chunk = 0;
      if (p0 < M) chunk |= al.w[(int)(p0 >> 5)];  // alpha's bits above M are zero
      // from beta: bits [p0 - M, p0 - M + 32)
      const int64_t q = p0 - M;
      if (q + 32 > 0 && q < (int64_t)32 * W) {
        const int64_t wi = q >= 0 ? (q >> 5) : -1;
        const int sh = (int)(q & 31);
        const uint64_t lo = (wi >= 0 && wi < W) ? be.w[wi] : 0u;
        const uint64_t hi = (wi + 1 >= 0 && wi + 1 < W) ? be.w[wi + 1] : 0u;
        const uint64_t pair = lo | (hi << 32);
        uint32_t part;
        if (q >= 0)
          part = (uint32_t)(pair >> sh);
        else
          part = (uint32_t)(((uint64_t)be.w[0]) << (int)(-q));  // -q < 32
        chunk |= part;
      }
      v |= (chunk & 0xffffffffull) << (32 * half);
    }
    out[l] = sub_k(v, kb, l, borrow);
  }
}

// any M (digits of W 32-bit words), one thread per chain
template <class Src>
__global__ void __launch_bounds__(64) recover_wide(Src src) {
  pdl_enter();
  int64_t local;
  const RecoverArgs &a = src.locate(blockIdx.x, local);
  uint64_t *h = a.h;
  const int ol = a.ol, kb = a.kb;
  int *status = a.status;
  int64_t gid = local * 64 + threadIdx.x;
  int r;
  if (!chain_index(a, gid, r)) return;
  const RecoverRun &R = a.run[r];
  const int M = a.M;
  const int W = (M + 31) / 32;
  const int64_t n = R.n, nwords = a.nwords;
  const ChainLane L = chain_lane(a, R, gid);
  Dig a_prev, a_cur, w_cur, w_next, u_next, beta, a_next, zero;
  for (int i = 0; i < W; i++) zero.w[i] = 0;
  uint32_t delta;
  if (!L.seeded) {
    a_prev = zero;
    dig_load(a_cur, L.A, nwords, L.offA + L.pA * (int64_t)M, M);
    delta = 0;
  } else {
    Dig b_prev, us, dp;
    if (a.seed_acc != nullptr) {
      uint32_t s0[kAccSeedWords], s1[kAccSeedWords];
      seed_value(a, L.vprev, s0);
      seed_value(a, L.vcur, s1);
      dig_load_local(a_prev, s0, kAccSeedWords, 0, M);
      dig_load_local(b_prev, s0, kAccSeedWords, M, M);
      dig_load_local(a_cur, s1, kAccSeedWords, 0, M);
    } else {
      const uint32_t *sp = a.seeds + L.vprev * a.seed_words;
      const uint32_t *sc = a.seeds + L.vcur * a.seed_words;
      dig_load_local(a_prev, sp, a.seed_words, 0, M);
      dig_load_local(b_prev, sp, a.seed_words, M, M);
      dig_load_local(a_cur, sc, a.seed_words, 0, M);
    }
    dig_load(us, L.A, nwords, L.offA + L.pA * (int64_t)M, M);
    Dig t1;
    dig_sub(t1, us, b_prev, 0, M);
    dig_sub(dp, t1, a_cur, 0, M);
    bool ok = dp.w[0] <= 1;
    for (int i = 1; i < W; i++) ok = ok && dp.w[i] == 0;
    if (!ok) atomicCAS(status, 0, 2);
    delta = dig_add_carry(b_prev, a_cur, dp.w[0] & 1u, M);
  }
  dig_load(w_cur, L.B, nwords, L.offB + L.pB * (int64_t)M, M);
  const int64_t last = n - 1 - L.pA;
  for (int64_t t = 0; t < L.len; t++) {
    uint64_t *out = h + (R.kbase + R.kstride * lane_coeff(L, t)) * ol;
    if (t != last) {
      dig_load(w_next, L.B, nwords, L.offB + (L.pB - t - 1) * (int64_t)M, M);
      const uint32_t eps = dig_gt(a_cur, w_next, W) ? 1u : 0u;
      dig_sub(beta, w_cur, a_prev, eps, M);
      dig_load(u_next, L.A, nwords, L.offA + (L.pA + t + 1) * (int64_t)M, M);
      dig_sub(a_next, u_next, beta, delta, M);
      const uint32_t dnext = dig_add_carry(beta, a_next, delta, M);
      write_coeff(out, ol, a_cur, beta, M, kb);
      a_prev = a_cur;
      a_cur = a_next;
      delta = dnext;
      w_cur = w_next;
    } else {
      dig_sub(beta, w_cur, a_prev, 0, M);
      write_coeff(out, ol, a_cur, beta, M, kb);
    }
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
  const int per = M <= 127 ? 128 : 64;
  blocks = (total + per - 1) / per;
  return 0;
}

int recover_class(int M) { return M <= 63 ? 1 : (M <= 127 ? 2 : 3); }

template <class Src>
static cudaError_t staged_attr(int smem) {
  static int done[64] = {0};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  if (smem > 48 * 1024 && smem > done[dev]) {
    e = cudaFuncSetAttribute(recover_staged1<Src>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             smem);
    if (e != cudaSuccess) return e;
    done[dev] = smem;
  }
  return cudaSuccess;
}

template <class Src>
static cudaError_t launch_recover_class(int cls, int64_t blocks, const Src &src, int smem,
                                        cudaStream_t s) {
  if (cls == 1) {
    const cudaError_t e = staged_attr<Src>(smem);
    if (e != cudaSuccess) return e;
    (void)launch_k(recover_staged1<Src>, dim3((unsigned)blocks), dim3(kRT), smem, s, src);
  } else if (cls == 2)
    (void)launch_k(recover_kernel2<Src>, dim3((unsigned)blocks), dim3(128), 0, s, src);
  else
    (void)launch_k(recover_wide<Src>, dim3((unsigned)blocks), dim3(64), 0, s, src);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_recover(const RecoverArgs &a, int64_t blocks, cudaStream_t s) {
  if (blocks == 0) return cudaSuccess;
  return launch_recover_class(recover_class(a.M), blocks, One<RecoverArgs>{a}, a.smem, s);
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
