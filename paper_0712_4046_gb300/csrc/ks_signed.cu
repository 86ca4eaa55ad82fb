// Signed coefficients (the paper treats non-negative ones, Sec. 3): every
// variant runs on the biased values f'_t = f_t + c, g'_t = g_t + c with
// c = 2^(b-1), which lie in [0, 2^b).  Since f = f' - c U_f and g = g' - c U_g
// (U the all-ones polynomials),
//
//   f g = f' g' - c (f * U_g + U_f * g) - c^2 U_f * U_g,
//
// (f * U_g)_k = sum of f_t over t in [max(0, k - Lg + 1), min(k, Lf - 1)] and
// (U_f * U_g)_k = number of such t.  The window sums are differences of prefix
// sums.  A signed coefficient is its low in_limbs limbs read unsigned, minus
// 2^(64 in_limbs) when negative, so each prefix sum is kept per limb as an
// exact 128-bit sum, plus the count of negative coefficients -- no carries
// cross coefficients.  The correction itself is computed mod 2^(64 ol),
// which is exact because the final coefficient fits ol limbs.
//
// Prefix sums: for polynomials of up to 2^16 coefficients a single launch in
// which each CTA also sums the blocks before its own; longer ones use a
// three-phase scan (block totals, scan of the totals, apply).
#include "ks_internal.cuh"
#include "ks_src.cuh"

namespace ks {

namespace {
constexpr int kThreads = 256;
constexpr int kElems = 8;
constexpr int kBlock = kThreads * kElems;
constexpr int kMaxIn = 32;   // in_limbs <= 32 (b <= 2048)
constexpr int kMaxOl = 72;

struct U2 {
  uint64_t lo, hi;
};
__device__ __forceinline__ U2 add2(U2 a, U2 b) {
  U2 r;
  r.lo = a.lo + b.lo;
  r.hi = a.hi + b.hi + (r.lo < a.lo ? 1ull : 0ull);
  return r;
}
__device__ __forceinline__ U2 sub2(U2 a, U2 b) {
  U2 r;
  r.lo = a.lo - b.lo;
  r.hi = a.hi - b.hi - (a.lo < b.lo ? 1ull : 0ull);
  return r;
}


// (block, polynomial) of this CTA
__device__ __forceinline__ int which(const PrefArgs &a, int64_t &blk) {
  if (blk < a.nblocks[0]) return 0;
  blk -= a.nblocks[0];
  return 1;
}

__device__ __forceinline__ U2 warp_incl(U2 v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    U2 o;
    o.lo = __shfl_up_sync(0xffffffffu, v.lo, off);
    o.hi = __shfl_up_sync(0xffffffffu, v.hi, off);
    if (lane >= off) v = add2(v, o);
  }
  return v;
}

// exclusive prefix over the block (thread order) and the block total
__device__ U2 block_excl(U2 v, U2 *total) {
  __shared__ U2 wt[kThreads / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  const U2 incl = warp_incl(v);
  if (lane == 31) wt[wid] = incl;
  __syncthreads();
  U2 pre = {0, 0}, tot = {0, 0};
  for (int w = 0; w < kThreads / 32; w++) {
    if (w < wid) pre = add2(pre, wt[w]);
    tot = add2(tot, wt[w]);
  }
  *total = tot;
  return add2(pre, sub2(incl, v));
}
}  // namespace

__global__ void __launch_bounds__(kThreads) pref_block_totals(PrefArgs a) {
  int64_t blk = blockIdx.x;
  const int q = which(a, blk);
  const int64_t t0 = blk * kBlock + (int64_t)threadIdx.x * kElems;
  const int il = a.il, rec = 2 * il + 1;
  uint64_t *out = a.bt + (int64_t)blockIdx.x * rec;
  for (int l = 0; l <= il; l++) {
    U2 v = {0, 0};
    for (int e = 0; e < kElems; e++) {
      const int64_t t = t0 + e;
      if (t >= a.L[q]) break;
      const uint64_t *c = a.x[q] + t * il;
      const uint64_t w = l < il ? c[l] : (c[il - 1] >> 63);
      v = add2(v, U2{w, 0});
    }
    U2 tot;
    block_excl(v, &tot);
    if (threadIdx.x == 0) {
      if (l < il) {
        out[2 * l] = tot.lo;
        out[2 * l + 1] = tot.hi;
      } else {
        out[2 * il] = tot.lo;
      }
    }
  }
}

// one thread per (polynomial, limb field): exclusive scan of the block totals
__global__ void pref_scan_totals(PrefArgs a) {
  const int il = a.il, rec = 2 * il + 1;
  const int q = blockIdx.x;
  const int64_t base = q == 0 ? 0 : a.nblocks[0];
  for (int l = threadIdx.x; l <= il; l += blockDim.x) {
    U2 run = {0, 0};
    for (int64_t bb = 0; bb < a.nblocks[q]; bb++) {
      uint64_t *r = a.bt + (base + bb) * rec;
      U2 v;
      if (l < il) {
        v = U2{r[2 * l], r[2 * l + 1]};
        r[2 * l] = run.lo;
        r[2 * l + 1] = run.hi;
      } else {
        v = U2{r[2 * il], 0};
        r[2 * il] = run.lo;
      }
      run = add2(run, v);
    }
  }
}

__global__ void __launch_bounds__(kThreads) pref_apply(PrefArgs a) {
  int64_t blk = blockIdx.x;
  const int q = which(a, blk);
  const int64_t t0 = blk * kBlock + (int64_t)threadIdx.x * kElems;
  const int il = a.il, rec = 2 * il + 1;
  const uint64_t *boff = a.bt + (int64_t)blockIdx.x * rec;
  for (int l = 0; l <= il; l++) {
    U2 mine = {0, 0};
    for (int e = 0; e < kElems; e++) {
      const int64_t t = t0 + e;
      if (t >= a.L[q]) break;
      const uint64_t *c = a.x[q] + t * il;
      mine = add2(mine, U2{l < il ? c[l] : (c[il - 1] >> 63), 0});
    }
    U2 tot;
    U2 run = block_excl(mine, &tot);
    run = add2(run, l < il ? U2{boff[2 * l], boff[2 * l + 1]} : U2{boff[2 * il], 0});
    for (int e = 0; e < kElems; e++) {
      const int64_t t = t0 + e;
      if (t >= a.L[q]) break;
      const uint64_t *c = a.x[q] + t * il;
      run = add2(run, U2{l < il ? c[l] : (c[il - 1] >> 63), 0});
      uint64_t *P = a.P[q] + t * rec;
      if (l < il) {
        P[2 * l] = run.lo;
        P[2 * l + 1] = run.hi;
      } else {
        P[2 * il] = run.lo;
      }
    }
  }
}

// Polynomials of up to kSmallL coefficients: a single launch.  Each CTA
// first sums every coefficient before its block (redundant across CTAs, at
// most kSmallL / 2 extra reads per CTA), then scans its own block.
constexpr int64_t kSmallL = 1 << 16;

template <class Src>
__global__ void __launch_bounds__(kThreads) pref_single(Src src) {
  int64_t blk;
  const PrefArgs &a = src.locate(blockIdx.x, blk);
  const int q = which(a, blk);
  const int64_t b0 = blk * kBlock;
  const int64_t t0 = b0 + (int64_t)threadIdx.x * kElems;
  const int il = a.il, rec = 2 * il + 1;
  for (int l = 0; l <= il; l++) {
    // sum of the preceding blocks (four independent partial sums per thread)
    U2 bp[4] = {{0, 0}, {0, 0}, {0, 0}, {0, 0}};
    int64_t t = threadIdx.x;
    for (; t + 3 * kThreads < b0; t += 4 * kThreads) {
#pragma unroll
      for (int u = 0; u < 4; u++) {
        const uint64_t *c = a.x[q] + (t + u * kThreads) * il;
        bp[u] = add2(bp[u], U2{l < il ? c[l] : (c[il - 1] >> 63), 0});
      }
    }
    for (; t < b0; t += kThreads) {
      const uint64_t *c = a.x[q] + t * il;
      bp[0] = add2(bp[0], U2{l < il ? c[l] : (c[il - 1] >> 63), 0});
    }
    const U2 before = add2(add2(bp[0], bp[1]), add2(bp[2], bp[3]));
    U2 tot_before;
    block_excl(before, &tot_before);
    U2 mine = {0, 0};
    for (int e = 0; e < kElems; e++) {
      const int64_t t = t0 + e;
      if (t >= a.L[q]) break;
      const uint64_t *c = a.x[q] + t * il;
      mine = add2(mine, U2{l < il ? c[l] : (c[il - 1] >> 63), 0});
    }
    U2 tot;
    U2 run = add2(block_excl(mine, &tot), tot_before);
    for (int e = 0; e < kElems; e++) {
      const int64_t t = t0 + e;
      if (t >= a.L[q]) break;
      const uint64_t *c = a.x[q] + t * il;
      run = add2(run, U2{l < il ? c[l] : (c[il - 1] >> 63), 0});
      uint64_t *P = a.P[q] + t * rec;
      if (l < il) {
        P[2 * l] = run.lo;
        P[2 * l + 1] = run.hi;
      } else {
        P[2 * il] = run.lo;
      }
    }
  }
}

// acc (ol limbs, mod 2^(64 ol)) += sign * (window sum of x over [lo, hi]),
// from the per-limb prefix records.
__device__ __forceinline__ void add_window(uint64_t *acc, int ol, const uint64_t *P, int il,
                                           int64_t lo, int64_t hi) {
  const int rec = 2 * il + 1;
  const uint64_t *A = P + hi * rec;
  const uint64_t *B = lo > 0 ? P + (lo - 1) * rec : nullptr;
  // sum over limbs l of D_l 2^(64 l), D_l = S_l(hi) - S_l(lo - 1) (exact, 128-bit)
  uint64_t carry = 0;
  uint64_t pending_hi = 0;
  for (int l = 0; l < ol; l++) {
    uint64_t add = pending_hi;
    pending_hi = 0;
    uint64_t d_lo = 0;
    if (l < il) {
      U2 d = U2{A[2 * l], A[2 * l + 1]};
      if (B) d = sub2(d, U2{B[2 * l], B[2 * l + 1]});
      d_lo = d.lo;
      pending_hi = d.hi;
    }
    // acc[l] += add + d_lo + carry
    uint64_t s1 = acc[l] + add;
    uint64_t c1 = s1 < add;
    uint64_t s2 = s1 + d_lo;
    uint64_t c2 = s2 < d_lo;
    uint64_t s3 = s2 + carry;
    uint64_t c3 = s3 < carry;
    acc[l] = s3;
    carry = c1 + c2 + c3;
  }
  // minus 2^(64 il) times the number of negative coefficients in the window
  uint64_t neg = A[2 * il] - (B ? B[2 * il] : 0ull);
  uint64_t borrow = 0;
  for (int l = il; l < ol; l++) {
    const uint64_t v = (l == il) ? neg : 0ull;
    const uint64_t d1 = acc[l] - v;
    const uint64_t b1 = acc[l] < v;
    const uint64_t d2 = d1 - borrow;
    const uint64_t b2 = d1 < borrow;
    acc[l] = d2;
    borrow = b1 | b2;
  }
}

// r -= x << sh  (mod 2^(64 ol))
__device__ __forceinline__ void sub_shifted(uint64_t *r, const uint64_t *x, int ol, int sh) {
  const int q = sh >> 6, rr = sh & 63;
  uint64_t borrow = 0;
  for (int l = 0; l < ol; l++) {
    const int a = l - q;
    uint64_t v = 0;
    if (a >= 0 && a < ol) v = x[a] << rr;
    if (rr && a - 1 >= 0 && a - 1 < ol) v |= x[a - 1] >> (64 - rr);
    const uint64_t d1 = r[l] - v;
    const uint64_t b1 = r[l] < v;
    const uint64_t d2 = d1 - borrow;
    const uint64_t b2 = d1 < borrow;
    r[l] = d2;
    borrow = b1 | b2;
  }
}

template <class Src>
__global__ void __launch_bounds__(128) signed_fix_kernel(Src src) {
  int64_t local;
  const FixArgs &fa = src.locate(blockIdx.x, local);
  uint64_t *h = fa.h;
  const int ol = fa.ol, b = fa.b, il = fa.il;
  const int64_t lf = fa.lf, lg = fa.lg;
  const uint64_t *pf = fa.pf, *pg = fa.pg;
  const int64_t lh = lf + lg - 1;
  {
    const int64_t k = local * 128 + threadIdx.x;
    if (k >= lh) return;
    uint64_t w[kMaxOl];
    for (int l = 0; l < ol; l++) w[l] = 0;
    const int64_t fhi = k < lf - 1 ? k : lf - 1;
    const int64_t flo = k - lg + 1 > 0 ? k - lg + 1 : 0;
    const int64_t ghi = k < lg - 1 ? k : lg - 1;
    const int64_t glo = k - lf + 1 > 0 ? k - lf + 1 : 0;
    add_window(w, ol, pf, il, flo, fhi);  // (f * U_g)_k
    add_window(w, ol, pg, il, glo, ghi);  // (U_f * g)_k
    uint64_t r[kMaxOl];
    uint64_t *hk = h + k * ol;
    for (int l = 0; l < ol; l++) r[l] = hk[l];
    sub_shifted(r, w, ol, b - 1);
    uint64_t cnt[kMaxOl];
    for (int l = 0; l < ol; l++) cnt[l] = 0;
    cnt[0] = (uint64_t)(fhi - flo + 1);
    sub_shifted(r, cnt, ol, 2 * b - 2);
    for (int l = 0; l < ol; l++) hk[l] = r[l];
  }
}

static int64_t nblocks_for(int64_t L) { return (L + kBlock - 1) / kBlock; }

bool make_signed_args(uint64_t *h, int ol, const uint64_t *f, int64_t lf, const uint64_t *g,
                      int64_t lg, int b, int in_limbs, uint64_t *prefix, PrefArgs &a,
                      FixArgs &fx, int64_t &pref_blocks, int64_t &fix_blocks) {
  const int rec = 2 * in_limbs + 1;
  a = PrefArgs{};
  a.x[0] = f;
  a.x[1] = g;
  a.L[0] = lf;
  a.L[1] = lg;
  a.nblocks[0] = nblocks_for(lf);
  a.nblocks[1] = nblocks_for(lg);
  a.il = in_limbs;
  a.P[0] = prefix;
  a.P[1] = prefix + lf * rec;
  a.bt = prefix + (lf + lg) * rec;
  fx = FixArgs{h, ol, lf, lg, b, in_limbs, a.P[0], a.P[1]};
  pref_blocks = a.nblocks[0] + a.nblocks[1];
  fix_blocks = (lf + lg - 1 + 127) / 128;
  return lf <= kSmallL && lg <= kSmallL;  // single-launch prefix possible
}

cudaError_t launch_signed_fix(uint64_t *h, int ol, const uint64_t *f, int64_t lf,
                              const uint64_t *g, int64_t lg, int b, int in_limbs,
                              uint64_t *prefix, cudaStream_t s) {
  if (ol > kMaxOl || in_limbs > kMaxIn) return cudaErrorInvalidValue;
  PrefArgs a;
  FixArgs fx;
  int64_t pb, fb;
  const bool single = make_signed_args(h, ol, f, lf, g, lg, b, in_limbs, prefix, a, fx, pb, fb);
  int launches = 2;
  if (single) {
    pref_single<One<PrefArgs>><<<(unsigned)pb, kThreads, 0, s>>>(One<PrefArgs>{a});
  } else {
    pref_block_totals<<<(unsigned)pb, kThreads, 0, s>>>(a);
    pref_scan_totals<<<2, 64, 0, s>>>(a);
    pref_apply<<<(unsigned)pb, kThreads, 0, s>>>(a);
    launches = 4;
  }
  signed_fix_kernel<One<FixArgs>><<<(unsigned)fb, 128, 0, s>>>(One<FixArgs>{fx});
  note_launches(launches);
  return cudaGetLastError();
}

cudaError_t launch_signed_batch(const PrefArgs *pa, const int64_t *pref_prefix,
                                const FixArgs *fa, const int64_t *fix_prefix, int n,
                                int64_t pref_blocks, int64_t fix_blocks, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  pref_single<Many<PrefArgs>><<<(unsigned)pref_blocks, kThreads, 0, s>>>(
      Many<PrefArgs>{pa, pref_prefix, n});
  signed_fix_kernel<Many<FixArgs>><<<(unsigned)fix_blocks, 128, 0, s>>>(
      Many<FixArgs>{fa, fix_prefix, n});
  note_launches(2);
  return cudaGetLastError();
}

size_t signed_prefix_bytes(int64_t lf, int64_t lg, int il) {
  const int rec = 2 * il + 1;
  return (size_t)(lf + lg + nblocks_for(lf) + nblocks_for(lg)) * rec * 8;
}

}  // namespace ks
