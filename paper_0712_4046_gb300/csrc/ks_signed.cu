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
// Prefix records: polynomials of up to 16384 coefficients are scanned in one
// launch of one CTA per 512-coefficient tile; longer ones by a three-phase
// scan (block totals, scan of the totals, apply).  The correction then reads
// four records per output k.
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

// ---------------------------------------------------------------- short polynomials
// Up to kScanL coefficients: one CTA per tile of 512 coefficients.  It sums
// the coefficients of every earlier tile (512 threads, at most 32 independent
// loads each), scans its own tile across the block, and writes the prefix
// records of the tile (coalesced).  No CTA waits on another.
constexpr int kPT = 512;
constexpr int64_t kScanL = (int64_t)kPT * 32;

// field l of coefficient t: limb l (l < il), or 1 when the coefficient is negative (l = il)
__device__ __forceinline__ uint64_t field(const uint64_t *x, int il, int64_t t, int l) {
  const uint64_t *c = x + t * il;
  return l < il ? c[l] : (c[il - 1] >> 63);
}

// inclusive block scan of v and block total of p (kPT threads)
__device__ __forceinline__ void tile_scan(U2 &v, U2 &p, U2 *wsum, U2 *wscan) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    U2 o, r;
    o.lo = __shfl_up_sync(0xffffffffu, v.lo, off);
    o.hi = __shfl_up_sync(0xffffffffu, v.hi, off);
    if (lane >= off) v = add2(v, o);
    r.lo = __shfl_xor_sync(0xffffffffu, p.lo, off);
    r.hi = __shfl_xor_sync(0xffffffffu, p.hi, off);
    p = add2(p, r);
  }
  __syncthreads();
  if (lane == 31) wscan[wid] = v;
  if (lane == 0) wsum[wid] = p;
  __syncthreads();
  U2 base = {0, 0};
#pragma unroll
  for (int w = 0; w < kPT / 32; w++) {
    base = add2(base, wsum[w]);
    if (w < wid) base = add2(base, wscan[w]);
  }
  v = add2(base, v);
}

template <class Src>
__global__ void __launch_bounds__(kPT) pref_tile(Src src) {
  __shared__ U2 wsum[kPT / 32];
  __shared__ U2 wscan[kPT / 32];
  int64_t blk;
  const PrefArgs &a = src.locate(blockIdx.x, blk);
  const int q = blk < a.nblocks[0] ? 0 : 1;
  if (q) blk -= a.nblocks[0];
  const uint64_t *x = q ? a.x[1] : a.x[0];
  const int64_t L = q ? a.L[1] : a.L[0];
  uint64_t *P = q ? a.P[1] : a.P[0];
  const int il = a.il, rec = 2 * il + 1;
  const int tid = threadIdx.x;
  const int64_t t = blk * kPT + tid;
  for (int l = 0; l < il; l++) {
    // element tid of every earlier tile (blk < 32): limb l, and for the top
    // limb also the count of negative coefficients, from the same loads
    U2 p = {0, 0}, pn = {0, 0};
    const bool top = l == il - 1;
    for (int64_t m0 = 0; m0 < blk; m0 += 16) {
      uint64_t v[16];
#pragma unroll
      for (int u = 0; u < 16; u++)
        v[u] = m0 + u < blk ? x[((m0 + u) * kPT + tid) * il + l] : 0ull;
#pragma unroll
      for (int u = 0; u < 16; u++) {
        p = add2(p, U2{v[u], 0});
        pn.lo += v[u] >> 63;
      }
    }
    const uint64_t e = t < L ? x[t * il + l] : 0ull;
    U2 sv = U2{e, 0};
    tile_scan(sv, p, wsum, wscan);
    if (t < L) {
      P[t * rec + 2 * l] = sv.lo;
      P[t * rec + 2 * l + 1] = sv.hi;
    }
    if (top) {
      U2 sn = U2{e >> 63, 0};
      tile_scan(sn, pn, wsum, wscan);
      if (t < L) P[t * rec + 2 * il] = sn.lo;
    }
  }
}

// r -= x << sh (mod 2^(64 ol)), fixed-size arrays
template <int OL>
__device__ __forceinline__ void sub_shifted_fixed(uint64_t (&r)[OL], const uint64_t (&x)[OL],
                                                  int ol, int sh) {
  const int q = sh >> 6, rr = sh & 63;
  uint64_t borrow = 0;
#pragma unroll
  for (int l = 0; l < OL; l++) {
    if (l < ol) {
      uint64_t v = 0;
#pragma unroll
      for (int m = 0; m < OL; m++) {  // limb l of x << sh, with static register indices
        if (m == l - q) v |= x[m] << rr;
        if (rr && m == l - q - 1) v |= x[m] >> (64 - rr);
      }
      const uint64_t d1 = r[l] - v;
      const uint64_t b1 = r[l] < v;
      const uint64_t d2 = d1 - borrow;
      const uint64_t b2 = d1 < borrow;
      r[l] = d2;
      borrow = b1 | b2;
    }
  }
}

// w += sign * (window sum from prefix records A - B, B null for an empty lower part)
template <int IL, int OL>
__device__ __forceinline__ void add_window_fixed(uint64_t (&w)[OL], const uint64_t *A,
                                                 const uint64_t *B, int il) {
#pragma unroll
  for (int l = 0; l < IL; l++) {
    if (l < il) {
      U2 d = U2{A[2 * l], A[2 * l + 1]};
      if (B) d = sub2(d, U2{B[2 * l], B[2 * l + 1]});
      uint64_t carry = 0;
#pragma unroll
      for (int m = 0; m < OL; m++) {
        if (m >= l) {
          const uint64_t add = m == l ? d.lo : (m == l + 1 ? d.hi : 0ull);
          const uint64_t s1 = w[m] + add;
          const uint64_t c1 = s1 < add;
          const uint64_t s2 = s1 + carry;
          const uint64_t c2 = s2 < carry;
          w[m] = s2;
          carry = c1 + c2;
        }
      }
    }
  }
  // minus 2^(64 il) times the count of negative coefficients in the window
  const uint64_t neg = A[2 * il] - (B ? B[2 * il] : 0ull);
  uint64_t borrow = 0;
#pragma unroll
  for (int m = 0; m < OL; m++) {
    if (m >= il) {
      const uint64_t v = m == il ? neg : 0ull;
      const uint64_t d1 = w[m] - v;
      const uint64_t b1 = w[m] < v;
      const uint64_t d2 = d1 - borrow;
      const uint64_t b2 = d1 < borrow;
      w[m] = d2;
      borrow = b1 | b2;
    }
  }
}

template <int IL, int OL>
__device__ __forceinline__ void signed_fix_body(const FixArgs &fa, int64_t k) {
  const int ol = fa.ol, il = fa.il, rec = 2 * il + 1;
  const int64_t lf = fa.lf, lg = fa.lg;
  if (k >= lf + lg - 1) return;
  uint64_t w[OL], r[OL], cnt[OL];
#pragma unroll
  for (int l = 0; l < OL; l++) w[l] = cnt[l] = 0;
  const int64_t fhi = k < lf - 1 ? k : lf - 1;
  const int64_t flo = k - lg + 1 > 0 ? k - lg + 1 : 0;
  const int64_t ghi = k < lg - 1 ? k : lg - 1;
  const int64_t glo = k - lf + 1 > 0 ? k - lf + 1 : 0;
  add_window_fixed<IL, OL>(w, fa.pf + fhi * rec, flo > 0 ? fa.pf + (flo - 1) * rec : nullptr, il);
  add_window_fixed<IL, OL>(w, fa.pg + ghi * rec, glo > 0 ? fa.pg + (glo - 1) * rec : nullptr, il);
  uint64_t *hk = fa.h + k * ol;
#pragma unroll
  for (int l = 0; l < OL; l++) r[l] = l < ol ? hk[l] : 0ull;
  cnt[0] = (uint64_t)(fhi - flo + 1);
  sub_shifted_fixed<OL>(r, w, ol, fa.b - 1);
  sub_shifted_fixed<OL>(r, cnt, ol, 2 * fa.b - 2);
#pragma unroll
  for (int l = 0; l < OL; l++)
    if (l < ol) hk[l] = r[l];
}

// h_k -= 2^(b-1) (W_f + W_g)_k + 2^(2b-2) cnt_k, one output per thread;
// the limb-count class is uniform per CTA (a batch may mix classes)
template <class Src>
__global__ void __launch_bounds__(128) signed_fix_fast(Src src) {
  int64_t local;
  const FixArgs &fa = src.locate(blockIdx.x, local);
  const int64_t k = local * 128 + threadIdx.x;
  switch (fa.il) {
    case 1: signed_fix_body<1, 3>(fa, k); break;
    case 2: signed_fix_body<2, 5>(fa, k); break;
    case 3:
    case 4: signed_fix_body<4, 9>(fa, k); break;
    default: signed_fix_body<8, 17>(fa, k); break;
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
  fx = FixArgs{h, ol, lf, lg, b, in_limbs, a.P[0], a.P[1], f, g, nullptr, nullptr};
  fix_blocks = (lf + lg - 1 + 127) / 128;
  const bool fast = lf <= kScanL && lg <= kScanL && in_limbs <= 8 && ol <= 17;
  if (fast) {  // tiles of 512 coefficients
    a.nblocks[0] = (lf + kPT - 1) / kPT;
    a.nblocks[1] = (lg + kPT - 1) / kPT;
  }
  pref_blocks = a.nblocks[0] + a.nblocks[1];
  return fast;
}

// The prefix records of f and g: they depend on the inputs only, so they may
// run concurrently with the products.
cudaError_t launch_signed_prefix(int ol, const uint64_t *f, int64_t lf, const uint64_t *g,
                                 int64_t lg, int b, int in_limbs, uint64_t *prefix,
                                 cudaStream_t s) {
  if (ol > kMaxOl || in_limbs > kMaxIn) return cudaErrorInvalidValue;
  PrefArgs a;
  FixArgs fx;
  int64_t pb, fb;
  if (make_signed_args(nullptr, ol, f, lf, g, lg, b, in_limbs, prefix, a, fx, pb, fb)) {
    pref_tile<One<PrefArgs>><<<(unsigned)pb, kPT, 0, s>>>(One<PrefArgs>{a});
    note_launches(1);
    return cudaGetLastError();
  }
  pref_block_totals<<<(unsigned)pb, kThreads, 0, s>>>(a);
  pref_scan_totals<<<2, 64, 0, s>>>(a);
  pref_apply<<<(unsigned)pb, kThreads, 0, s>>>(a);
  note_launches(3);
  return cudaGetLastError();
}

// The correction of h from the prefix records (after launch_signed_prefix).
cudaError_t launch_signed_apply(uint64_t *h, int ol, const uint64_t *f, int64_t lf,
                                const uint64_t *g, int64_t lg, int b, int in_limbs,
                                uint64_t *prefix, cudaStream_t s) {
  if (ol > kMaxOl || in_limbs > kMaxIn) return cudaErrorInvalidValue;
  PrefArgs a;
  FixArgs fx;
  int64_t pb, fb;
  make_signed_args(h, ol, f, lf, g, lg, b, in_limbs, prefix, a, fx, pb, fb);
  if (in_limbs <= 8 && ol <= 17)
    signed_fix_fast<One<FixArgs>><<<(unsigned)fb, 128, 0, s>>>(One<FixArgs>{fx});
  else
    signed_fix_kernel<One<FixArgs>><<<(unsigned)fb, 128, 0, s>>>(One<FixArgs>{fx});
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_signed_fix(uint64_t *h, int ol, const uint64_t *f, int64_t lf,
                              const uint64_t *g, int64_t lg, int b, int in_limbs,
                              uint64_t *prefix, cudaStream_t s) {
  const cudaError_t e = launch_signed_prefix(ol, f, lf, g, lg, b, in_limbs, prefix, s);
  if (e != cudaSuccess) return e;
  return launch_signed_apply(h, ol, f, lf, g, lg, b, in_limbs, prefix, s);
}

cudaError_t launch_signed_prefix_batch(const PrefArgs *pa, const int64_t *pref_prefix, int n,
                                       int64_t pref_blocks, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  pref_tile<Many<PrefArgs>><<<(unsigned)pref_blocks, kPT, 0, s>>>(
      Many<PrefArgs>{pa, pref_prefix, n});
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_signed_apply_batch(const FixArgs *fa, const int64_t *fix_prefix, int n,
                                      int64_t fix_blocks, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  signed_fix_fast<Many<FixArgs>><<<(unsigned)fix_blocks, 128, 0, s>>>(
      Many<FixArgs>{fa, fix_prefix, n});
  note_launches(1);
  return cudaGetLastError();
}

size_t signed_prefix_bytes(int64_t lf, int64_t lg, int il) {
  const int rec = 2 * il + 1;
  return (size_t)(lf + lg + nblocks_for(lf) + nblocks_for(lg)) * rec * 8;
}

}  // namespace ks
