// Exact seeds of the reconstruction chains (Sec. 3.2): the values
//
//   h'_k = sum_t f_t g_(k-t)   (+ K = 2^kb for signed inputs)
//
// for clusters of C consecutive k (the pair c_(s-1), c_s of one run, or of
// both runs of Sec. 3.4 at once).  A chain started from such a pair needs no
// predecessor, so the recurrence runs in parallel chains.
//
// Narrow operands (both at most 64 bits, one limb): a CTA of 128 threads takes
// one cluster and a slice of kTSlice indices t, kTPer consecutive ones per
// thread.  A thread loads its f_t and the window of g they meet (kTPer + C - 1
// values, shared by the C values of the cluster) before it uses any, so the
// slice costs one memory round trip, then multiplies:
//   * b <= 48: the values split into 24-bit halves, x = xl + 2^24 xh
//     (xl unsigned, xh signed), three 32 x 32 -> 64-bit multiply-adds per pair
//     (xl yl, xh yh and the Karatsuba middle term (xl + xh)(yl + yh)), whose
//     sums over one slice fit 64 bits;
//   * 48 < b <= 64: full 64 x 64 -> 128-bit products (signed or unsigned)
//     into 192-bit two's complement sums.
// The CTA reduces its sums and stores each value's 192-bit two's complement
// partial (slice 0 adds K) as six words in a slot of its own; the
// reconstruction adds the slices' words as column sums and carries them into
// the value mod 2^192 (exact: the values are non-negative and below 2^192).
//
// Wide operands: one CTA per value; a thread multiplies the magnitudes of its
// terms word by word (NW 32-bit words, a compile-time size) and keeps signed
// 64-bit column sums; the CTA adds them and one thread carries them (and K)
// into the value's words.
#include "ks_internal.cuh"
#include "ks_src.cuh"

namespace ks {

namespace {
constexpr int kST = 128;            // threads of a narrow seed CTA
constexpr int kTPer = 16;           // consecutive indices t per thread
constexpr int64_t kTSlice = kST * kTPer;  // indices t per narrow CTA
constexpr int kWT = 128;            // threads of a wide seed CTA

// a one-limb coefficient of b = 64 - sh bits as a 64-bit value: sign-extended
// from bit b - 1 (signed) or its low b bits (unsigned)
__device__ __forceinline__ uint64_t extend64(uint64_t raw, int sh, int sgn) {
  const uint64_t up = raw << sh;
  return sgn ? (uint64_t)((int64_t)up >> sh) : up >> sh;
}
__device__ __forceinline__ uint64_t coeff64(const uint64_t *p, int64_t i, int b, int sgn) {
  return extend64(__ldg(p + i), 64 - b, sgn);
}

// 192-bit two's complement accumulator
struct W3 {
  uint64_t w0, w1, w2;
};
__device__ __forceinline__ void add3(W3 &a, uint64_t b0, uint64_t b1, uint64_t b2) {
  a.w0 += b0;
  const uint64_t c0 = a.w0 < b0;
  const uint64_t t = a.w1 + b1;
  const uint64_t c1 = t < b1;
  a.w1 = t + c0;
  const uint64_t c2 = a.w1 < c0;
  a.w2 += b2 + c1 + c2;
}
// v << sh as 192 bits (v signed, 0 <= sh < 64)
__device__ __forceinline__ void shl3(int64_t v, int sh, uint64_t &w0, uint64_t &w1,
                                     uint64_t &w2) {
  w0 = (uint64_t)v << sh;
  w1 = sh ? (uint64_t)(v >> (64 - sh)) : (uint64_t)(v >> 63);
  w2 = (uint64_t)(v >> 63);
}

__device__ __forceinline__ unsigned long long warp_sum(unsigned long long v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  return v;
}

// Shared-memory index of staged element i: one padding word per 16, so the
// 16-element ranges of consecutive threads start in different banks.
__device__ __forceinline__ int spad(int i) { return i + (i >> 4); }

// one CTA: cluster j, slice `slice`; PATH 0: b <= 48 (24-bit halves), 1: signed
// 64-bit, 2: unsigned 64-bit.  The slice's f_t (t in [s_lo, s_lo + kTSlice))
// and the window of g they meet are staged in shared memory by coalesced loads
// (zero outside the polynomials); thread tid then takes t = s_lo + kTPer tid + u,
// u < kTPer, whose g values g_(k0 + r - t) form a window of kTPer + C - 1
// consecutive staged values, read once into registers (the loop over u is
// unrolled, so the window slides by register renaming).
template <int PATH, int C>
__device__ __forceinline__ void seed_narrow_body(const SeedArgs &a, int64_t local) {
  constexpr int kSF = kTSlice + kTSlice / 16;
  constexpr int kGW = kTSlice + C - 1;  // g window length
  __shared__ uint64_t sf[kSF];
  __shared__ uint64_t sg[kGW + kGW / 16 + 1];
  __shared__ unsigned long long red[kST / 32][4][6];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int64_t j = local / a.slices, slice = local - j * a.slices;
  const int64_t k0 = a.k00 + a.kstep * j;
  const int64_t lf = a.lf, lg = a.lg;
  int64_t tlo = k0 - (lg - 1);
  if (tlo < 0) tlo = 0;
  int64_t thi = k0 + C - 1;
  if (thi > lf - 1) thi = lf - 1;
  const int64_t s_lo = tlo + slice * a.tslice;
  int64_t s_hi = s_lo + a.tslice - 1;
  if (s_hi > thi) s_hi = thi;
  // this item's partial of value r: six words at part + 6 r (a slot per slice,
  // so items never share memory and nothing needs clearing)
  unsigned long long *part = a.acc + (j * C * a.slices + slice) * 6;
  const int64_t vstride = a.slices * 6;  // between the values of the cluster
  if (s_lo > s_hi) {  // nothing in this slice (uniform over the CTA): a zero partial
    if (tid < 6 * C) part[(tid / 6) * vstride + tid % 6] = 0ull;
    return;
  }
  const int bf = a.bf, bg = a.bg, sgn = a.sgn;
  // staged g window: element i is g_(jg_lo + i), jg_lo = k0 - (s_lo + kTSlice - 1)
  const int64_t jg_lo = k0 - (s_lo + kTSlice - 1);
  {
    // all loads first (one round trip); bounds checked only near the ends
    uint64_t rf[kTSlice / kST], rg[(kGW + kST - 1) / kST];
    const uint64_t *fs = a.f + s_lo, *gs0 = a.g + jg_lo;
    if (s_lo + kTSlice - 1 <= s_hi) {
#pragma unroll
      for (int v = 0; v < kTSlice / kST; v++) rf[v] = __ldg(fs + tid + v * kST);
    } else {
#pragma unroll
      for (int v = 0; v < kTSlice / kST; v++)
        rf[v] = s_lo + tid + v * kST <= s_hi ? __ldg(fs + tid + v * kST) : 0ull;
    }
    if (jg_lo >= 0 && jg_lo + kGW <= lg) {
#pragma unroll
      for (int v = 0; v < (kGW + kST - 1) / kST; v++) {
        const int i = tid + v * kST;
        rg[v] = i < kGW ? __ldg(gs0 + i) : 0ull;
      }
    } else {
#pragma unroll
      for (int v = 0; v < (kGW + kST - 1) / kST; v++) {
        const int i = tid + v * kST;
        const int64_t jg = jg_lo + i;
        rg[v] = (i < kGW && jg >= 0 && jg < lg) ? __ldg(a.g + jg) : 0ull;
      }
    }
    // the b-bit values, sign-extended (signed) or masked (unsigned), once
    const int shf = 64 - bf, shg = 64 - bg;
#pragma unroll
    for (int v = 0; v < kTSlice / kST; v++) rf[v] = extend64(rf[v], shf, sgn);
#pragma unroll
    for (int v = 0; v < (kGW + kST - 1) / kST; v++) rg[v] = extend64(rg[v], shg, sgn);
#pragma unroll
    for (int v = 0; v < kTSlice / kST; v++) sf[spad(tid + v * kST)] = rf[v];
#pragma unroll
    for (int v = 0; v < (kGW + kST - 1) / kST; v++) {
      const int i = tid + v * kST;
      if (i < kGW) sg[spad(i)] = rg[v];
    }
  }
  __syncthreads();
  // this thread: f at staged kTPer tid + u; its g window from staged
  // wb = kTSlice - kTPer (tid + 1): pair (u, r) is window entry kTPer - 1 - u + r
  uint64_t fv[kTPer], gv[kTPer + C - 1];
  const int fb = kTPer * tid, wb = (int)kTSlice - kTPer * (tid + 1);
#pragma unroll
  for (int u = 0; u < kTPer; u++) fv[u] = sf[spad(fb + u)];
#pragma unroll
  for (int o = 0; o < kTPer + C - 1; o++) gv[o] = sg[spad(wb + o)];
  if (PATH == 0) {
    unsigned long long ll[C];
    long long hh[C], ss[C];
#pragma unroll
    for (int r = 0; r < C; r++) ll[r] = hh[r] = ss[r] = 0;
    // every g value split once: (low 24 bits, the rest signed, their sum)
    uint32_t gl[kTPer + C - 1];
    int32_t gh[kTPer + C - 1], gs[kTPer + C - 1];
#pragma unroll
    for (int o = 0; o < kTPer + C - 1; o++) {
      const int64_t y = (int64_t)gv[o];
      gl[o] = (uint32_t)y & 0xFFFFFFu;
      gh[o] = (int32_t)(y >> 24);
      gs[o] = (int32_t)gl[o] + gh[o];
    }
#pragma unroll
    for (int u = 0; u < kTPer; u++) {
      const int64_t x = (int64_t)fv[u];
      const uint32_t xl = (uint32_t)x & 0xFFFFFFu;
      const int32_t xh = (int32_t)(x >> 24);
      const int32_t xs = (int32_t)xl + xh;
#pragma unroll
      for (int r = 0; r < C; r++) {
        const int o = r - u + kTPer - 1;
        ll[r] += (unsigned long long)xl * gl[o];
        hh[r] += (long long)xh * gh[o];
        ss[r] += (long long)xs * gs[o];
      }
    }
    // the 3 C sums of the CTA through shared memory (the staging buffer is free
    // once every thread has its values): quantity q of thread i at sf[q kST + i];
    // 8 threads per quantity add 16 each, then one thread per value adds 8
    __syncthreads();
    unsigned long long *rq = reinterpret_cast<unsigned long long *>(sf);
#pragma unroll
    for (int r = 0; r < C; r++) {
      rq[(3 * r + 0) * kST + tid] = ll[r];
      rq[(3 * r + 1) * kST + tid] = (unsigned long long)hh[r];
      rq[(3 * r + 2) * kST + tid] = (unsigned long long)ss[r];
    }
    __syncthreads();
    unsigned long long *rq2 = rq + 3 * C * kST;
    if (tid < 3 * C * 8) {
      const int q = tid >> 3, part8 = tid & 7;
      unsigned long long v = 0;
#pragma unroll
      for (int i = 0; i < kST / 8; i++) v += rq[q * kST + part8 * (kST / 8) + i];
      rq2[tid] = v;
    }
    __syncthreads();
    (void)red;
    (void)lane;
    (void)wid;
    if (tid < C) {
      unsigned long long L = 0, H = 0, S = 0;
#pragma unroll
      for (int i = 0; i < 8; i++) {
        L += rq2[(3 * tid + 0) * 8 + i];
        H += rq2[(3 * tid + 1) * 8 + i];
        S += rq2[(3 * tid + 2) * 8 + i];
      }
      const long long mid = (long long)(S - L - H);  // exact: |mid| < 2^61
      W3 v = {L, 0, 0};
      uint64_t b0, b1, b2;
      shl3(mid, 24, b0, b1, b2);
      add3(v, b0, b1, b2);
      shl3((long long)H, 48, b0, b1, b2);
      add3(v, b0, b1, b2);
      if (slice == 0 && a.kb >= 0) {
        const int kb = a.kb;
        add3(v, kb < 64 ? 1ull << kb : 0, (kb >= 64 && kb < 128) ? 1ull << (kb - 64) : 0,
             kb >= 128 ? 1ull << (kb - 128) : 0);
      }
      const uint32_t wd[6] = {(uint32_t)v.w0, (uint32_t)(v.w0 >> 32), (uint32_t)v.w1,
                              (uint32_t)(v.w1 >> 32), (uint32_t)v.w2, (uint32_t)(v.w2 >> 32)};
#pragma unroll
      for (int w = 0; w < 6; w++) part[tid * vstride + w] = wd[w];
    }
  } else {
    W3 s3[C];
#pragma unroll
    for (int r = 0; r < C; r++) s3[r] = W3{0, 0, 0};
#pragma unroll
    for (int u = 0; u < kTPer; u++) {
      const uint64_t x = fv[u];
#pragma unroll
      for (int r = 0; r < C; r++) {
        const uint64_t y = gv[r - u + kTPer - 1];
        const uint64_t lo = x * y;
        uint64_t hi, ext;
        if (PATH == 1) {
          hi = (uint64_t)__mul64hi((long long)x, (long long)y);
          ext = (uint64_t)((int64_t)hi >> 63);
        } else {
          hi = __umul64hi(x, y);
          ext = 0;
        }
        add3(s3[r], lo, hi, ext);
      }
    }
    unsigned long long col[C][6];
#pragma unroll
    for (int r = 0; r < C; r++) {
      col[r][0] = (uint32_t)s3[r].w0;
      col[r][1] = s3[r].w0 >> 32;
      col[r][2] = (uint32_t)s3[r].w1;
      col[r][3] = s3[r].w1 >> 32;
      col[r][4] = (uint32_t)s3[r].w2;
      col[r][5] = s3[r].w2 >> 32;
#pragma unroll
      for (int w = 0; w < 6; w++) {
        col[r][w] = warp_sum(col[r][w]);
        if (lane == 0) red[wid][r][w] = col[r][w];
      }
    }
    __syncthreads();
    if (tid < 6 * C) {
      const int r = tid / 6, w = tid - 6 * r;
      unsigned long long v = 0;
#pragma unroll
      for (int q = 0; q < kST / 32; q++) v += red[q][r][w];
      if (slice == 0 && a.kb >= 0 && (a.kb >> 5) == w) v += 1ull << (a.kb & 31);
      part[r * vstride + w] = v;
    }
  }
}

// One CTA per item (cluster, slice) of every product.
template <int PATH, int C, class Src>
__global__ void __launch_bounds__(kST) seed_narrow(Src src) {
  int64_t local;
  const SeedArgs &a = src.locate(blockIdx.x, local);
  seed_narrow_body<PATH, C>(a, local);
}

// The NW 32-bit words of |c| for a coefficient of b bits in il limbs, and its
// sign (signed inputs: two's complement from bit b - 1).
template <int NW>
__device__ __forceinline__ bool mag_words(const uint64_t *c, int il, int b, int sgn,
                                          uint32_t (&w)[NW]) {
#pragma unroll
  for (int i = 0; i < NW; i++) {
    const int lo = 32 * i;
    uint32_t v = 0;
    if (lo < b) {
      const uint64_t limb = c[lo >> 6];
      v = (uint32_t)(limb >> (lo & 63));
      const int keep = b - lo;
      if (keep < 32) v &= (1u << keep) - 1u;
    }
    w[i] = v;
  }
  const bool neg = sgn && ((c[(b - 1) >> 6] >> ((b - 1) & 63)) & 1ull);
  if (neg) {  // sign-extend to NW words, then negate
    uint64_t carry = 1;
#pragma unroll
    for (int i = 0; i < NW; i++) {
      const int lo = 32 * i;
      uint32_t ext = w[i];
      if (lo + 32 > b) ext |= lo >= b ? 0xFFFFFFFFu : ~((1u << (b - lo)) - 1u);
      const uint64_t t = (uint64_t)(uint32_t)~ext + carry;
      w[i] = (uint32_t)t;
      carry = t >> 32;
    }
  }
  return neg;
}

template <int NW, class Src>
__global__ void __launch_bounds__(kWT) seed_wide(Src src) {
  __shared__ unsigned long long colsum[kMaxSeedWords];
  int64_t vid;
  const SeedArgs &a = src.locate(blockIdx.x, vid);
  const int64_t j = vid / a.C;
  const int r = (int)(vid - j * a.C);
  const int64_t k = a.k00 + a.kstep * j + r;
  const int seed_words = a.seed_words;
  for (int w = threadIdx.x; w < seed_words; w += kWT) colsum[w] = 0ull;
  __syncthreads();
  long long loc[2 * NW];
#pragma unroll
  for (int w = 0; w < 2 * NW; w++) loc[w] = 0;
  int64_t t_lo = k - (a.lg - 1);
  if (t_lo < 0) t_lo = 0;
  const int64_t t_hi = k < a.lf - 1 ? k : a.lf - 1;
  for (int64_t t = t_lo + threadIdx.x; t <= t_hi; t += kWT) {
    uint32_t fw[NW], gw[NW], pr[2 * NW];
    const bool nf = mag_words<NW>(a.f + t * a.ilf, a.ilf, a.bf, a.sgn, fw);
    const bool ng = mag_words<NW>(a.g + (k - t) * a.ilg, a.ilg, a.bg, a.sgn, gw);
#pragma unroll
    for (int w = 0; w < 2 * NW; w++) pr[w] = 0u;
#pragma unroll
    for (int x = 0; x < NW; x++) {
      uint64_t carry = 0;
#pragma unroll
      for (int y = 0; y < NW; y++) {
        const uint64_t tt = (uint64_t)fw[x] * gw[y] + pr[x + y] + carry;
        pr[x + y] = (uint32_t)tt;
        carry = tt >> 32;
      }
      pr[x + NW] = (uint32_t)carry;
    }
    if (nf != ng) {
#pragma unroll
      for (int w = 0; w < 2 * NW; w++) loc[w] -= pr[w];
    } else {
#pragma unroll
      for (int w = 0; w < 2 * NW; w++) loc[w] += pr[w];
    }
  }
#pragma unroll
  for (int w = 0; w < 2 * NW; w++)
    if (w < seed_words && loc[w]) atomicAdd(&colsum[w], (unsigned long long)loc[w]);
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t *out = a.seeds + vid * seed_words;
    long long carry = 0;
    for (int w = 0; w < seed_words; w++) {
      long long v = (long long)colsum[w] + carry;
      if (a.kb >= 0 && (a.kb >> 5) == w) v += 1ll << (a.kb & 31);
      out[w] = (uint32_t)v;
      carry = v >> 32;  // arithmetic: the column sums are signed
    }
  }
}

template <class Src>
void launch_kind(int kind, int64_t blocks, const Src &src, cudaStream_t s) {
  const unsigned grid = (unsigned)blocks;
  switch (kind) {
    case 1: seed_narrow<0, 2, Src><<<grid, kST, 0, s>>>(src); break;
    case 2: seed_narrow<0, 4, Src><<<grid, kST, 0, s>>>(src); break;
    case 3: seed_narrow<1, 2, Src><<<grid, kST, 0, s>>>(src); break;
    case 4: seed_narrow<1, 4, Src><<<grid, kST, 0, s>>>(src); break;
    case 5: seed_narrow<2, 2, Src><<<grid, kST, 0, s>>>(src); break;
    case 6: seed_narrow<2, 4, Src><<<grid, kST, 0, s>>>(src); break;
    case 102: seed_wide<2, Src><<<grid, kWT, 0, s>>>(src); break;
    case 104: seed_wide<4, Src><<<grid, kWT, 0, s>>>(src); break;
    case 108: seed_wide<8, Src><<<grid, kWT, 0, s>>>(src); break;
    case 116: seed_wide<16, Src><<<grid, kWT, 0, s>>>(src); break;
    case 132: seed_wide<32, Src><<<grid, kWT, 0, s>>>(src); break;
    case 164: seed_wide<64, Src><<<grid, kWT, 0, s>>>(src); break;
  }
}
}  // namespace

// the t range of a cluster spans at most min(Lf, Lg + C - 1) indices
int64_t seed_slices(int64_t lf, int64_t lg, int C) {
  const int64_t span = lf < lg + C - 1 ? lf : lg + C - 1;
  return (span + kTSlice - 1) / kTSlice;
}

const int kSeedKindList[kSeedKinds] = {1, 2, 3, 4, 5, 6, 102, 104, 108, 116, 132, 164};

int seed_kind_index(int kind) {
  for (int i = 0; i < kSeedKinds; i++)
    if (kSeedKindList[i] == kind) return i;
  return -1;
}

int make_seed_plan(const uint64_t *f, int64_t lf, int bf, const uint64_t *g, int64_t lg, int bg,
                   int sgn, int kb, int64_t k00, int64_t kstep, int64_t ncl, int C,
                   unsigned long long *acc, uint32_t *seeds, int seed_words, SeedPlan &sp) {
  sp = SeedPlan{};
  sp.nvalues = ncl * C;
  if (sp.nvalues == 0) return 0;
  if (C != 2 && C != 4) return -1;
  SeedArgs &a = sp.a;
  a.f = f;
  a.g = g;
  a.lf = lf;
  a.lg = lg;
  a.bf = bf;
  a.bg = bg;
  a.ilf = (bf + 63) / 64;
  a.ilg = (bg + 63) / 64;
  a.sgn = sgn ? 1 : 0;
  a.kb = sgn ? kb : -1;
  a.k00 = k00;
  a.kstep = kstep;
  a.ncl = ncl;
  a.C = C;
  a.acc = acc;
  a.seeds = seeds;
  a.seed_words = seed_words;
  if (bf <= 64 && bg <= 64) {
    if (a.kb >= 192) return -1;
    a.tslice = kTSlice;
    a.slices = seed_slices(lf, lg, C);
    // narrow kinds 1-6: (b <= 48 | signed 64-bit | unsigned 64-bit) x (C = 2 | 4)
    const int path = (bf <= 48 && bg <= 48) ? 0 : (sgn ? 1 : 2);
    sp.kind = 1 + 2 * path + (C == 4 ? 1 : 0);
    sp.blocks = ncl * a.slices;
    return 0;
  }
  if (seed_words > kMaxSeedWords) return -1;
  const int nw = ((bf > bg ? bf : bg) + 31) / 32;
  int cls = 2;
  while (cls < nw) cls *= 2;
  if (cls > 64) return -1;
  sp.kind = 100 + cls;
  sp.blocks = sp.nvalues;
  return 0;
}

cudaError_t launch_seed_plan(const SeedPlan &sp, cudaStream_t s) {
  if (sp.kind == 0 || sp.blocks == 0) return cudaSuccess;
  launch_kind(sp.kind, sp.blocks, One<SeedArgs>{sp.a}, s);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_seeds_batch(int kind, const SeedArgs *d, const int64_t *prefix, int n,
                               int64_t blocks, cudaStream_t s) {
  if (n == 0 || blocks == 0) return cudaSuccess;
  launch_kind(kind, blocks, Many<SeedArgs>{d, prefix, n}, s);
  note_launches(1);
  return cudaGetLastError();
}

}  // namespace ks
