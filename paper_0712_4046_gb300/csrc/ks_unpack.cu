// Unpack (Sec. 3.1, 3.3), reciprocal reconstruction (Sec. 3.2, used twice by
// Sec. 3.4), the signed-bias correction and the reduction mod p (Sec. 4).
#include "ks_internal.cuh"
#include "ks_src.cuh"

namespace ks {

// ------------------------------------------------------------------ unpack
// h'_k = bits [off + kN, off + kN + width) of V (or of V_odd for odd k).
// KS1: V = h(2^N), off = 0, width N.  KS2: V = P+ + P- = 2 h0(X^2) and
// V_odd = P+ - P- = 2X h1(X^2); then both even and odd coefficients sit at
// bit 1 + kN, width 2N (Sec. 3.3).
// One CTA writes 1024 consecutive output limbs, four per thread (strided by
// the block, so every store is coalesced and the four loads are independent).
constexpr int kUnpackPer = 4;
template <class Src>
__global__ void __launch_bounds__(256) unpack_kernel(Src src) {
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
    uint64_t v = 0;
    if (rem > 0) {
      v = get_bits64(src_w, a.nwords, a.off + k * a.N + 64 * (int64_t)l);
      if (rem < 64) v &= (1ull << rem) - 1ull;
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
  unpack_kernel<One<UnpackArgs>><<<(unsigned)unpack_blocks(a), 256, 0, s>>>(One<UnpackArgs>{a});
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_unpack_batch(const UnpackArgs *d, const int64_t *prefix, int n,
                                int64_t blocks, cudaStream_t s) {
  if (blocks == 0) return cudaSuccess;
  unpack_kernel<Many<UnpackArgs>><<<(unsigned)blocks, 256, 0, s>>>(Many<UnpackArgs>{d, prefix, n});
  note_launches(1);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ seeds
// Exact h'_k = sum_t f'_t g'_(k-t) (biased, non-negative b-bit inputs) for the
// chain starts of the reconstruction: one CTA per coefficient.  A thread
// multiplies its terms word by word (NW 32-bit words per coefficient, a
// compile-time size so the words stay in registers) and keeps 64-bit per-word
// sums; the CTA adds those into shared 64-bit word sums and one thread
// propagates the carries.
namespace {
constexpr int kSeedThreads = 128;
}  // namespace

template <int NW>
__device__ __forceinline__ void coeff_words(const uint64_t *c, int in_limbs, int b, int flip,
                                            uint32_t *w) {
#pragma unroll
  for (int i = 0; i < NW; i++) {
    const int rem = b - 32 * i;
    w[i] = rem > 0 ? coeff_slice(c, in_limbs, b, flip, 32 * i, rem < 32 ? rem : 32) : 0u;
  }
}

template <int NW, class Src>
__global__ void __launch_bounds__(kSeedThreads) seed_kernel(Src src) {
  __shared__ unsigned long long colsum[kMaxSeedWords];
  int64_t sid;
  const SeedArgs &a = src.locate(blockIdx.x, sid);
  uint32_t *seeds = a.seeds;
  const int seed_words = a.seed_words;
  const uint64_t *f = a.f, *g = a.g;
  const int64_t lf = a.lf, lg = a.lg;
  const int b = a.b, in_limbs = a.in_limbs, flip = a.flip;
  int r = 0;
  int64_t per_run = 2 * (a.run[0].nchains - 1);
  while (r + 1 < a.nruns && sid >= per_run) {
    sid -= per_run;
    r++;
    per_run = 2 * (a.run[r].nchains - 1);
  }
  const RecoverRun &R = a.run[r];
  const int64_t c = sid / 2 + 1;
  const int64_t i = c * a.chain - 1 + (sid & 1);
  const int64_t k = R.kbase + R.kstride * i;
  for (int w = threadIdx.x; w < seed_words; w += blockDim.x) colsum[w] = 0ull;
  __syncthreads();

  unsigned long long loc[2 * NW];
#pragma unroll
  for (int w = 0; w < 2 * NW; w++) loc[w] = 0ull;
  int64_t t_lo = k - (lg - 1);
  if (t_lo < 0) t_lo = 0;
  const int64_t t_hi = k < lf - 1 ? k : lf - 1;
  for (int64_t t = t_lo + threadIdx.x; t <= t_hi; t += blockDim.x) {
    uint32_t fw[NW], gw[NW], pr[2 * NW];
    coeff_words<NW>(f + t * in_limbs, in_limbs, b, flip, fw);
    coeff_words<NW>(g + (k - t) * in_limbs, in_limbs, b, flip, gw);
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
#pragma unroll
    for (int w = 0; w < 2 * NW; w++) loc[w] += pr[w];
  }
#pragma unroll
  for (int w = 0; w < 2 * NW; w++)
    if (w < seed_words && loc[w]) atomicAdd(&colsum[w], loc[w]);
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t *out = seeds + (R.seed_base + sid) * seed_words;
    unsigned long long carry = 0;
    for (int w = 0; w < seed_words; w++) {
      const unsigned long long v = colsum[w] + carry;
      out[w] = (uint32_t)v;
      carry = v >> 32;
    }
  }
}

// b <= 64: each coefficient is one 64-bit word; products are 128-bit and a
// thread keeps a 192-bit running sum in three registers.
template <class Src>
__global__ void __launch_bounds__(kSeedThreads) seed_kernel64(Src src) {
  __shared__ unsigned long long colsum[kMaxSeedWords];
  int64_t sid;
  const SeedArgs &a = src.locate(blockIdx.x, sid);
  uint32_t *seeds = a.seeds;
  const int seed_words = a.seed_words;
  const uint64_t *f = a.f, *g = a.g;
  const int64_t lf = a.lf, lg = a.lg;
  const int b = a.b, in_limbs = a.in_limbs, flip = a.flip;
  int r = 0;
  int64_t per_run = 2 * (a.run[0].nchains - 1);
  while (r + 1 < a.nruns && sid >= per_run) {
    sid -= per_run;
    r++;
    per_run = 2 * (a.run[r].nchains - 1);
  }
  const RecoverRun &R = a.run[r];
  const int64_t c = sid / 2 + 1;
  const int64_t i = c * a.chain - 1 + (sid & 1);
  const int64_t k = R.kbase + R.kstride * i;
  for (int w = threadIdx.x; w < seed_words; w += blockDim.x) colsum[w] = 0ull;
  __syncthreads();
  const uint64_t mask = b >= 64 ? ~0ull : ((1ull << b) - 1ull);
  const uint64_t fl = flip ? (1ull << (b - 1)) : 0ull;
  uint64_t a0 = 0, a1 = 0, a2 = 0;
  int64_t t_lo = k - (lg - 1);
  if (t_lo < 0) t_lo = 0;
  const int64_t t_hi = k < lf - 1 ? k : lf - 1;
  for (int64_t t = t_lo + threadIdx.x; t <= t_hi; t += blockDim.x) {
    const uint64_t x = (f[t * in_limbs] & mask) ^ fl;
    const uint64_t y = (g[(k - t) * in_limbs] & mask) ^ fl;
    const uint64_t lo = x * y, hi = __umul64hi(x, y);
    a0 += lo;
    const uint64_t c1 = a0 < lo;
    const uint64_t h1 = hi + c1;  // hi <= 2^64 - 2
    a1 += h1;
    a2 += a1 < h1;
  }
  const uint32_t w6[6] = {(uint32_t)a0, (uint32_t)(a0 >> 32), (uint32_t)a1,
                          (uint32_t)(a1 >> 32), (uint32_t)a2, (uint32_t)(a2 >> 32)};
#pragma unroll
  for (int w = 0; w < 6; w++)
    if (w < seed_words && w6[w]) atomicAdd(&colsum[w], (unsigned long long)w6[w]);
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t *out = seeds + (R.seed_base + sid) * seed_words;
    unsigned long long carry = 0;
    for (int w = 0; w < seed_words; w++) {
      const unsigned long long v = colsum[w] + carry;
      out[w] = (uint32_t)v;
      carry = v >> 32;
    }
  }
}

// Blocked seeds, b <= 64: a CTA computes kSG consecutive seeds of one run.
// For each chunk of kST indices t it stages f'_t and the window of g' those
// seeds need in shared memory (the seeds' k differ by at most kSW - kST), so
// every input word is read from L2 once per CTA rather than once per seed.
// 16 threads per seed accumulate 192-bit sums over a strided part of the chunk.
namespace {
constexpr int kSG = 16;
constexpr int kST = 512;
constexpr int kSW = 2048;
constexpr int64_t kSlice = 2048;  // indices t per CTA
__device__ __forceinline__ int64_t seed_k(const RecoverRun &R, int64_t chain, int64_t sid) {
  const int64_t c = sid / 2 + 1;
  return R.kbase + R.kstride * (c * chain - 1 + (sid & 1));
}
}  // namespace

// 32 x 32 -> 64-bit multiply-add (one instruction)
__device__ __forceinline__ void mad_wide(unsigned long long &acc, uint32_t x, uint32_t y) {
  asm("mad.wide.u32 %0, %1, %2, %0;" : "+l"(acc) : "r"(x), "r"(y));
}

// b <= 48: values split into 24-bit halves, x = xl + 2^24 xh, with xs = xl + xh;
// x y = xl yl + (xs ys - xl yl - xh yh) 2^24 + xh yh 2^48, three multiply-adds per
// pair whose sums over one slice (2048 t, 32 per thread) stay below 2^56.
// Thread (sub, sq): t = sub, sub + 64, ... of each chunk, seeds sq + 4 r (r < 4),
// one load of x serving four seeds.
__device__ __forceinline__ uint4 split24(uint64_t v) {
  const uint32_t lo = (uint32_t)(v & 0xFFFFFFull), hi = (uint32_t)(v >> 24);
  return make_uint4(lo, hi, lo + hi, 0u);
}

template <class Src>
__global__ void __launch_bounds__(256) seed_blocked64(Src src) {
  __shared__ __align__(16) uint8_t sraw[kST * 16 + kSW * 16];
  __shared__ unsigned long long colsum[kSG][6];
  int64_t bid;
  const SeedBArgs &a = src.locate(blockIdx.x, bid);
  unsigned long long *acc = a.acc;
  const uint64_t *f = a.f, *g = a.g;
  const int64_t lf = a.lf, lg = a.lg;
  const int b = a.b, in_limbs = a.in_limbs, flip = a.flip;
  const int64_t slice = bid % a.slices;
  int64_t gid = bid / a.slices;
  int r = 0;
  while (r + 1 < a.nruns && gid >= a.groups[r]) {
    gid -= a.groups[r];
    r++;
  }
  const RecoverRun &R = a.run[r];
  const int64_t nseeds = 2 * (R.nchains - 1);
  const int64_t sid0 = gid * kSG;
  const int nS = (int)(nseeds - sid0 < kSG ? nseeds - sid0 : kSG);
  const int tid = threadIdx.x;
  for (int i = tid; i < kSG * 6; i += 256) (&colsum[0][0])[i] = 0ull;
  const int64_t kmin = seed_k(R, a.chain, sid0);
  const int64_t kmax = seed_k(R, a.chain, sid0 + nS - 1);
  const uint64_t mask = b >= 64 ? ~0ull : ((1ull << b) - 1ull);
  const uint64_t fl = flip ? (1ull << (b - 1)) : 0ull;
  const bool split = b <= 48;
  // this CTA's slice of the t range
  int64_t tlo = kmin - lg + 1 > 0 ? kmin - lg + 1 : 0;
  int64_t thi = kmax < lf - 1 ? kmax : lf - 1;
  const int64_t s_lo = tlo + slice * kSlice;
  const int64_t s_hi = s_lo + kSlice - 1 < thi ? s_lo + kSlice - 1 : thi;
  if (s_lo > s_hi) return;  // the group's t range ends before this slice (uniform)
  if (split) {
    uint4 *sf = reinterpret_cast<uint4 *>(sraw);
    uint4 *sg = sf + kST;
    const int sub = tid & 63, sq = tid >> 6;
    int64_t kk[4];
#pragma unroll
    for (int u = 0; u < 4; u++) kk[u] = sq + 4 * u < nS ? seed_k(R, a.chain, sid0 + sq + 4 * u) : -1;
    unsigned long long ll[4] = {0, 0, 0, 0}, hh[4] = {0, 0, 0, 0}, ss[4] = {0, 0, 0, 0};
    for (int64_t t0 = s_lo; t0 <= s_hi; t0 += kST) {
      const int T = (int)(s_hi - t0 + 1 < kST ? s_hi - t0 + 1 : kST);
      const int64_t jlo = kmin - t0 - T + 1;
      const int W = (int)(kmax - kmin + T);
      // every global load of the chunk is issued before any of them is used
      uint64_t vf[kST / 256], vg[kSW / 256];
#pragma unroll
      for (int m = 0; m < kST / 256; m++) {
        const int i = tid + 256 * m;
        vf[m] = i < T ? f[(t0 + i) * in_limbs] : 0ull;
      }
#pragma unroll
      for (int m = 0; m < kSW / 256; m++) {
        const int i = tid + 256 * m;
        const int64_t j = jlo + i;
        vg[m] = (i < W && j >= 0 && j < lg) ? g[j * in_limbs] : 0ull;
      }
      __syncthreads();
#pragma unroll
      for (int m = 0; m < kST / 256; m++) {
        const int i = tid + 256 * m;
        if (i < T) sf[i] = split24((vf[m] & mask) ^ fl);
      }
#pragma unroll
      for (int m = 0; m < kSW / 256; m++) {
        const int i = tid + 256 * m;
        const int64_t j = jlo + i;
        if (i < W) sg[i] = split24((j >= 0 && j < lg) ? ((vg[m] & mask) ^ fl) : 0ull);
      }
      __syncthreads();
      int base[4];
#pragma unroll
      for (int u = 0; u < 4; u++) base[u] = kk[u] >= 0 ? (int)(kk[u] - t0 - jlo) : 0;
      for (int i = sub; i < T; i += 64) {
        const uint4 x = sf[i];
#pragma unroll
        for (int u = 0; u < 4; u++) {
          if (kk[u] >= 0) {
            const uint4 y = sg[base[u] - i];
            mad_wide(ll[u], x.x, y.x);
            mad_wide(hh[u], x.y, y.y);
            mad_wide(ss[u], x.z, y.z);
          }
        }
      }
    }
    // sums over the 64 threads of each seed: a shuffle tree in each of its two
    // warps, then red[seed][value][warp]
    __syncthreads();
    unsigned long long *red = reinterpret_cast<unsigned long long *>(sraw);
    const int half = (tid >> 5) & 1, lane = tid & 31;
#pragma unroll
    for (int u = 0; u < 4; u++) {
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) {
        ll[u] += __shfl_xor_sync(0xffffffffu, ll[u], off);
        hh[u] += __shfl_xor_sync(0xffffffffu, hh[u], off);
        ss[u] += __shfl_xor_sync(0xffffffffu, ss[u], off);
      }
      if (lane == 0) {
        const int sd = sq + 4 * u;
        red[(sd * 3 + 0) * 2 + half] = ll[u];
        red[(sd * 3 + 1) * 2 + half] = hh[u];
        red[(sd * 3 + 2) * 2 + half] = ss[u];
      }
    }
    __syncthreads();
    if (tid < nS) {
      const unsigned long long *q = red + tid * 6;
      const unsigned long long l = q[0] + q[1], hv = q[2] + q[3], sv = q[4] + q[5];
      // ll + (ss - ll - hh) 2^24 + hh 2^48 as 128 bits (the middle term is non-negative)
      const uint64_t mid = sv - l - hv;
      const uint64_t ml = mid << 24, mh = mid >> 40;
      const uint64_t hl = hv << 48, hhi = hv >> 16;
      uint64_t lo = l + ml;
      uint64_t hi = mh + hhi + (lo < ml);
      lo += hl;
      hi += lo < hl;
      colsum[tid][0] = (uint32_t)lo;
      colsum[tid][1] = (uint32_t)(lo >> 32);
      colsum[tid][2] = (uint32_t)hi;
      colsum[tid][3] = (uint32_t)(hi >> 32);
    }
  } else {
    uint64_t *sf = reinterpret_cast<uint64_t *>(sraw);
    uint64_t *sg = sf + kST;
    const int sl = tid >> 4, sub = tid & 15;
    const int64_t kk = sl < nS ? seed_k(R, a.chain, sid0 + sl) : -1;
    uint64_t a0 = 0, a1 = 0, a2 = 0;
    for (int64_t t0 = s_lo; t0 <= s_hi; t0 += kST) {
      const int T = (int)(s_hi - t0 + 1 < kST ? s_hi - t0 + 1 : kST);
      const int64_t jlo = kmin - t0 - T + 1;
      const int W = (int)(kmax - kmin + T);
      __syncthreads();
      for (int i = tid; i < T; i += 256) sf[i] = (f[(t0 + i) * in_limbs] & mask) ^ fl;
      for (int i = tid; i < W; i += 256) {
        const int64_t j = jlo + i;
        sg[i] = (j >= 0 && j < lg) ? ((g[j * in_limbs] & mask) ^ fl) : 0ull;
      }
      __syncthreads();
      if (kk >= 0) {
        // four independent 192-bit partial sums keep several products in flight
        uint64_t b0[4] = {0, 0, 0, 0}, b1[4] = {0, 0, 0, 0}, b2[4] = {0, 0, 0, 0};
        const int base = (int)(kk - t0 - jlo);  // sg index of t = t0
        int i = sub;
        for (; i + 48 < T; i += 64) {
#pragma unroll
          for (int u = 0; u < 4; u++) {
            const uint64_t x = sf[i + 16 * u];
            const uint64_t y = sg[base - i - 16 * u];
            const uint64_t lo = x * y, hi = __umul64hi(x, y);
            b0[u] += lo;
            const uint64_t h1 = hi + (b0[u] < lo);
            b1[u] += h1;
            b2[u] += b1[u] < h1;
          }
        }
        for (; i < T; i += 16) {
          const uint64_t x = sf[i];
          const uint64_t y = sg[base - i];
          const uint64_t lo = x * y, hi = __umul64hi(x, y);
          b0[0] += lo;
          const uint64_t h1 = hi + (b0[0] < lo);
          b1[0] += h1;
          b2[0] += b1[0] < h1;
        }
#pragma unroll
        for (int u = 0; u < 4; u++) {
          a0 += b0[u];
          const uint64_t c0 = a0 < b0[u];
          const uint64_t m = b1[u] + c0;
          const uint64_t c1 = m < c0;
          a1 += m;
          a2 += b2[u] + c1 + (a1 < m);
        }
      }
    }
    if (kk >= 0) {
      const uint32_t w6[6] = {(uint32_t)a0, (uint32_t)(a0 >> 32), (uint32_t)a1,
                              (uint32_t)(a1 >> 32), (uint32_t)a2, (uint32_t)(a2 >> 32)};
#pragma unroll
      for (int w = 0; w < 6; w++)
        if (w6[w]) atomicAdd(&colsum[sl][w], (unsigned long long)w6[w]);
    }
  }
  __syncthreads();
  if (tid < nS * 6) {
    const int sidx = tid / 6, w = tid % 6;
    const unsigned long long v = colsum[sidx][w];
    if (v) atomicAdd(acc + (R.seed_base + sid0 + sidx) * 6 + w, v);
  }
}

int make_seed_plan(uint32_t *seeds, int seed_words, unsigned long long *seed_acc,
                   const RecoverRun *runs, int nruns, int64_t chain, const uint64_t *f, int64_t lf,
                   const uint64_t *g, int64_t lg, int b, int in_limbs, int flip, SeedPlan &sp) {
  sp = SeedPlan{};
  int64_t n = 0;
  for (int r = 0; r < nruns; r++) n += 2 * (runs[r].nchains - 1);
  sp.nseeds = n;
  if (n == 0) return 0;
  if (seed_words > kMaxSeedWords) return -1;
  SeedArgs &a = sp.a;
  for (int r = 0; r < nruns; r++) a.run[r] = runs[r];
  a.nruns = nruns;
  a.chain = chain;
  a.seeds = seeds;
  a.seed_words = seed_words;
  a.f = f;
  a.g = g;
  a.lf = lf;
  a.lg = lg;
  a.b = b;
  a.in_limbs = in_limbs;
  a.flip = flip;
  sp.blocks = n;
  // blocked path when the seeds of a group lie close enough together
  bool blocked = b <= 64 && seed_words <= kAccSeedWords;
  for (int r = 0; r < nruns && blocked; r++)
    if (runs[r].kstride * (chain * (kSG / 2) + 1) + kST > kSW) blocked = false;
  if (blocked) {
    SeedBArgs &sb = sp.bl;
    int64_t groups = 0;
    for (int r = 0; r < nruns; r++) {
      sb.run[r] = runs[r];
      sb.groups[r] = (2 * (runs[r].nchains - 1) + kSG - 1) / kSG;
      groups += sb.groups[r];
    }
    sb.nruns = nruns;
    sb.chain = chain;
    const int64_t lmin = lf < lg ? lf : lg;
    // a group's t range is at most min(Lf, Lg) plus the spread of its k (< kSW)
    sb.slices = (lmin + kSW + kSlice - 1) / kSlice;
    sb.nseeds = n;
    sb.acc = seed_acc;
    sb.f = f;
    sb.g = g;
    sb.lf = lf;
    sb.lg = lg;
    sb.b = b;
    sb.in_limbs = in_limbs;
    sb.flip = flip;
    sp.kind = 1;
    sp.blocks = groups * sb.slices;
    return 0;
  }
  const int nw = (b + 31) / 32;
  if (b <= 64) {
    sp.kind = 2;
  } else {
    int cls = 2;
    while (cls < nw) cls *= 2;
    if (cls > 64) return -1;
    sp.kind = 100 + cls;  // word-count class of the templated kernel
  }
  return 0;
}

template <class Src>
static void launch_seed_kind(int kind, int64_t blocks, const Src &src, cudaStream_t s) {
  const unsigned grid = (unsigned)blocks;
  switch (kind) {
    case 2: seed_kernel64<Src><<<grid, kSeedThreads, 0, s>>>(src); break;
    case 102: seed_kernel<2, Src><<<grid, kSeedThreads, 0, s>>>(src); break;
    case 104: seed_kernel<4, Src><<<grid, kSeedThreads, 0, s>>>(src); break;
    case 108: seed_kernel<8, Src><<<grid, kSeedThreads, 0, s>>>(src); break;
    case 116: seed_kernel<16, Src><<<grid, kSeedThreads, 0, s>>>(src); break;
    case 132: seed_kernel<32, Src><<<grid, kSeedThreads, 0, s>>>(src); break;
    case 164: seed_kernel<64, Src><<<grid, kSeedThreads, 0, s>>>(src); break;
  }
}

cudaError_t launch_seed_plan(const SeedPlan &sp, cudaStream_t s) {
  if (sp.nseeds == 0) return cudaSuccess;
  if (sp.kind == 1) {
    if (!sp.acc_cleared) {
      cudaError_t e = cudaMemsetAsync(sp.bl.acc, 0, (size_t)sp.nseeds * 6 * 8, s);
      if (e != cudaSuccess) return e;
    }
    const One<SeedBArgs> one{sp.bl};
    seed_blocked64<One<SeedBArgs>><<<(unsigned)sp.blocks, 256, 0, s>>>(one);
    note_launches(1);
  } else {
    launch_seed_kind(sp.kind, sp.blocks, One<SeedArgs>{sp.a}, s);
    note_launches(1);
  }
  return cudaGetLastError();
}

// batches: blocked (kind 1) products, then per kind the others
cudaError_t launch_seeds_blocked_batch(const SeedBArgs *d, const int64_t *prefix_blocks, int n,
                                       int64_t blocks, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  seed_blocked64<Many<SeedBArgs>><<<(unsigned)blocks, 256, 0, s>>>(
      Many<SeedBArgs>{d, prefix_blocks, n});
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_seeds_kind_batch(int kind, const SeedArgs *d, const int64_t *prefix, int n,
                                    int64_t blocks, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  launch_seed_kind(kind, blocks, Many<SeedArgs>{d, prefix, n}, s);
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
// sequential; chains of `chain` steps run in parallel, chain c starting at
// s = c * chain from the exact seeds h'_(s-1), h'_s: alpha_(s-1), alpha_s,
// beta_(s-1) follow directly, and delta_(s-1) = u_s - beta_(s-1) - alpha_s
// (mod X, necessarily 0 or 1) gives delta_s = (beta_(s-1) + alpha_s +
// delta_(s-1) - u_s) / X.
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
// out limbs of alpha + 2^M beta
__device__ void write_coeff(uint64_t *out, int ol, const Dig &al, const Dig &be, int M) {
  const int W = (M + 31) / 32;
  for (int l = 0; l < ol; l++) {
    uint64_t v = 0;
    for (int half = 0; half < 2; half++) {
      const int64_t p0 = 64 * (int64_t)l + 32 * half;  // bit position of this 32-bit chunk
      uint64_t chunk = 0;
      // from alpha: bits [p0, p0+32) below M
      if (p0 < M) {
        const int wi = (int)(p0 >> 5);
        uint32_t x = al.w[wi];
        chunk |= x;  // alpha's bits above M are zero
      }
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
    out[l] = v;
  }
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
// Seed value i of a run as kAccSeedWords 32-bit words (the top ones zero): the
// finished seed words, or carried from the blocked seed kernel's 64-bit column sums
// (nw <= kAccSeedWords there).
__device__ __forceinline__ void seed_value(const RecoverRun &R, int64_t i, int nw,
                                           uint32_t (&out)[kAccSeedWords]) {
  if (R.seed_acc != nullptr) {
    const unsigned long long *acc = R.seed_acc + i * 6;
    unsigned long long carry = 0;
#pragma unroll
    for (int w = 0; w < kAccSeedWords; w++) {
      const unsigned long long v = (w < 6 ? acc[w] : 0ull) + carry;
      out[w] = w < nw ? (uint32_t)v : 0u;
      carry = v >> 32;
    }
  } else {
#pragma unroll
    for (int w = 0; w < kAccSeedWords; w++) out[w] = w < nw ? R.seeds[i * nw + w] : 0u;
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
// out limbs of alpha + 2^M beta, alpha, beta < 2^M
__device__ __forceinline__ void write_h1(uint64_t *out, int ol, uint64_t a, uint64_t be, int M) {
  out[0] = a | (be << M);
  if (ol > 1) out[1] = be >> (64 - M);
  for (int l = 2; l < ol; l++) out[l] = 0;
}
__device__ __forceinline__ void write_h2(uint64_t *out, int ol, D2 a, D2 be, int M) {
  uint64_t s[5] = {a.lo, a.hi, 0, 0, 0};
  const int r = M & 63;  // beta starts in limb 1 (64 <= M < 128)
  s[1] |= be.lo << r;
  s[2] |= (r ? (be.lo >> (64 - r)) : 0ull) | (be.hi << r);
  s[3] |= r ? (be.hi >> (64 - r)) : 0ull;
  for (int l = 0; l < ol; l++) out[l] = l < 5 ? s[l] : 0ull;
}

__device__ __forceinline__ bool chain_index(const RecoverArgs &a, int64_t &gid, int &r) {
  r = 0;
  while (r < a.nruns && gid >= a.run[r].nchains) {
    gid -= a.run[r].nchains;
    r++;
  }
  return r < a.nruns;
}

// ---- bulk copies into shared memory (one thread issues, all wait, bounded)
__device__ __forceinline__ uint32_t smem_addr(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void stage_init(uint64_t *bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(bar)) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void stage_expect(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void stage_copy(void *dst, const void *src, uint32_t bytes,
                                           uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}
// wait for phase 0 of the barrier, about one second at most; false on timeout
__device__ __forceinline__ bool stage_wait(uint64_t *bar) {
  uint64_t t0;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
  for (;;) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar))
        : "memory");
    if (ok) return true;
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    if (t - t0 > 1000000000ull) return false;
  }
}

// M <= 63, digits staged in shared memory.  A CTA of 128 threads runs cpc
// consecutive chains of one run (cpc <= 32, cpc * chain <= 2048):
//  1. one bulk copy of the bit ranges of V_f and V_r those chains read (the
//     chains are contiguous, so are their digits);
//  2. all threads extract the digits u_j, w_m into 64-bit arrays;
//  3. warp 0, one lane per chain, runs the recurrence of Sec. 3.2 from shared
//     memory and stages the coefficients;
//  4. all threads write the coefficients out.
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
// digits of one string, [step t in 0..chain][lane]: lanes read consecutive words
__host__ __device__ __forceinline__ int64_t staged_digits(int64_t chain, int cpc) {
  return (chain + 1) * cpc;
}
__host__ __device__ __forceinline__ int64_t staged_bytes(int64_t chain, int M, int cpc) {
  return 2 * staged_words(chain, M, cpc) * 4 + 2 * staged_digits(chain, cpc) * 8 +
         cpc * chain * 2 * 8;
}

template <class Src>
__global__ void __launch_bounds__(kRT) recover_staged1(Src src) {
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
  const int M = a.M, ol = a.ol;
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
    if (tid == 0) atomicExch(status, 3);  // not for a plan from make_recover_args
    return;
  }
  uint32_t *su = stg, *sw = stg + capw;
  // [t][lane] layouts: du(t, i) = u_(s_i + t), dw(t, i) = w_(n - s_i - t) with
  // s_i = j0 + i chain (t = chain reaches the next chain's start), so(t, i) =
  // coefficient s_i + t
  uint64_t *du = reinterpret_cast<uint64_t *>(stg + 2 * capw);
  uint64_t *dw = du + capd;
  uint64_t *so = dw + capd;
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
  __syncthreads();
  if (!__syncthreads_and(stage_wait(&bar))) {
    if (tid == 0) atomicExch(status, 1);
    stage_wait(&bar);  // once more (bounded) for the copies in flight before leaving
    return;
  }
  // 2. digits (chain and cpc are powers of two)
  const int lc = __ffsll((long long)chain) - 1, lp = __ffs(cpc) - 1;
  const int64_t pu = R.off_f - ub0 * 32, pw = R.off_r - wb0 * 32;  // staged bit offsets
  for (int q = tid; q < (int)capd; q += kRT) {
    const int t = q >> lp, i = q & (cpc - 1);
    const int64_t j = j0 + ((int64_t)i << lc) + t;
    const bool in = j <= jhi;
    du[q] = in ? sbits64(su, nu, pu + j * (int64_t)M) & mask : 0ull;
    dw[q] = in ? sbits64(sw, nw, pw + (n - j) * (int64_t)M) & mask : 0ull;
  }
  __syncthreads();
  // 3. the chains (warp 0)
  const int64_t gid = c0 + tid;
  if (tid < 32 && gid < c1) {
    const int64_t ln = tid;
    auto u = [&](int64_t j) { return du[(j - j0 - (ln << lc)) * cpc + ln]; };
    auto w = [&](int64_t m) { return dw[(n - m - j0 - (ln << lc)) * cpc + ln]; };
    const int64_t s = gid * chain;
    const int64_t e = (s + chain < n) ? s + chain : n;
    uint64_t a_prev, a_cur, delta;
    if (s == 0) {
      a_prev = 0;
      a_cur = u(0);
      delta = 0;
    } else {
      uint32_t s0[kAccSeedWords], s1[kAccSeedWords];
      seed_value(R, R.seed_base + 2 * (gid - 1), a.seed_words, s0);
      seed_value(R, R.seed_base + 2 * (gid - 1) + 1, a.seed_words, s1);
      a_prev = load_d1(s0, kAccSeedWords, 0, M);
      const uint64_t b_prev = load_d1(s0, kAccSeedWords, M, M);
      a_cur = load_d1(s1, kAccSeedWords, 0, M);
      const uint64_t us = u(s);
      const uint64_t dprev = (us - b_prev - a_cur) & mask;
      if (dprev > 1) atomicExch(status, 2);
      delta = (b_prev + a_cur + dprev - us) >> M;
    }
    uint64_t w_cur = w(n - s);
    // step t reads du(t + 1, ln) and dw(t + 1, ln); eight steps are loaded ahead
    const uint64_t *pdu = du + cpc + ln, *pdw = dw + cpc + ln;
    uint64_t *po = so + 2 * ln;
    constexpr int kAhead = 8;
    uint64_t ub[kAhead], wb[kAhead];
#pragma unroll
    for (int q = 0; q < kAhead; q++) {
      ub[q] = q < chain ? pdu[q * cpc] : 0ull;
      wb[q] = q < chain ? pdw[q * cpc] : 0ull;
    }
    for (int64_t j = s; j < e; j++) {
      const int t = (int)(j - s);
      uint64_t *out = po + 2 * t * cpc;
      const uint64_t u_next = ub[0], w_next = wb[0];
#pragma unroll
      for (int q = 0; q + 1 < kAhead; q++) {
        ub[q] = ub[q + 1];
        wb[q] = wb[q + 1];
      }
      ub[kAhead - 1] = t + kAhead < chain ? pdu[(t + kAhead) * cpc] : 0ull;
      wb[kAhead - 1] = t + kAhead < chain ? pdw[(t + kAhead) * cpc] : 0ull;
      if (j <= n - 2) {
        const uint64_t eps = a_cur > w_next ? 1ull : 0ull;
        const uint64_t beta = (w_cur - a_prev - eps) & mask;
        const uint64_t a_next = (u_next - beta - delta) & mask;
        const uint64_t dnext = (beta + a_next + delta - u_next) >> M;
        if (dnext > 1) atomicExch(status, 2);
        out[0] = a_cur | (beta << M);
        out[1] = beta >> (64 - M);
        a_prev = a_cur;
        a_cur = a_next;
        delta = dnext;
        w_cur = w_next;
      } else {
        const uint64_t beta = (w_cur - a_prev) & mask;
        out[0] = a_cur | (beta << M);
        out[1] = beta >> (64 - M);
      }
    }
  }
  __syncthreads();
  // 4. coefficients out
  uint64_t *h = a.h;
  uint64_t *hb = h + (R.kbase + R.kstride * j0) * ol;
  const int64_t hs = R.kstride * ol;
  for (int q = tid; q < (int)((jhi - j0) * ol); q += kRT) {
    const int jj = ol == 2 ? q >> 1 : q;
    const int l = q - jj * ol;
    const int i = jj >> lc, t = jj & (int)(chain - 1);
    hb[jj * hs + l] = so[((t << lp) + i) * 2 + l];
  }
}

// 64 <= M <= 127
template <class Src>
__global__ void __launch_bounds__(128) recover_kernel2(Src src) {
  int64_t local;
  const RecoverArgs &a = src.locate(blockIdx.x, local);
  uint64_t *h = a.h;
  const int ol = a.ol;
  int *status = a.status;
  int64_t gid = local * 128 + threadIdx.x;
  int r;
  if (!chain_index(a, gid, r)) return;
  const RecoverRun &R = a.run[r];
  const int M = a.M;
  const int64_t n = R.n;
  const int64_t s = gid * a.chain;
  const int64_t e = (s + a.chain < n) ? s + a.chain : n;
  const D2 zero = {0ull, 0ull};
  D2 a_prev, a_cur;
  uint64_t delta;
  if (s == 0) {
    a_prev = zero;
    a_cur = load_d2(R.Vf, a.nwords, R.off_f, M);
    delta = 0;
  } else {
    uint32_t s0[kAccSeedWords], s1[kAccSeedWords];
    seed_value(R, R.seed_base + 2 * (gid - 1), a.seed_words, s0);
    seed_value(R, R.seed_base + 2 * (gid - 1) + 1, a.seed_words, s1);
    a_prev = load_d2(s0, kAccSeedWords, 0, M);
    const D2 b_prev = load_d2(s0, kAccSeedWords, M, M);
    a_cur = load_d2(s1, kAccSeedWords, 0, M);
    const D2 us = load_d2(R.Vf, a.nwords, R.off_f + s * (int64_t)M, M);
    const D2 dprev = sub_d2(sub_d2(us, b_prev, 0, M), a_cur, 0, M);
    if (dprev.hi != 0 || dprev.lo > 1) atomicExch(status, 2);
    delta = carry_d2(b_prev, a_cur, dprev.lo & 1ull, M);
  }
  D2 w_cur = load_d2(R.Vr, a.nwords, R.off_r + (n - s) * (int64_t)M, M);
  for (int64_t j = s; j < e; j++) {
    uint64_t *out = h + (R.kbase + R.kstride * j) * ol;
    if (j <= n - 2) {
      const D2 w_next = load_d2(R.Vr, a.nwords, R.off_r + (n - j - 1) * (int64_t)M, M);
      const uint64_t eps = gt_d2(a_cur, w_next) ? 1ull : 0ull;
      const D2 beta = sub_d2(sub_d2(w_cur, a_prev, 0, M), zero, eps, M);
      const D2 u_next = load_d2(R.Vf, a.nwords, R.off_f + (j + 1) * (int64_t)M, M);
      const D2 a_next = sub_d2(sub_d2(u_next, beta, 0, M), zero, delta, M);
      const uint64_t dnext = carry_d2(beta, a_next, delta, M);
      write_h2(out, ol, a_cur, beta, M);
      a_prev = a_cur;
      a_cur = a_next;
      delta = dnext;
      w_cur = w_next;
    } else {
      write_h2(out, ol, a_cur, sub_d2(w_cur, a_prev, 0, M), M);
    }
  }
}

template <class Src>
__global__ void __launch_bounds__(64) recover_wide(Src src) {
  int64_t local;
  const RecoverArgs &a = src.locate(blockIdx.x, local);
  uint64_t *h = a.h;
  const int ol = a.ol;
  int *status = a.status;
  int64_t gid = local * 64 + threadIdx.x;
  int r = 0;
  while (r < a.nruns && gid >= a.run[r].nchains) {
    gid -= a.run[r].nchains;
    r++;
  }
  if (r >= a.nruns) return;
  const RecoverRun &R = a.run[r];
  const int M = a.M;
  const int W = (M + 31) / 32;
  const int64_t n = R.n;
  const int64_t s = gid * a.chain;
  const int64_t e = (s + a.chain < n) ? s + a.chain : n;
  Dig a_prev, a_cur, delta_d, w_cur, w_next, u_next, beta, a_next, zero;
  for (int i = 0; i < W; i++) zero.w[i] = 0;
  uint32_t delta;
  if (s == 0) {
    a_prev = zero;
    dig_load(a_cur, R.Vf, a.nwords, R.off_f, M);
    delta = 0;
  } else {
    Dig b_prev, us, dp;
    if (R.seed_acc != nullptr) {
      uint32_t s0[kAccSeedWords], s1[kAccSeedWords];
      seed_value(R, R.seed_base + 2 * (gid - 1), a.seed_words, s0);
      seed_value(R, R.seed_base + 2 * (gid - 1) + 1, a.seed_words, s1);
      dig_load_local(a_prev, s0, kAccSeedWords, 0, M);
      dig_load_local(b_prev, s0, kAccSeedWords, M, M);
      dig_load_local(a_cur, s1, kAccSeedWords, 0, M);
    } else {
      const uint32_t *sd = R.seeds + (R.seed_base + 2 * (gid - 1)) * a.seed_words;
      dig_load_local(a_prev, sd, a.seed_words, 0, M);
      dig_load_local(b_prev, sd, a.seed_words, M, M);
      dig_load_local(a_cur, sd + a.seed_words, a.seed_words, 0, M);
    }
    dig_load(us, R.Vf, a.nwords, R.off_f + s * (int64_t)M, M);
    Dig t1;
    dig_sub(t1, us, b_prev, 0, M);
    dig_sub(dp, t1, a_cur, 0, M);
    bool ok = dp.w[0] <= 1;
    for (int i = 1; i < W; i++) ok = ok && dp.w[i] == 0;
    if (!ok) atomicExch(status, 2);
    delta = dig_add_carry(b_prev, a_cur, dp.w[0] & 1u, M);
  }
  (void)delta_d;
  dig_load(w_cur, R.Vr, a.nwords, R.off_r + (n - s) * (int64_t)M, M);
  for (int64_t j = s; j < e; j++) {
    uint64_t *out = h + (R.kbase + R.kstride * j) * ol;
    if (j <= n - 2) {
      dig_load(w_next, R.Vr, a.nwords, R.off_r + (n - j - 1) * (int64_t)M, M);
      const uint32_t eps = dig_gt(a_cur, w_next, W) ? 1u : 0u;
      dig_sub(beta, w_cur, a_prev, eps, M);
      dig_load(u_next, R.Vf, a.nwords, R.off_f + (j + 1) * (int64_t)M, M);
      dig_sub(a_next, u_next, beta, delta, M);
      const uint32_t dnext = dig_add_carry(beta, a_next, delta, M);
      write_coeff(out, ol, a_cur, beta, M);
      a_prev = a_cur;
      a_cur = a_next;
      delta = dnext;
      w_cur = w_next;
    } else {
      dig_sub(beta, w_cur, a_prev, 0, M);
      write_coeff(out, ol, a_cur, beta, M);
    }
  }
}

int make_recover_args(uint64_t *h, int ol, const RecoverRun *runs, int nruns, int64_t nwords,
                      int M, int64_t chain, int seed_words, int *status, RecoverArgs &a,
                      int64_t &blocks) {
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
  a.seed_words = seed_words;
  a.h = h;
  a.ol = ol;
  a.status = status;
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
    recover_staged1<Src><<<(unsigned)blocks, kRT, smem, s>>>(src);
  } else if (cls == 2)
    recover_kernel2<Src><<<(unsigned)blocks, 128, 0, s>>>(src);
  else
    recover_wide<Src><<<(unsigned)blocks, 64, 0, s>>>(src);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_recover(uint64_t *h, int ol, const RecoverRun *runs, int nruns,
                           int64_t nwords, int M, int64_t chain, int seed_words, int *status,
                           cudaStream_t s) {
  RecoverArgs a;
  int64_t blocks;
  if (make_recover_args(h, ol, runs, nruns, nwords, M, chain, seed_words, status, a, blocks) != 0)
    return cudaErrorInvalidValue;
  if (blocks == 0) return cudaSuccess;
  return launch_recover_class(recover_class(M), blocks, One<RecoverArgs>{a}, a.smem, s);
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
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < lh;
       k += (int64_t)gridDim.x * blockDim.x) {
    uint64_t r = 0;
    for (int l = ol - 1; l >= 0; l--) r = mod_128(r, h[k * ol + l], p);
    out[k] = r;
  }
}

cudaError_t launch_reduce_mod(uint64_t *out, const uint64_t *h, int ol, int64_t lh, uint64_t p,
                              cudaStream_t s) {
  reduce_mod_kernel<<<grid_for(lh, 256), 256, 0, s>>>(out, h, ol, lh, p);
  note_launches(1);
  return cudaGetLastError();
}

}  // namespace ks
