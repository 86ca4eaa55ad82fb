// Carry normalization (and the +- combine of Sec. 3.3 / 3.4):
//
//   V = sum_k (c1_k + sigma c2_k) 2^(d k)   ->   32-bit words of V
//
// where c1, c2 are the signed 64-bit column sums of one or two sub-products.
// With sigma = +1 and sigma = -1 this yields P+ + P- = 2 h0(X^2) and
// P+ - P- = 2X h1(X^2) directly (Sec. 3.3), so the combine costs no pass of
// its own.  Steps, all exact:
//
//  1. slice: every column value times 2^(dk mod 32) is a 96-bit two's
//     complement number; its three 32-bit slices land in words q, q+1, q+2
//     (q = floor(dk/32)).  T_j = sum of the slices landing in word j
//     (|T_j| < 2^38).
//  2. fold: s_j = (T_j mod 2^32) + floor(T_(j-1) / 2^32), so that
//     V = sum_j s_j 2^(32j) with s_j in [-2^7, 2^32 + 2^7).
//  3. carry-lookahead: the carry into word j is in {-1, 0, 1}; word j maps an
//     incoming carry c to floor((s_j + c) / 2^32), a function on the three
//     carry values.  Functions compose associatively, so the carries are a
//     parallel prefix: warp shuffles, then the block, then the tiles (one
//     tile = 512 words per CTA), then a second pass applies them.
#include "ks_internal.cuh"
#include "ks_src.cuh"

namespace ks {

namespace {
constexpr int kThreads = 128;
constexpr int kWPT = 4;                     // words per thread
constexpr int kTileWords = kThreads * kWPT; // words per tile
constexpr uint32_t kIdentity = 0u | (1u << 2) | (2u << 4);

// carry-transfer function: 2 bits per input carry c in {-1,0,1}, value c'+1
__device__ __forceinline__ int apply_fn(uint32_t f, int c) {
  return (int)((f >> (2 * (c + 1))) & 3u) - 1;
}
// g after f
__device__ __forceinline__ uint32_t compose(uint32_t g, uint32_t f) {
  uint32_t h = 0;
#pragma unroll
  for (int c = -1; c <= 1; c++) h |= (uint32_t)(apply_fn(g, apply_fn(f, c)) + 1) << (2 * (c + 1));
  return h;
}
__device__ __forceinline__ uint32_t word_fn(int64_t s) {
  uint32_t h = 0;
#pragma unroll
  for (int c = -1; c <= 1; c++) h |= (uint32_t)(((s + c) >> 32) + 1) << (2 * (c + 1));
  return h;
}

__device__ __forceinline__ int64_t column(const NormJob &J, int64_t k) {
  int64_t v = 0;
  if (k < J.n1) v = J.c1[k];
  if (J.c2 != nullptr && k < J.n2) v += (J.sigma > 0) ? J.c2[k] : -J.c2[k];
  return v;
}

// T_j: the slices of all column values that land in word j.
__device__ int64_t slice_sum(const NormJob &J, int d, int64_t j) {
  if (j < 0) return 0;
  const int64_t ncol = J.n1 > J.n2 ? J.n1 : J.n2;
  int64_t kmin = (j >= 2) ? (32 * (j - 2) + d - 1) / d : 0;
  int64_t kmax = (32 * j + 31) / d;
  if (kmax > ncol - 1) kmax = ncol - 1;
  int64_t T = 0;
  for (int64_t k = kmin; k <= kmax; k++) {
    const int64_t bit = (int64_t)d * k;
    const int64_t q = bit >> 5;
    if (q < j - 2 || q > j) continue;
    const __int128 x = (__int128)column(J, k) << (int)(bit & 31);
    if (q == j)
      T += (int64_t)(uint32_t)x;
    else if (q == j - 1)
      T += (int64_t)(uint32_t)(x >> 32);
    else
      T += (int64_t)(int32_t)(uint32_t)(x >> 64);
  }
  return T;
}

// s_j for the kWPT words of this thread, and their composed transfer function.
__device__ uint32_t thread_words(const NormJob &J, int d, int64_t j0, int64_t s[kWPT]) {
  int64_t Tprev = slice_sum(J, d, j0 - 1);
  uint32_t agg = kIdentity;
#pragma unroll
  for (int w = 0; w < kWPT; w++) {
    const int64_t T = slice_sum(J, d, j0 + w);
    s[w] = (int64_t)(uint32_t)T + (Tprev >> 32);
    Tprev = T;
    agg = compose(word_fn(s[w]), agg);
  }
  return agg;
}

// Block-wide exclusive scan of transfer functions (thread order); returns the
// exclusive prefix of this thread and writes the block total.
__device__ uint32_t block_exclusive(uint32_t v, uint32_t *total) {
  __shared__ uint32_t warp_tot[kThreads / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  uint32_t incl = v;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    uint32_t o = __shfl_up_sync(0xffffffffu, incl, off);
    if (lane >= off) incl = compose(incl, o);
  }
  uint32_t excl = __shfl_up_sync(0xffffffffu, incl, 1);
  if (lane == 0) excl = kIdentity;
  if (lane == 31) warp_tot[wid] = incl;
  __syncthreads();
  uint32_t wpre = kIdentity;
  for (int w = 0; w < wid; w++) wpre = compose(warp_tot[w], wpre);
  if (total != nullptr) {
    uint32_t t = kIdentity;
    for (int w = 0; w < kThreads / 32; w++) t = compose(warp_tot[w], t);
    *total = t;
  }
  return compose(excl, wpre);
}

template <class Src>
__global__ void __launch_bounds__(kThreads) norm_aggregate(Src src) {
  int64_t bid;
  const NormArgs &a = src.locate(blockIdx.x, bid);
  const NormJob &J = a.job[bid / a.ntiles];
  const int64_t tile = bid % a.ntiles;
  const int64_t j0 = tile * kTileWords + (int64_t)threadIdx.x * kWPT;
  int64_t s[kWPT];
  const uint32_t agg = thread_words(J, a.d, j0, s);
  uint32_t total;
  block_exclusive(agg, &total);
  if (threadIdx.x == 0) J.agg[tile] = (uint8_t)total;
}

// One CTA per job: carries into every tile (the first tile gets 0), by a
// parallel prefix of the tile functions (each thread composes a run of tiles,
// then warp shuffles and one more level across the warps).
template <class Src>
__global__ void __launch_bounds__(1024) norm_tiles(Src src) {
  int64_t jid;
  const NormArgs &a = src.locate(blockIdx.x, jid);
  const NormJob &J = a.job[jid];
  __shared__ uint32_t wtot[32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int64_t per = (a.ntiles + 1023) / 1024;
  const int64_t t0 = (int64_t)threadIdx.x * per;
  uint32_t f = kIdentity;
  for (int64_t t = t0; t < t0 + per && t < a.ntiles; t++) f = compose(J.agg[t], f);
  uint32_t incl = f;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const uint32_t o = __shfl_up_sync(0xffffffffu, incl, off);
    if (lane >= off) incl = compose(incl, o);
  }
  uint32_t excl = __shfl_up_sync(0xffffffffu, incl, 1);
  if (lane == 0) excl = kIdentity;
  if (lane == 31) wtot[wid] = incl;
  __syncthreads();
  if (wid == 0) {
    uint32_t v = wtot[lane];
    uint32_t wi = v;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const uint32_t o = __shfl_up_sync(0xffffffffu, wi, off);
      if (lane >= off) wi = compose(wi, o);
    }
    uint32_t we = __shfl_up_sync(0xffffffffu, wi, 1);
    if (lane == 0) we = kIdentity;
    wtot[lane] = we;
  }
  __syncthreads();
  int c = apply_fn(compose(excl, wtot[wid]), 0);
  for (int64_t t = t0; t < t0 + per && t < a.ntiles; t++) {
    J.cin[t] = (int8_t)c;
    c = apply_fn(J.agg[t], c);
  }
}

template <class Src>
__global__ void __launch_bounds__(kThreads) norm_apply(Src src) {
  int64_t bid;
  const NormArgs &a = src.locate(blockIdx.x, bid);
  const NormJob &J = a.job[bid / a.ntiles];
  const int64_t tile = bid % a.ntiles;
  const int64_t j0 = tile * kTileWords + (int64_t)threadIdx.x * kWPT;
  int64_t s[kWPT];
  const uint32_t agg = thread_words(J, a.d, j0, s);
  const uint32_t pre = block_exclusive(agg, nullptr);
  int c = apply_fn(pre, (int)J.cin[tile]);
#pragma unroll
  for (int w = 0; w < kWPT; w++) {
    const int64_t v = s[w] + c;
    if (j0 + w < a.nwords) J.out[j0 + w] = (uint32_t)v;
    c = (int)(v >> 32);
  }
}

}  // namespace

int make_norm_args(const NormJob *jobs, int njobs, int d, int64_t nwords, int64_t ntiles,
                   NormArgs &a) {
  if (njobs < 1 || njobs > 4) return -1;
  if (ntiles * kTileWords < nwords) return -1;
  a = NormArgs{};
  for (int i = 0; i < njobs; i++) a.job[i] = jobs[i];
  a.njobs = njobs;
  a.d = d;
  a.nwords = nwords;
  a.ntiles = ntiles;
  return 0;
}

cudaError_t launch_normalize(const NormJob *jobs, int njobs, int d, int64_t nwords,
                             int64_t ntiles, cudaStream_t s) {
  NormArgs a;
  if (make_norm_args(jobs, njobs, d, nwords, ntiles, a) != 0) return cudaErrorInvalidValue;
  const One<NormArgs> one{a};
  norm_aggregate<One<NormArgs>><<<(unsigned)(ntiles * njobs), kThreads, 0, s>>>(one);
  norm_tiles<One<NormArgs>><<<njobs, 1024, 0, s>>>(one);
  norm_apply<One<NormArgs>><<<(unsigned)(ntiles * njobs), kThreads, 0, s>>>(one);
  note_launches(3);
  return cudaGetLastError();
}

// prefix_tiles: block prefix over njobs * ntiles; prefix_jobs: over njobs
cudaError_t launch_normalize_batch(const NormArgs *d, const int64_t *prefix_tiles,
                                   const int64_t *prefix_jobs, int n, int64_t tiles,
                                   int64_t jobs, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  norm_aggregate<Many<NormArgs>><<<(unsigned)tiles, kThreads, 0, s>>>(
      Many<NormArgs>{d, prefix_tiles, n});
  norm_tiles<Many<NormArgs>><<<(unsigned)jobs, 1024, 0, s>>>(Many<NormArgs>{d, prefix_jobs, n});
  norm_apply<Many<NormArgs>><<<(unsigned)tiles, kThreads, 0, s>>>(
      Many<NormArgs>{d, prefix_tiles, n});
  note_launches(3);
  return cudaGetLastError();
}

int64_t norm_tiles_for(int64_t nwords) { return (nwords + kTileWords - 1) / kTileWords; }

}  // namespace ks
