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
//     parallel prefix: warp shuffles, then the block, then across tiles.
//
// One launch does all of it (a single-pass scan with decoupled look-back).
// Every CTA takes the next tile index from a counter, so the tiles it looks
// back on were claimed by CTAs that are already running.  It stages the
// columns its tile needs in shared memory (one coalesced read of the column
// sums; a thread's words are exactly its columns' bit span, so all slicing
// offsets are compile-time constants of the digit width), forms s_j, scans
// its tile, publishes the tile's transfer
// function, and then one warp looks back over the preceding tiles' flags
// (32 tiles per step) until it meets a tile that has published its carry-out;
// it then publishes its own carry-out, and the CTA writes its words.  The ±
// pair of a two- or four-point product (same c1, c2, opposite sigma) is done
// by one CTA from one staged copy of c1 and c2, so those columns are read once.
// A tile whose composed transfer function is constant publishes its
// carry-out before looking back (it does not depend on the carry in), which
// keeps the look-back short whatever the number of tiles in flight.
// Flags and the counter must be zero before the launch; every wait is bounded
// (about one second), after which the kernel records status 1 and finishes
// with carry 0.
#include "ks_internal.cuh"
#include "ks_src.cuh"

namespace ks {

namespace {
constexpr int kThreads = 128;
constexpr uint32_t kIdentity = 0u | (1u << 2) | (2u << 4);
constexpr uint32_t kFlagAgg = 1u << 8;      // the tile's transfer function is published
constexpr uint32_t kFlagPre = 1u << 9;      // the tile's carry-out is published
constexpr uint64_t kWaitNs = 1000000000ull;

// Per digit width D: every thread takes WPT words = 32 WPT bits = CPT columns
// exactly (32 WPT = D CPT), so each column sits at a compile-time bit offset
// from the thread's first word; BACK earlier columns still reach its first
// word or the word before it (their slices span three words).
template <int D>
struct Geo;
template <>
struct Geo<16> {
  static constexpr int WPT = 4, CPT = 8, BACK = 6;
};
template <>
struct Geo<28> {
  static constexpr int WPT = 7, CPT = 8, BACK = 3;
};
// staged columns of a tile: 128 CPT + BACK, one padding slot per 8 (banks)
constexpr int kStage = (kThreads * 8 + 8) + (kThreads * 8 + 8) / 8 + 8;
__device__ __forceinline__ int pad8(int i) { return i + (i >> 3); }

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
// two functions side by side (bits 0-5 and 8-13), composed lane-wise
__device__ __forceinline__ uint32_t compose2(uint32_t g, uint32_t f) {
  return compose(g & 63u, f & 63u) | (compose((g >> 8) & 63u, (f >> 8) & 63u) << 8);
}

__device__ __forceinline__ uint64_t globaltimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ uint32_t ld_acquire(const uint32_t *p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(uint32_t *p, uint32_t v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Looks back from `tile` over the flags of the preceding tiles (one warp, 32
// tiles per step) and returns the carry into `tile`; publishes the tile's
// carry-out.  `total` is the tile's own transfer function.
__device__ int look_back(uint32_t *flags, int64_t tile, uint32_t total, int lane, int *status) {
  if (tile == 0) {
    if (lane == 0) st_release(&flags[0], kFlagPre | (uint32_t)(apply_fn(total, 0) + 1));
    return 0;
  }
  // A tile whose transfer function is constant (some word in it absorbs any
  // incoming carry, the usual case) knows its carry-out already: publish it
  // at once, so that the next tile never has to look past this one.
  const int out_m = apply_fn(total, -1), out_z = apply_fn(total, 0);
  const bool constant = out_m == out_z && out_z == apply_fn(total, 1);
  if (lane == 0)
    st_release(&flags[tile], constant ? (kFlagPre | (uint32_t)(out_z + 1)) : (kFlagAgg | total));
  uint32_t acc = kIdentity;  // the functions of the tiles passed so far
  int64_t top = tile - 1;
  uint64_t t0 = 0;
  int cin = 0;
  while (true) {
    const int64_t ti = top - lane;
    // lanes before tile 0 read as "carry-out 0"; tile 0 always publishes one
    const uint32_t v = ti >= 0 ? ld_acquire(&flags[ti]) : (kFlagPre | 1u);
    const unsigned pre = __ballot_sync(0xffffffffu, (v & kFlagPre) != 0);
    const unsigned ready = __ballot_sync(0xffffffffu, (v & (kFlagPre | kFlagAgg)) != 0);
    const int fp = pre ? __ffs(pre) - 1 : 32;  // nearest tile with a carry-out
    const unsigned need = fp == 32 ? 0xffffffffu : ((1u << fp) - 1u);
    if ((ready & need) != need) {
      if (t0 == 0) {
        t0 = globaltimer();
      } else if (globaltimer() - t0 > kWaitNs) {
        if (lane == 0) atomicExch(status, 1);
        cin = 0;
        break;
      }
      __nanosleep(32);
      continue;
    }
    // compose the functions of lanes 0 .. fp-1 (lane 0 is the latest tile)
    uint32_t f = lane < fp ? (v & 63u) : kIdentity;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const uint32_t o = __shfl_down_sync(0xffffffffu, f, off);
      if (lane + off < 32) f = compose(f, o);
    }
    f = __shfl_sync(0xffffffffu, f, 0);
    acc = compose(acc, f);
    if (fp < 32) {
      const uint32_t vp = __shfl_sync(0xffffffffu, v, fp);
      cin = apply_fn(acc, (int)(vp & 3u) - 1);
      break;
    }
    top -= 32;
    t0 = 0;
  }
  if (lane == 0 && !constant)
    st_release(&flags[tile], kFlagPre | (uint32_t)(apply_fn(total, cin) + 1));
  return cin;
}

// s_j of a thread's WPT words from its BACK + CPT staged columns (x[i] is
// column kstart - BACK + i); every offset and shift is a compile-time constant.
template <int D>
__device__ __forceinline__ void thread_words(const int64_t (&x)[Geo<D>::BACK + Geo<D>::CPT],
                                             int64_t (&s)[Geo<D>::WPT]) {
  constexpr int WPT = Geo<D>::WPT, CPT = Geo<D>::CPT, BACK = Geo<D>::BACK;
  int64_t T[WPT + 1];  // T[w + 1]: slices landing in word j0 + w, w = -1 .. WPT-1
#pragma unroll
  for (int w = 0; w <= WPT; w++) T[w] = 0;
#pragma unroll
  for (int i = 0; i < BACK + CPT; i++) {
    const int c = i - BACK;                            // column offset from kstart
    const int bit = D * c;                             // bit offset from word j0
    const int q = bit >= 0 ? bit / 32 : -((-bit + 31) / 32);  // floor(bit / 32)
    const int sh = bit - 32 * q;
    const __int128 v = (__int128)x[i] << sh;
    const int64_t sl0 = (int64_t)(uint32_t)v;
    const int64_t sl1 = (int64_t)(uint32_t)(v >> 32);
    const int64_t sl2 = (int64_t)(int32_t)(uint32_t)(v >> 64);
    if (q >= -1 && q <= WPT - 1) T[q + 1] += sl0;
    if (q + 1 >= -1 && q + 1 <= WPT - 1) T[q + 2] += sl1;
    if (q + 2 >= -1 && q + 2 <= WPT - 1) T[q + 3] += sl2;
  }
#pragma unroll
  for (int w = 0; w < WPT; w++) s[w] = (int64_t)(uint32_t)T[w + 1] + (T[w] >> 32);
}

// counter: tiles claimed so far in this launch (zero before the launch)
template <int D, class Src>
__global__ void __launch_bounds__(kThreads) norm_kernel(Src src, unsigned int *counter,
                                                        int *status) {
  constexpr int WPT = Geo<D>::WPT, CPT = Geo<D>::CPT, BACK = Geo<D>::BACK;
  constexpr int NX = BACK + CPT;
  constexpr int TW = kThreads * WPT;  // words per tile
  __shared__ int64_t s_c1[kStage];
  __shared__ int64_t s_c2[kStage];
  __shared__ uint32_t s_warp[kThreads / 32];
  __shared__ int s_cin[2];
  __shared__ unsigned int s_vid;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  if (tid == 0) s_vid = atomicAdd(counter, 1u);
  __syncthreads();
  int64_t bid;
  const NormArgs &a = src.locate((int64_t)s_vid, bid);
  const int64_t group = bid / a.ntiles;
  const int64_t tile = bid - group * a.ntiles;
  const int nsub = a.paired ? 2 : 1;
  const NormJob &J0 = a.job[nsub * group];
  const int64_t W0 = tile * TW;
  const bool two = J0.c2 != nullptr;

  // stage the tile's columns kt .. kt + 128 CPT + BACK - 1 (kt = first column
  // of thread 0 minus BACK), zero outside [0, n)
  const int64_t kt = tile * (int64_t)(kThreads * CPT) - BACK;
  constexpr int cnt = kThreads * CPT + BACK;
  for (int i = tid; i < cnt; i += kThreads) {
    const int64_t k = kt + i;
    s_c1[pad8(i)] = (k >= 0 && k < J0.n1) ? J0.c1[k] : 0;
    if (two) s_c2[pad8(i)] = (k >= 0 && k < J0.n2) ? J0.c2[k] : 0;
  }
  __syncthreads();

  // s_j of this thread's words, for each sub-job, and the thread's transfer
  // function (bits 0-5 sub-job 0, bits 8-13 sub-job 1), found by running the
  // three possible incoming carries through its words
  const int64_t j0 = W0 + (int64_t)tid * WPT;
  int64_t s[2][WPT];
  uint32_t agg = kIdentity | (kIdentity << 8);
  bool all_const = true;
#pragma unroll
  for (int u = 0; u < 2; u++) {
    if (u >= nsub) break;
    const int sigma = a.job[nsub * group + u].sigma;
    int64_t x[NX];
#pragma unroll
    for (int i = 0; i < NX; i++) {
      const int idx = pad8(tid * CPT + i);
      int64_t v = s_c1[idx];
      if (two) v += sigma > 0 ? s_c2[idx] : -s_c2[idx];
      x[i] = v;
    }
    thread_words<D>(x, s[u]);
    int64_t cm = -1, cz = 0, cp = 1;
#pragma unroll
    for (int w = 0; w < WPT; w++) {
      cm = (s[u][w] + cm) >> 32;
      cz = (s[u][w] + cz) >> 32;
      cp = (s[u][w] + cp) >> 32;
    }
    const uint32_t f = (uint32_t)(cm + 1) | ((uint32_t)(cz + 1) << 2) | ((uint32_t)(cp + 1) << 4);
    all_const = all_const && cm == cz && cz == cp;
    agg = u == 0 ? ((agg & ~63u) | f) : ((agg & 63u) | (f << 8));
  }
  // usual case: every thread's function is constant (some word of it absorbs
  // any incoming carry); then a thread's carry in is its predecessor's
  // constant carry out, and no composition is needed
  const bool fast = __syncthreads_and(all_const) != 0;

  uint32_t pre = kIdentity | (kIdentity << 8), total;
  if (fast) {
    if (lane == 31) s_warp[wid] = agg;
    __syncthreads();
    total = s_warp[kThreads / 32 - 1];  // thread 127's constant functions
  } else {
    // block-wide exclusive scan of the (paired) functions in thread order
    uint32_t incl = agg;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const uint32_t o = __shfl_up_sync(0xffffffffu, incl, off);
      if (lane >= off) incl = compose2(incl, o);
    }
    uint32_t excl = __shfl_up_sync(0xffffffffu, incl, 1);
    if (lane == 0) excl = kIdentity | (kIdentity << 8);
    if (lane == 31) s_warp[wid] = incl;
    __syncthreads();
    uint32_t wpre = kIdentity | (kIdentity << 8);
    total = kIdentity | (kIdentity << 8);
#pragma unroll
    for (int w = 0; w < kThreads / 32; w++) {
      if (w < wid) wpre = compose2(s_warp[w], wpre);
      total = compose2(s_warp[w], total);
    }
    pre = compose2(excl, wpre);
  }

  // warp u looks back for sub-job u
  if (wid < nsub) {
    const NormJob &J = a.job[nsub * group + wid];
    const int c = look_back(J.flags, tile, (total >> (8 * wid)) & 63u, lane, status);
    if (lane == 0) s_cin[wid] = c;
  }
  __syncthreads();

  // predecessor's functions (fast path): the previous lane, or the previous
  // warp's last lane; thread 0 takes the tile's carry in
  const uint32_t prev_lane = __shfl_up_sync(0xffffffffu, agg, 1);
  const uint32_t prev = lane > 0 ? prev_lane : (wid > 0 ? s_warp[wid - 1] : 0u);
#pragma unroll
  for (int u = 0; u < 2; u++) {
    if (u >= nsub) break;
    const NormJob &J = a.job[nsub * group + u];
    int c;
    if (fast)
      c = tid == 0 ? s_cin[u] : apply_fn((prev >> (8 * u)) & 63u, 0);
    else
      c = apply_fn((pre >> (8 * u)) & 63u, s_cin[u]);
    uint32_t o[WPT];
#pragma unroll
    for (int w = 0; w < WPT; w++) {
      const int64_t v = s[u][w] + c;
      o[w] = (uint32_t)v;
      c = (int)(v >> 32);
    }
    if (WPT == 4) {
      // nwords is a multiple of four: the four words are all inside or all outside
      if (j0 < a.nwords)
        *reinterpret_cast<uint4 *>(J.out + j0) = make_uint4(o[0], o[1], o[2], o[3 % WPT]);
    } else {
#pragma unroll
      for (int w = 0; w < WPT; w++)
        if (j0 + w < a.nwords) J.out[j0 + w] = o[w];
    }
  }
}

template <int D>
constexpr int tile_words() { return kThreads * Geo<D>::WPT; }

}  // namespace

int norm_tile_words(int d) { return d == 28 ? tile_words<28>() : tile_words<16>(); }

int64_t norm_tiles_for(int64_t nwords, int d) {
  const int tw = norm_tile_words(d);
  return (nwords + tw - 1) / tw;
}

int make_norm_args(const NormJob *jobs, int njobs, int d, int64_t nwords, int64_t ntiles,
                   NormArgs &a) {
  if (njobs < 1 || njobs > 4) return -1;
  if (d != 16 && d != 28) return -1;
  if (ntiles * norm_tile_words(d) < nwords || (nwords & 3) != 0) return -1;
  a = NormArgs{};
  for (int i = 0; i < njobs; i++) a.job[i] = jobs[i];
  a.njobs = njobs;
  a.d = d;
  a.nwords = nwords;
  a.ntiles = ntiles;
  // the +- pairs of Sec. 3.3 / 3.4 share their inputs
  bool paired = njobs % 2 == 0;
  for (int i = 0; paired && i < njobs; i += 2) {
    const NormJob &x = jobs[i], &y = jobs[i + 1];
    paired = x.c2 != nullptr && x.c1 == y.c1 && x.c2 == y.c2 && x.n1 == y.n1 && x.n2 == y.n2;
  }
  a.paired = paired ? 1 : 0;
  return 0;
}

int64_t norm_blocks(const NormArgs &a) {
  return (a.paired ? a.njobs / 2 : a.njobs) * a.ntiles;
}

cudaError_t launch_normalize(const NormJob *jobs, int njobs, int d, int64_t nwords,
                             int64_t ntiles, unsigned int *counter, int *status, cudaStream_t s) {
  NormArgs a;
  if (make_norm_args(jobs, njobs, d, nwords, ntiles, a) != 0) return cudaErrorInvalidValue;
  const unsigned grid = (unsigned)norm_blocks(a);
  if (d == 28)
    norm_kernel<28, One<NormArgs>><<<grid, kThreads, 0, s>>>(One<NormArgs>{a}, counter, status);
  else
    norm_kernel<16, One<NormArgs>><<<grid, kThreads, 0, s>>>(One<NormArgs>{a}, counter, status);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_normalize_batch(int d, const NormArgs *da, const int64_t *prefix, int n,
                                   int64_t blocks, unsigned int *counter, int *status,
                                   cudaStream_t s) {
  if (n == 0 || blocks == 0) return cudaSuccess;
  const Many<NormArgs> src{da, prefix, n};
  if (d == 28)
    norm_kernel<28, Many<NormArgs>><<<(unsigned)blocks, kThreads, 0, s>>>(src, counter, status);
  else
    norm_kernel<16, Many<NormArgs>><<<(unsigned)blocks, kThreads, 0, s>>>(src, counter, status);
  note_launches(1);
  return cudaGetLastError();
}

// flag words of a product: one counter word, one spare, one flag per tile per job
int64_t norm_flag_bytes(int njobs, int64_t ntiles) {
  return ((8 + 4 * (int64_t)njobs * ntiles) + 7) & ~(int64_t)7;
}

}  // namespace ks
