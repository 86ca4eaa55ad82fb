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
// Tiles.  Every CTA of norm_tiles takes one tile of words (one or both of a +- pair
// of combinations: same c1, c2, opposite sigma, so those columns are read
// once).  It stages the columns the tile needs in shared memory (one
// coalesced read of the column sums; a thread's words are exactly its
// columns' bit span, so all slicing offsets are compile-time constants of the
// digit width), forms s_j, and composes the tile's transfer function.  Usually
// every thread's function is constant (a word that absorbs any incoming
// carry), and then a thread's carry in is simply its predecessor's carry out.
//
// The carry into a tile comes from the tiles before it.  While the tiles of a
// launch fit in about one wave of CTAs, by a single-pass scan
// with look-back (the decoupled look-back of Merrill and Garland's single-pass
// prefix scan): the tile publishes its function in its flag word, then composes
// the predecessors' published functions, newest first, until the composition
// is constant or a predecessor has already published its carry out -- almost
// always after the previous tile alone, since its function is constant -- and
// publishes its own carry out.  Tiles are handed to CTAs by a counter in the
// order the CTAs start, so every predecessor a tile waits for is running or
// done; each wait is bounded (1 s, then status 1).  The flags and the counter
// must be clear before the launch (the product's first kernel clears them).
//
// Larger launches (tens of thousands of tiles, where those waits add up) take
// two: norm_tiles writes each tile's words with carry 0 and records its
// function, and norm_carry, one CTA per 256 tiles, composes the functions of
// the earlier tiles (walking back 256 at a time until the composition is
// constant, usually one step), scans its own 256, and adds each tile's carry
// in to its stored words -- an exact increment or decrement of the tile's
// value, which stops at the first word that absorbs it.
#include <atomic>

#include "ks_internal.cuh"
#include "ks_src.cuh"

namespace ks {

namespace {
constexpr int kThreads = 128;
constexpr int kCarryThreads = 256;  // tiles per CTA of norm_carry
// launches of at most this many tile CTAs (about one wave at 16 per SM) take
// the single pass; larger ones the tile pass and the carry pass, whose tiles
// never wait (with tens of thousands of tiles, the look-back costs more than
// the second launch)
constexpr int64_t kSinglePassCtas = 2048;
constexpr uint32_t kIdentity = 0u | (1u << 2) | (2u << 4);
// a tile's flag: its two functions (bits 0-5, 8-13), then whether they are
// the tile's own (kFlagAgg) or the constant carry out of it (kFlagPrefix)
constexpr uint32_t kFnMask = 63u | (63u << 8);
constexpr uint32_t kFlagAgg = 1u << 30, kFlagPrefix = 1u << 31;
constexpr uint64_t kFlagWaitNs = 1000000000ull;  // bound of a wait for a predecessor (1 s)

// Per digit width D: every thread takes WPT words = 32 WPT bits = CPT columns
// exactly (32 WPT = D CPT), so each column sits at a compile-time bit offset
// from the thread's first word; BACK earlier columns still reach its first
// word or the word before it (their slices span three words).
template <int D>
struct Geo;
// Two words per thread keep a thread's dependent chain short and give a
// product four times the CTAs of eight words per thread.
template <>
struct Geo<16> {
  static constexpr int WPT = 2, CPT = 4, BACK = 6;
};
template <>
struct Geo<32> {
  static constexpr int WPT = 2, CPT = 2, BACK = 3;  // column -3's top slice is word -1's
};
// staged columns of a tile: 128 CPT + BACK, one padding slot per 8 (banks)
constexpr int kStage = (kThreads * 4 + 8) + (kThreads * 4 + 8) / 8 + 8;
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
__device__ __forceinline__ bool is_const(uint32_t f) {  // monotone: f(-1) = f(1)
  return apply_fn(f, -1) == apply_fn(f, 1);
}
__device__ __forceinline__ uint32_t const_fn(int v) {
  const uint32_t e = (uint32_t)(v + 1);
  return e | (e << 2) | (e << 4);
}
// flags are read past the L1 (another CTA writes them) and written whole
__device__ __forceinline__ uint32_t flag_load(const uint32_t *p) { return __ldcv(p); }
__device__ __forceinline__ void flag_store(uint32_t *p, uint32_t v) { atomicExch(p, v); }
__device__ __forceinline__ uint64_t now_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// two functions side by side (bits 0-5 and 8-13), composed lane-wise
__device__ __forceinline__ uint32_t compose2(uint32_t g, uint32_t f) {
  return compose(g & 63u, f & 63u) | (compose((g >> 8) & 63u, (f >> 8) & 63u) << 8);
}

// s_j of a thread's WPT words from its BACK + CPT staged columns (x[i] is
// column kstart - BACK + i); every offset and shift is a compile-time constant.
//
// J's shift pattern (one bit at pstart + i pstride, i < pcount: the K U(Y) of
// signed coefficients) is added to T before the fold, so that its carries
// travel with the others.
template <int D>
__device__ __forceinline__ void thread_words(const int64_t (&x)[Geo<D>::BACK + Geo<D>::CPT],
                                             int64_t (&s)[Geo<D>::WPT], const NormJob &J,
                                             int64_t j0) {
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
  if (J.pcount > 0) {
    // pattern bits in words j0 - 1 .. j0 + WPT - 1, bits [b0, b1)
    const int64_t b0 = 32 * (j0 - 1), b1 = 32 * (j0 + WPT);
    int64_t i = b0 > J.pstart ? (b0 - J.pstart + J.pstride - 1) / J.pstride : 0;
    for (; i < J.pcount; i++) {
      const int64_t rel = J.pstart + i * J.pstride - b0;
      if (rel >= b1 - b0) break;
      const int w = (int)(rel >> 5);
      const int64_t bit = (int64_t)1 << (rel & 31);
#pragma unroll
      for (int q = 0; q <= WPT; q++)
        if (q == w) T[q] += bit;
    }
  }
#pragma unroll
  for (int w = 0; w < WPT; w++) s[w] = (int64_t)(uint32_t)T[w + 1] + (T[w] >> 32);
}

template <int D, bool kSingle, class Src>
__global__ void __launch_bounds__(kThreads) norm_tiles(Src src) {
  pdl_enter();
  constexpr int WPT = Geo<D>::WPT, CPT = Geo<D>::CPT, BACK = Geo<D>::BACK;
  constexpr int NX = BACK + CPT;
  constexpr int TW = kThreads * WPT;  // words per tile
  __shared__ int64_t s_c1[kStage];
  __shared__ int64_t s_c2[kStage];
  __shared__ uint32_t s_warp[kThreads / 32];
  __shared__ uint32_t s_idx;
  __shared__ int s_cin[2];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  int64_t bid;
  const NormArgs &a = src.locate(blockIdx.x, bid);
  // single pass: tiles go to CTAs in the order the CTAs start (a counter
  // after the flags), so every tile's predecessors have started before it
  // looks back at them
  if (kSingle) {
    if (tid == 0) s_idx = atomicAdd(a.job[0].flags + (int64_t)a.njobs * a.ntiles, 1u);
    __syncthreads();
  }
  const int64_t idx = kSingle ? (int64_t)s_idx : bid;
  const int64_t group = idx / a.ntiles;
  const int64_t tile = idx - group * a.ntiles;
  const int nsub = a.paired ? 2 : 1;
  const NormJob &J0 = a.job[nsub * group];
  const int64_t W0 = tile * TW;
  const bool two = J0.c2 != nullptr;

  // stage the tile's columns kt .. kt + 128 CPT + BACK - 1 (kt = first column
  // of thread 0 minus BACK), zero outside [0, n)
  const int64_t kt = tile * (int64_t)(kThreads * CPT) - BACK;
  constexpr int cnt = kThreads * CPT + BACK;
  constexpr int kIt = (cnt + kThreads - 1) / kThreads;
  {
    // all of a thread's loads first (read-only path), then the stores
    int64_t r1[kIt], r2[kIt];
#pragma unroll
    for (int it = 0; it < kIt; it++) {
      const int i = tid + it * kThreads;
      const int64_t k = kt + i;
      r1[it] = (i < cnt && k >= 0 && k < J0.n1) ? __ldg(J0.c1 + k) : 0;
      r2[it] = (two && i < cnt && k >= 0 && k < J0.n2) ? __ldg(J0.c2 + k) : 0;
    }
#pragma unroll
    for (int it = 0; it < kIt; it++) {
      const int i = tid + it * kThreads;
      if (i < cnt) {
        s_c1[pad8(i)] = r1[it];
        s_c2[pad8(i)] = r2[it];
      }
    }
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
    thread_words<D>(x, s[u], a.job[nsub * group + u], j0);
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

  // the carry into the tile: publish the tile's functions, then compose the
  // predecessors' back to the first one that is constant or already holds its
  // carry out (usually the previous tile alone), and publish that carry out
  if (!kSingle) {
    // two passes: the tile's functions for norm_carry, and carry 0 here
    if (tid == 0) {
      for (int u = 0; u < nsub; u++) a.job[nsub * group + u].flags[tile] = (total >> (8 * u)) & 63u;
      s_cin[0] = 0;
      s_cin[1] = 0;
    }
  } else if (tid == 0) {
    uint32_t *fl = a.job[nsub * group].flags;
    const uint32_t used = nsub == 2 ? kFnMask : 63u;
    flag_store(fl + tile, (total & used) | kFlagAgg);
    uint32_t acc = kIdentity | (kIdentity << 8);
    bool ok = true;
    for (int64_t j = tile - 1; j >= 0; j--) {
      uint32_t v = flag_load(fl + j);
      if ((v & (kFlagAgg | kFlagPrefix)) == 0) {
        const uint64_t t0 = now_ns();
        while (((v = flag_load(fl + j)) & (kFlagAgg | kFlagPrefix)) == 0)
          if (now_ns() - t0 > kFlagWaitNs) {
            ok = false;
            break;
          }
        if (!ok) break;
      }
      acc = compose2(acc, (v & used) | (~used & (kIdentity | (kIdentity << 8))));
      if ((v & kFlagPrefix) || (is_const(acc & 63u) && (nsub == 1 || is_const((acc >> 8) & 63u))))
        break;
    }
    if (!ok && a.status != nullptr) atomicCAS(a.status, 0, 1);
    const int c0 = apply_fn(acc & 63u, 0), c1 = apply_fn((acc >> 8) & 63u, 0);
    const int o0 = apply_fn(total & 63u, c0), o1 = apply_fn((total >> 8) & 63u, c1);
    flag_store(fl + tile, ((const_fn(o0) | (const_fn(o1) << 8)) & used) | kFlagPrefix);
    s_cin[0] = c0;
    s_cin[1] = c1;
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
    const int cin = s_cin[u];
    int c;
    if (fast)
      c = tid == 0 ? cin : apply_fn((prev >> (8 * u)) & 63u, 0);
    else
      c = apply_fn((pre >> (8 * u)) & 63u, cin);
    uint32_t o[WPT];
#pragma unroll
    for (int w = 0; w < WPT; w++) {
      const int64_t v = s[u][w] + c;
      o[w] = (uint32_t)v;
      c = (int)(v >> 32);
    }
    if (WPT == 2) {
      // nwords is a multiple of four: the two words are both inside or both outside
      if (j0 < a.nwords) *reinterpret_cast<uint2 *>(J.out + j0) = make_uint2(o[0], o[1 % WPT]);
    } else {
#pragma unroll
      for (int w = 0; w < WPT; w++)
        if (j0 + w < a.nwords) J.out[j0 + w] = o[w];
    }
  }
}

// Ordered block-wide composition: returns, in every thread, the composition
// of the threads' functions in thread order (thread 0 innermost), and in
// `excl` this thread's exclusive prefix.
__device__ __forceinline__ uint32_t block_compose(uint32_t f, uint32_t &excl, uint32_t *s_warp) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  uint32_t incl = f;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const uint32_t o = __shfl_up_sync(0xffffffffu, incl, off);
    if (lane >= off) incl = compose(incl, o);
  }
  uint32_t e = __shfl_up_sync(0xffffffffu, incl, 1);
  if (lane == 0) e = kIdentity;
  __syncthreads();
  if (lane == 31) s_warp[wid] = incl;
  __syncthreads();
  uint32_t wpre = kIdentity, total = kIdentity;
  for (int w = 0; w < kCarryThreads / 32; w++) {
    if (w < wid) wpre = compose(s_warp[w], wpre);
    total = compose(s_warp[w], total);
  }
  excl = compose(e, wpre);
  return total;
}

// One CTA per 256 tiles of one group: carries into the tiles, added to the
// stored words (tile t's words were written as if its carry in were 0).
template <int D, class Src>
__global__ void __launch_bounds__(kCarryThreads) norm_carry(Src src) {
  pdl_enter();
  constexpr int TW = kThreads * Geo<D>::WPT;
  __shared__ uint32_t s_warp[kCarryThreads / 32];
  int64_t bid;
  const NormArgs &a = src.locate(blockIdx.x, bid);
  const int64_t per = (a.ntiles + kCarryThreads - 1) / kCarryThreads;  // CTAs per group
  const int64_t group = bid / per;
  const int64_t t0 = (bid - group * per) * kCarryThreads;  // first tile of this CTA
  const int nsub = a.paired ? 2 : 1;
  const int tid = threadIdx.x;
  for (int u = 0; u < nsub; u++) {
    const NormJob &J = a.job[nsub * group + u];
    // the composition of the functions of tiles 0 .. t0 - 1, walked back from
    // t0 in windows of 256 (one flag per thread, composed in order); it stops
    // at the first window after which the composition is constant (usually the
    // first: some tile absorbs any incoming carry), or at tile 0
    uint32_t before = kIdentity, excl;
    for (int64_t w1 = t0; w1 > 0; w1 -= kCarryThreads) {
      const int64_t w0 = w1 - kCarryThreads;
      const int64_t i = w0 + tid;
      const uint32_t f = i >= 0 ? (J.flags[i] & 63u) : kIdentity;
      before = compose(before, block_compose(f, excl, s_warp));
      if (apply_fn(before, -1) == apply_fn(before, 1)) break;  // constant (monotone)
    }
    const int c0 = apply_fn(before, 0);
    // this CTA's tiles: exclusive prefix of their functions
    const int64_t t = t0 + tid;
    const uint32_t ft = t < a.ntiles ? (J.flags[t] & 63u) : kIdentity;
    block_compose(ft, excl, s_warp);
    int c = apply_fn(excl, c0);
    if (t < a.ntiles && c != 0) {
      const int64_t w0 = t * TW;
      int64_t w1 = w0 + TW;
      if (w1 > a.nwords) w1 = a.nwords;
      for (int64_t j = w0; j < w1 && c != 0; j++) {
        const int64_t v = (int64_t)J.out[j] + c;
        J.out[j] = (uint32_t)v;
        c = (int)(v >> 32);
      }
    }
  }
}

template <int D>
constexpr int tile_words() { return kThreads * Geo<D>::WPT; }

}  // namespace

int norm_tile_words(int d) { return d == 32 ? tile_words<32>() : tile_words<16>(); }

int64_t norm_tiles_for(int64_t nwords, int d) {
  const int tw = norm_tile_words(d);
  return (nwords + tw - 1) / tw;
}

int make_norm_args(const NormJob *jobs, int njobs, int d, int64_t nwords, int64_t ntiles,
                   int *status, NormArgs &a) {
  if (njobs < 1 || njobs > 4) return -1;
  if (d != 16 && d != 32) return -1;
  if (ntiles * norm_tile_words(d) < nwords || (nwords & 3) != 0) return -1;
  if (ntiles * 2 > 0x7fffffffLL) return -1;  // the tile counter is 32 bits
  a = NormArgs{};
  for (int i = 0; i < njobs; i++) a.job[i] = jobs[i];
  a.njobs = njobs;
  a.d = d;
  a.nwords = nwords;
  a.ntiles = ntiles;
  a.status = status;
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

int64_t norm_carry_blocks(const NormArgs &a) {
  return (a.paired ? a.njobs / 2 : a.njobs) * ((a.ntiles + kCarryThreads - 1) / kCarryThreads);
}

// test hook: 0 by size, 1 always the single pass, 2 always the two passes
static std::atomic<int> g_norm_form{0};

bool norm_single_pass(int64_t tile_blocks) {
  const int f = g_norm_form.load(std::memory_order_relaxed);
  return f == 1 || (f == 0 && tile_blocks <= kSinglePassCtas);
}

cudaError_t launch_normalize(const NormJob *jobs, int njobs, int d, int64_t nwords,
                             int64_t ntiles, int *status, cudaStream_t s) {
  NormArgs a;
  if (make_norm_args(jobs, njobs, d, nwords, ntiles, status, a) != 0)
    return cudaErrorInvalidValue;
  const One<NormArgs> one{a};
  const unsigned g1 = (unsigned)norm_blocks(a), g2 = (unsigned)norm_carry_blocks(a);
  if (norm_single_pass(g1)) {
    if (d == 32)
      (void)launch_k(norm_tiles<32, true, One<NormArgs>>, dim3(g1), dim3(kThreads), 0, s, one);
    else
      (void)launch_k(norm_tiles<16, true, One<NormArgs>>, dim3(g1), dim3(kThreads), 0, s, one);
    note_launches(1);
  } else {
    if (d == 32) {
      (void)launch_k(norm_tiles<32, false, One<NormArgs>>, dim3(g1), dim3(kThreads), 0, s, one);
      (void)launch_k(norm_carry<32, One<NormArgs>>, dim3(g2), dim3(kCarryThreads), 0, s, one);
    } else {
      (void)launch_k(norm_tiles<16, false, One<NormArgs>>, dim3(g1), dim3(kThreads), 0, s, one);
      (void)launch_k(norm_carry<16, One<NormArgs>>, dim3(g2), dim3(kCarryThreads), 0, s, one);
    }
    note_launches(2);
  }
  return cudaGetLastError();
}

cudaError_t launch_normalize_batch(int d, const NormArgs *da, const int64_t *prefix_tiles,
                                   const int64_t *prefix_carry, int n, int64_t tile_blocks,
                                   int64_t carry_blocks, cudaStream_t s) {
  if (n == 0 || tile_blocks == 0) return cudaSuccess;
  const Many<NormArgs> t{da, prefix_tiles, n}, c{da, prefix_carry, n};
  const dim3 g1((unsigned)tile_blocks), g2((unsigned)carry_blocks);
  if (norm_single_pass(tile_blocks)) {
    if (d == 32)
      (void)launch_k(norm_tiles<32, true, Many<NormArgs>>, g1, dim3(kThreads), 0, s, t);
    else
      (void)launch_k(norm_tiles<16, true, Many<NormArgs>>, g1, dim3(kThreads), 0, s, t);
    note_launches(1);
  } else {
    if (d == 32) {
      (void)launch_k(norm_tiles<32, false, Many<NormArgs>>, g1, dim3(kThreads), 0, s, t);
      (void)launch_k(norm_carry<32, Many<NormArgs>>, g2, dim3(kCarryThreads), 0, s, c);
    } else {
      (void)launch_k(norm_tiles<16, false, Many<NormArgs>>, g1, dim3(kThreads), 0, s, t);
      (void)launch_k(norm_carry<16, Many<NormArgs>>, g2, dim3(kCarryThreads), 0, s, c);
    }
    note_launches(2);
  }
  return cudaGetLastError();
}

// flag words of a product: one per tile per job, then the tile counter
int64_t norm_flag_bytes(int njobs, int64_t ntiles) {
  return ((4 * (int64_t)njobs * ntiles + 4) + 7) & ~(int64_t)7;
}

}  // namespace ks

extern "C" void ks_debug_norm_form(int form) {
  ks::g_norm_form.store(form == 1 || form == 2 ? form : 0);
  ks::bump_epoch();  // host-call graphs captured the other form
}
