// Exact seeds of the reconstruction chains (Sec. 3.2): the values
//
//   h'_k = sum_t f_t g_(k-t)   (+ K = 2^kb for signed inputs)
//
// for clusters of C consecutive k (the pair c_(s-1), c_s of one run, or of
// both runs of Sec. 3.4 at once).  A chain started from such a pair needs no
// predecessor, so the recurrence runs in parallel chains.
//
// Narrow operands (both at most 64 bits, one limb) ride the tensor cores.
// Every coefficient is written as P balanced 8-bit digits, x = sum_p d_p 256^p
// with d_p in [-128, 128] (P = ceil(b / 8) for signed inputs, ceil((b + 1) / 8)
// unsigned, rounded up to 2, 4, 6, 8 or 9), into digit planes (fp16 holds the
// digits exactly).  With r = r' + r'' (r' in {0, 1}, r'' in {0, 2}) and t = t' + r'':
//   h'_(k0+r) = sum_(p,q) 256^(p+q) Z[q r'][p r''],
//   Z[q r'][p r''] = sum_t' G_q[k0 + r' - t'] F_p[t' + r''],
// a matrix product over K = t': rows (q, r') of A hold g digits, columns
// (p, r'') of B f digits.  The planes hold two copies of each operand, shifted
// so that every fragment a lane reads is one aligned 16-byte load: the f copies
// by r'', the g copies reversed and shifted by r' from an origin Z = k00
// (mod 8) (every cluster start k0 is k00 mod 8).  Inside a block of 64
// indices t' a lane's eight 32-bit fragment words are 16 consecutive indices;
// the same permutation of t' on both sides leaves the sum unchanged.
// A CTA takes a group of consecutive clusters over one window of 1024
// indices t', staged in shared memory; its warps run mma.sync m16n8k16 (fp16
// in, fp32 accumulate) over at most 512 indices t' each: every partial sum is
// an integer of magnitude at most 512 * 128^2 = 2^23, which fp32 holds
// exactly.  The entries are added along the digit diagonals p + q, carried
// into a 192-bit two's complement partial per value and window, and its six
// 32-bit words are added to the value's six 64-bit column sums (window 0
// adds K); the reconstruction carries them into the value mod 2^192 (exact:
// the values are non-negative and below 2^192).
//
// Wide operands: one CTA per value; a thread multiplies the magnitudes of its
// terms word by word (NW 32-bit words, a compile-time size) and keeps signed
// 64-bit column sums; the CTA adds them and one thread carries them (and K)
// into the value's words.
#include "ks_internal.cuh"
#include "ks_src.cuh"

namespace ks {

namespace {
constexpr int kWT = 128;            // threads of a wide seed CTA

// a one-limb coefficient of b = 64 - sh bits as a 64-bit value: sign-extended
// from bit b - 1 (signed) or its low b bits (unsigned)
__device__ __forceinline__ uint64_t extend64(uint64_t raw, int sh, int sgn) {
  const uint64_t up = raw << sh;
  return sgn ? (uint64_t)((int64_t)up >> sh) : up >> sh;
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


// ---- digit planes
constexpr int kPad = 16;   // zero columns before every plane (indices t' >= -8)
constexpr int kTail = 88;  // and after it (a warp's last 64-index block overshoots)
__host__ __device__ __forceinline__ int64_t plane_stride(int64_t len) {
  return (len + kPad + kTail + 7) & ~(int64_t)7;  // every plane starts 16-byte aligned
}
// halves of the digit planes: two copies of P planes of each operand
__host__ __device__ __forceinline__ int64_t planes_halves(int64_t lf, int64_t lg, int P) {
  return 2 * (int64_t)P * (plane_stride(lf) + plane_stride(lg));
}

// The P balanced 8-bit digits of a coefficient of b = 64 - sh bits (two's
// complement if sgn), written at out[p stride]: bytes balanced upward with a
// carry, the top digit takes the rest of the value.
__device__ __forceinline__ void write_digits8(uint64_t raw, int sh, int sgn, int P, __half *out,
                                              int64_t stride) {
  const uint64_t x = extend64(raw, sh, sgn);
  int32_t c = 0;
#pragma unroll
  for (int p = 0; p < 9; p++) {
    if (p >= P) break;
    int32_t d;
    if (p < P - 1) {
      const int32_t t = (int32_t)((x >> (8 * p)) & 255u) + c;
      c = t >= 128 ? 1 : 0;
      d = t - 256 * c;
    } else {
      const int top = 8 * p;
      int32_t rest;
      if (top >= 64)
        rest = sgn ? (int32_t)((int64_t)x >> 63) : 0;
      else
        rest = sgn ? (int32_t)((int64_t)x >> top) : (int32_t)(x >> top);
      d = rest + c;
    }
    out[p * stride] = __int2half_rn(d);
  }
}
__device__ __forceinline__ void write_zeros(int P, __half *out, int64_t stride) {
  for (int p = 0; p < P; p++) out[p * stride] = __int2half_rn(0);
}

// Digit planes, a thread per column (and the zeroing of the seed values'
// column sums, which the seed kernel then accumulates):
//   f copy c (c = 0, 1), plane p at planes + (c P + p) fs: column x holds
//     digit p of f_(x - kPad + 2c);
//   g copy c, plane q at planes + 2 P fs + (c P + q) gs: column y holds digit q
//     of g_(Z + c - (y - kPad));
// zero outside the polynomials.  One launch covers a batch (any P).
template <class Src>
__global__ void __launch_bounds__(256) seed_planes(Src src) {
  pdl_enter();
  int64_t local;
  const SeedArgs &a = src.locate(blockIdx.x, local);
  const int P = a.P;
  const int64_t fs = plane_stride(a.lf), gs = plane_stride(a.lg);
  const int64_t i = local * 256 + threadIdx.x;
  if (i < a.ncl * a.C * 6) a.acc[i] = 0ull;
  if (i < fs) {
    for (int c = 0; c < 2; c++) {
      const int64_t t = i - kPad + 2 * c;
      __half *out = a.planes + (int64_t)c * P * fs + i;
      if (t >= 0 && t < a.lf)
        write_digits8(__ldg(a.f + t), 64 - a.bf, a.sgn, P, out, fs);
      else
        write_zeros(P, out, fs);
    }
  } else if (i < fs + gs) {
    const int64_t y = i - fs;
    for (int c = 0; c < 2; c++) {
      const int64_t jg = a.Z + c - (y - kPad);
      __half *out = a.planes + 2 * (int64_t)P * fs + (int64_t)c * P * gs + y;
      if (jg >= 0 && jg < a.lg)
        write_digits8(__ldg(a.g + jg), 64 - a.bg, a.sgn, P, out, gs);
      else
        write_zeros(P, out, gs);
    }
  }
}

__device__ __forceinline__ void mma16816(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2,
                                         uint32_t a3, uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, "
      "{%8, %9}, {%0, %1, %2, %3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}
__device__ __forceinline__ uint32_t word(const uint4 &v, int i) {
  return i == 0 ? v.x : i == 1 ? v.y : i == 2 ? v.z : v.w;
}

// v << sh as 192 bits (v signed, 0 <= sh < 192)
__device__ __forceinline__ void shl192(int64_t v, int sh, uint64_t &w0, uint64_t &w1,
                                       uint64_t &w2) {
  const uint64_t ext = (uint64_t)(v >> 63);
  uint64_t x0 = (uint64_t)v, x1 = ext, x2 = ext;
  if (sh >= 128) {
    x2 = x0;
    x1 = 0;
    x0 = 0;
    sh -= 128;
  } else if (sh >= 64) {
    x2 = x1;
    x1 = x0;
    x0 = 0;
    sh -= 64;
  }
  if (sh) {
    x2 = (x2 << sh) | (x1 >> (64 - sh));
    x1 = (x1 << sh) | (x0 >> (64 - sh));
    x0 <<= sh;
  }
  w0 = x0;
  w1 = x1;
  w2 = x2;
}

constexpr int kSeedWarps = 8;
constexpr int kWin = 1024;    // indices t' per window (a CTA's share of the contraction)
constexpr int kRowPad = 32;   // staged rows are 32 halves (mod 64) apart: conflict-free reads
constexpr int kSeedSmemMax = 96 * 1024;  // staged bytes per CTA (at least two CTAs per SM)

// staged bytes of a CTA: two copies of the A rows (P x (kWin + kstep (G - 1))
// each) and NB copies of the B rows (P x kWin each), laid out as in
// seed_mma_body
__host__ __device__ __forceinline__ int64_t seed_smem(int P, int C, int G, int64_t kstep) {
  const int64_t lys = kWin + kstep * (G - 1) + kRowPad;
  const int64_t ca = P * lys + (P % 2 == 0 ? kRowPad : 0);
  const int64_t cb = P * (int64_t)(kWin + kRowPad) + (P % 2 == 0 ? kRowPad : 0);
  return 2 * (2 * ca + (C / 2) * cb);
}

// the operand fragments of one block of 64 indices t'
template <int MT, int NT>
struct Frag {
  uint4 a[MT][2][2], b[NT][2];
};
template <int MT, int NT>
__device__ __forceinline__ void load_frag(Frag<MT, NT> &fr, const uint4 *const (&pa)[MT][2],
                                          const uint4 *const (&pb)[NT], int ib, bool in) {
  const uint4 z4 = make_uint4(0u, 0u, 0u, 0u);
  const int o = 8 * ib;  // 16-byte words per block: 64 halves
#pragma unroll
  for (int mt = 0; mt < MT; mt++)
#pragma unroll
    for (int h = 0; h < 2; h++)
#pragma unroll
      for (int h2 = 0; h2 < 2; h2++)
        fr.a[mt][h][h2] = (in && pa[mt][h]) ? pa[mt][h][o + 4 * h2] : z4;
#pragma unroll
  for (int nt = 0; nt < NT; nt++)
#pragma unroll
    for (int h2 = 0; h2 < 2; h2++) fr.b[nt][h2] = (in && pb[nt]) ? pb[nt][o + 4 * h2] : z4;
}
// k-step st of a block: fragment words 2 (st & 1) (indices 2 tig, 2 tig + 1 of
// the step) and 2 (st & 1) + 1 (2 tig + 8, 2 tig + 9) of half st >> 1; the
// steps go to NA independent accumulator sets (short dependency chains)
template <int NA, int MT, int NT>
__device__ __forceinline__ void mma_frag(float (&acc)[NA][MT][NT][4], const Frag<MT, NT> &fr) {
#pragma unroll
  for (int st = 0; st < 4; st++) {
    const int h2 = st >> 1, w0 = 2 * (st & 1);
#pragma unroll
    for (int mt = 0; mt < MT; mt++)
#pragma unroll
      for (int nt = 0; nt < NT; nt++)
        mma16816(acc[st % NA][mt][nt], word(fr.a[mt][0][h2], w0), word(fr.a[mt][1][h2], w0),
                 word(fr.a[mt][0][h2], w0 + 1), word(fr.a[mt][1][h2], w0 + 1),
                 word(fr.b[nt][h2], w0), word(fr.b[nt][h2], w0 + 1));
  }
}

// the t' range [tlo, thi] of cluster j (tlo aligned down to 8; the extra
// indices read zero padding)
__device__ __forceinline__ void cluster_range(const SeedArgs &a, int64_t j, int64_t &k0,
                                              int64_t &tlo, int64_t &thi) {
  k0 = a.k00 + a.kstep * j;
  tlo = k0 - (a.lg - 1);
  if (tlo < -2) tlo = -2;
  tlo &= ~(int64_t)7;
  thi = k0 + 1;
  if (thi > a.lf - 1) thi = a.lf - 1;
}

// One CTA: the G clusters j0 .. j0 + G - 1 of a group over window w, the
// indices t' in [T, T + kWin), T = -8 + w kWin.  The window's f digits and the
// g digits every cluster of the group reads there (cluster j's g columns are
// those of the group's last cluster shifted by kstep (jlast - j)) are staged
// in shared memory; 8 / G warps per cluster split the window.  A thread adds
// its entries Z[q r'][p r''] along the digit diagonals s = p + q (one sum
// per diagonal it holds) into the CTA's diagonal sums (32-bit); one thread per
// value then carries sum_s D_s 256^s into 192 bits.  Every (value, window)
// slot of the group is written, zero where the window misses the cluster's
// range; window 0 adds K.
template <int P, int C>
__device__ __forceinline__ void seed_mma_body(const SeedArgs &a, int64_t local, __half *sm) {
  constexpr int NB = C / 2;              // f copies in use: shifts r'' = 0 (and 2)
  constexpr int MT = (2 * P + 15) / 16;  // m16 tiles: A rows m = 2 q + r'
  constexpr int NT = (NB * P + 7) / 8;   // n8 tiles: B columns n = NB p + c
  constexpr int NA = MT * NT <= 2 ? 2 : 1;  // accumulator sets
  constexpr int ND = 2 * P - 1;          // digit diagonals s = p + q
  __shared__ int dsum[4][C][ND];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int grp = lane >> 2, tig = lane & 3;
  const int G = a.G;
  const int64_t gi = (int)local / (int)a.slices, w = local - gi * a.slices;
  const int64_t j0 = gi * G;
  const int gact = (int)(a.ncl - j0 < G ? a.ncl - j0 : G);
  const int64_t T = -8 + w * kWin;
  // is the window inside some cluster's range?  (tlo and thi grow with j)
  int64_t k0l, tlo0, thi0, tlol, thil;
  cluster_range(a, j0, k0l, tlo0, thi0);
  cluster_range(a, j0 + gact - 1, k0l, tlol, thil);
  const bool any = tlo0 <= T + kWin - 1 && thil >= T && tlo0 <= thil;
  const int wpc = kSeedWarps / G;  // warps per cluster
  if (!any) {  // block-uniform: nothing to add but K (window 0)
    if (w == 0 && a.kb >= 0 && tid < gact * C)
      atomicAdd(&a.acc[(j0 * C + tid) * 6 + (a.kb >> 5)], 1ull << (a.kb & 31));
    return;
  }
  for (int i = tid; i < 4 * C * ND; i += kSeedWarps * 32) (&dsum[0][0][0])[i] = 0;
  // staging: A rows (c, q) at sm + c ca + q lys, column i <-> g plane column
  // ybase + i; B rows (c, p) at smB + c cb + p bs, column i <-> f plane
  // column kPad + T + i.  One thread copies the part of every row inside its
  // plane with a bulk copy (all boundaries are multiples of 8 halves: 16-byte
  // aligned); the rest of a row (past a plane's ends) is zero-filled.
  // Row strides are 64 bytes (mod 128) and a copy starts 64 bytes (mod 128)
  // after the same row of the other copy: the eight lanes of a 16-byte read
  // phase (rows (0, k), (1, k)) fall in opposite halves of the banks.
  const int fs = (int)plane_stride(a.lf), gs = (int)plane_stride(a.lg);
  const int ly = kWin + (int)a.kstep * (gact - 1), lys = ly + kRowPad;
  constexpr int bs = kWin + kRowPad;
  const int ca = P * lys + (P % 2 == 0 ? kRowPad : 0);
  constexpr int cb = P * bs + (P % 2 == 0 ? kRowPad : 0);
  const int64_t ybase = kPad + a.Z - k0l + T;  // k0l: the group's last cluster start
  __half *smB = sm + 2 * ca;
  {
    __shared__ __align__(8) uint64_t sbar;
    // the in-plane columns [ya, yb) of the A rows, [xa, xb) of the B rows
    const int64_t ya = ybase < 0 ? 0 : ybase, yb = ybase + ly < gs ? ybase + ly : gs;
    const int64_t xs = kPad + T, xa = xs < 0 ? 0 : xs, xb = xs + kWin < fs ? xs + kWin : fs;
    const int na = yb > ya ? (int)(yb - ya) : 0, nbx = xb > xa ? (int)(xb - xa) : 0;
    const __half *fpl = a.planes, *gpl = a.planes + 2 * (int64_t)P * fs;
    if (tid == 0) {
      stage_init(&sbar);
      stage_expect(&sbar, (uint32_t)(2 * (2 * P * na + NB * P * nbx)));
      if (na > 0)
        for (int row = 0; row < 2 * P; row++)
          stage_copy(sm + (row / P) * ca + (row % P) * lys + (ya - ybase),
                     gpl + (int64_t)row * gs + ya, 2u * na, &sbar);
      if (nbx > 0)
        for (int row = 0; row < NB * P; row++)
          stage_copy(smB + (row / P) * cb + (row % P) * bs + (xa - xs),
                     fpl + (int64_t)row * fs + xa, 2u * nbx, &sbar);
    }
    // zeros where a row reaches past its plane (block-uniform conditions)
    const uint4 z4 = make_uint4(0u, 0u, 0u, 0u);
    if (na < ly) {
      const int lo = (int)(ya - ybase), hi = lo + na;  // in-plane columns of a row
      for (int i = tid; i < 2 * P * (ly / 8); i += kSeedWarps * 32) {
        const int row = i / (ly / 8), col = 8 * (i - row * (ly / 8));
        if (col < lo || col >= hi)
          *reinterpret_cast<uint4 *>(sm + (row / P) * ca + (row % P) * lys + col) = z4;
      }
    }
    if (nbx < kWin) {
      const int lo = (int)(xa - xs), hi = lo + nbx;
      for (int i = tid; i < NB * P * (kWin / 8); i += kSeedWarps * 32) {
        const int row = i / (kWin / 8), col = 8 * (i - row * (kWin / 8));
        if (col < lo || col >= hi)
          *reinterpret_cast<uint4 *>(smB + (row / P) * cb + (row % P) * bs + col) = z4;
      }
    }
    __syncthreads();  // the barrier's initialization, the zeros
    if (!__syncthreads_and(stage_wait(&sbar))) {
      if (tid == 0) atomicCAS(a.status, 0, 1);
      stage_wait(&sbar);  // once more (bounded) for the copies in flight before leaving
      return;
    }
  }
  const int ci = warp / wpc, part_i = warp - ci * wpc;
  if (ci < gact) {
    int64_t k0, tlo, thi;
    cluster_range(a, j0 + ci, k0, tlo, thi);
    const int sw = kWin / wpc;       // the warp's indices: [T + part_i sw, + sw)
    const int64_t s0 = T + (int64_t)part_i * sw;
    // blocks of 64 that meet [tlo, thi]
    int64_t b0 = tlo > s0 ? (tlo - s0) / 64 : 0;
    int64_t b1 = thi - s0 < sw ? (thi - s0) / 64 : sw / 64 - 1;
    if (thi < s0) b1 = -1;
    if (b0 <= b1) {
      // lane (grp, tig) reads indices t' = block + 32 h2 + 8 tig + [0, 8) as
      // one 16-byte word per operand row or column and half h2 of the block
      const int rp = grp & 1;  // r' of every A row of this lane
      const int ua = (int)a.kstep * (gact - 1 - ci) + (int)(s0 - T) + 64 * (int)b0 + 8 * tig;
      const int ub = (int)(s0 - T) + 64 * (int)b0 + 8 * tig;
      const uint4 *pa[MT][2];
#pragma unroll
      for (int mt = 0; mt < MT; mt++)
#pragma unroll
        for (int h = 0; h < 2; h++) {
          const int q = (16 * mt + grp + 8 * h) >> 1;
          pa[mt][h] = q < P ? reinterpret_cast<const uint4 *>(sm + rp * ca + q * lys + ua) : nullptr;
        }
      const uint4 *pb[NT];
#pragma unroll
      for (int nt = 0; nt < NT; nt++) {
        const int n = 8 * nt + grp;
        const int p = NB == 2 ? n >> 1 : n, c = NB == 2 ? (n & 1) : 0;
        pb[nt] = p < P ? reinterpret_cast<const uint4 *>(smB + c * cb + p * bs + ub) : nullptr;
      }
      float acc[NA][MT][NT][4];
#pragma unroll
      for (int k = 0; k < NA; k++)
#pragma unroll
        for (int mt = 0; mt < MT; mt++)
#pragma unroll
          for (int nt = 0; nt < NT; nt++)
#pragma unroll
            for (int e = 0; e < 4; e++) acc[k][mt][nt][e] = 0.f;
      const int nblk = (int)(b1 - b0 + 1);
      // two register stages: the next block's reads are in flight during a block's MMAs
      Frag<MT, NT> f0, f1;
      load_frag(f0, pa, pb, 0, true);
      for (int ib = 0; ib < nblk; ib += 2) {
        load_frag(f1, pa, pb, ib + 1, ib + 1 < nblk);
        mma_frag(acc, f0);
        load_frag(f0, pa, pb, ib + 2, ib + 2 < nblk);
        if (ib + 1 < nblk) mma_frag(acc, f1);
      }
      // entry (row m, column n) of tile (mt, nt): d0/d1 row grp, d2/d3 row
      // grp + 8, columns 2 tig and 2 tig + 1; q = m >> 1, p and the copy c
      // from n: value r' + 2 c, diagonal p + q.  Exact: every accumulator
      // holds an integer of magnitude at most 512 * 128^2 = 2^23, and a
      // diagonal sum of a CTA at most 8 warps * 9 entries * 2^23 < 2^31.
      // the diagonal of an entry: base + off, base = (grp >> 1) + tig (C = 4)
      // or (grp >> 1) + 2 tig (C = 2), off = 8 mt + 4 h + 4 nt (C = 4) or
      // 8 mt + 4 h + 8 nt + (e & 1) (C = 2): off is known at compile time
      constexpr int NOFF = 8 * (MT - 1) + 4 + (NB == 2 ? 4 * (NT - 1) : 8 * (NT - 1) + 1) + 1;
      const int base = (grp >> 1) + (NB == 2 ? tig : 2 * tig);
#pragma unroll
      for (int c = 0; c < NB; c++) {
        int d[NOFF];
#pragma unroll
        for (int k = 0; k < NOFF; k++) d[k] = 0;
#pragma unroll
        for (int mt = 0; mt < MT; mt++)
#pragma unroll
          for (int nt = 0; nt < NT; nt++)
#pragma unroll
            for (int e = 0; e < 4; e++) {
              const int h = e >> 1;
              const int q = 8 * mt + 4 * h + (grp >> 1);
              const int n = 8 * nt + 2 * tig + (e & 1);
              const int p = NB == 2 ? n >> 1 : n, cc = NB == 2 ? (e & 1) : 0;
              const int off = 8 * mt + 4 * h + (NB == 2 ? 4 * nt : 8 * nt + (e & 1));
              if (cc == c && q < P && p < P) {
                float z = 0.f;
#pragma unroll
                for (int k = 0; k < NA; k++) z += acc[k][mt][nt][e];
                d[off] += __float2int_rn(z);
              }
            }
        // the diagonals this thread holds (the others stay zero)
#pragma unroll
        for (int k = 0; k < NOFF; k++)
          if (d[k]) atomicAdd(&dsum[ci][rp + 2 * c][base + k], d[k]);
      }
    }
  }
  __syncthreads();
  // value (cluster cc, r): sum_s D_s 256^s (mod 2^192) as six 32-bit words
  if (tid < gact * C) {
    const int cc = tid / C, rv = tid - cc * C;
    W3 v = {0, 0, 0};
#pragma unroll
    for (int k = 0; k < ND; k++) {
      uint64_t v0, v1, v2;
      shl192((int64_t)dsum[cc][rv][k], 8 * k, v0, v1, v2);
      add3(v, v0, v1, v2);
    }
    unsigned long long *o = a.acc + ((j0 + cc) * C + rv) * 6;
#pragma unroll
    for (int wd = 0; wd < 6; wd++) {
      const uint64_t wv = wd < 2 ? v.w0 : wd < 4 ? v.w1 : v.w2;
      unsigned long long x = (uint32_t)(wv >> (32 * (wd & 1)));
      if (w == 0 && a.kb >= 0 && (a.kb >> 5) == wd) x += 1ull << (a.kb & 31);
      if (x) atomicAdd(&o[wd], x);
    }
  }
}

// One CTA per item (group, window) of every product; dynamic shared memory
// holds the staged digits.
template <int P, int C, class Src>
__global__ void __launch_bounds__(kSeedWarps * 32, P >= 9 ? 1 : 3) seed_mma(Src src) {
  pdl_enter();
  extern __shared__ __align__(16) __half seed_sm[];
  int64_t local;
  const SeedArgs &a = src.locate(blockIdx.x, local);
  seed_mma_body<P, C>(a, local, seed_sm);
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
  pdl_enter();
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
  // the CTA's column sums: a shuffle tree in every warp, then one add per warp
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int w = 0; w < 2 * NW; w++) {
    long long v = loc[w];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    if (lane == 0 && w < seed_words && v) atomicAdd(&colsum[w], (unsigned long long)v);
  }
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

// the staged digits may take more than the default 48 KB: opt in once per device
template <int P, int C, class Src>
cudaError_t launch_mma(int64_t blocks, int smem, const Src &src, cudaStream_t s) {
  static bool done[64] = {false};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  if (!done[dev]) {
    e = cudaFuncSetAttribute(seed_mma<P, C, Src>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             kSeedSmemMax);
    if (e != cudaSuccess) return e;
    done[dev] = true;
  }
  (void)launch_k(seed_mma<P, C, Src>, dim3((unsigned)blocks), dim3(kSeedWarps * 32), smem, s, src);
  return cudaSuccess;
}

template <class Src>
cudaError_t launch_kind(int kind, int64_t blocks, int smem, const Src &src, cudaStream_t s) {
  const unsigned grid = (unsigned)blocks;
  switch (kind) {
    case 22: return launch_mma<2, 2>(blocks, smem, src, s);
    case 24: return launch_mma<2, 4>(blocks, smem, src, s);
    case 42: return launch_mma<4, 2>(blocks, smem, src, s);
    case 44: return launch_mma<4, 4>(blocks, smem, src, s);
    case 62: return launch_mma<6, 2>(blocks, smem, src, s);
    case 64: return launch_mma<6, 4>(blocks, smem, src, s);
    case 82: return launch_mma<8, 2>(blocks, smem, src, s);
    case 84: return launch_mma<8, 4>(blocks, smem, src, s);
    case 92: return launch_mma<9, 2>(blocks, smem, src, s);
    case 94: return launch_mma<9, 4>(blocks, smem, src, s);
    case 102: (void)launch_k(seed_wide<2, Src>, dim3(grid), dim3(kWT), 0, s, src); break;
    case 104: (void)launch_k(seed_wide<4, Src>, dim3(grid), dim3(kWT), 0, s, src); break;
    case 108: (void)launch_k(seed_wide<8, Src>, dim3(grid), dim3(kWT), 0, s, src); break;
    case 116: (void)launch_k(seed_wide<16, Src>, dim3(grid), dim3(kWT), 0, s, src); break;
    case 132: (void)launch_k(seed_wide<32, Src>, dim3(grid), dim3(kWT), 0, s, src); break;
    case 164: (void)launch_k(seed_wide<64, Src>, dim3(grid), dim3(kWT), 0, s, src); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaSuccess;
}

}  // namespace

int64_t planes_blocks(const SeedArgs &a) {
  int64_t n = plane_stride(a.lf) + plane_stride(a.lg);
  if (a.ncl * a.C * 6 > n) n = a.ncl * a.C * 6;
  return (n + 255) / 256;
}
int64_t seed_planes_bytes(int64_t lf, int64_t lg, int P) { return planes_halves(lf, lg, P) * 2; }

// digits per coefficient: the top digit x >> 8 (P - 1) must lie in [-128, 127]
int seed_digits(int bf, int bg, int sgn) {
  int need = 0;
  for (const int b : {bf, bg}) {
    const int n = sgn ? (b + 7) / 8 : (b + 8) / 8;
    if (n > need) need = n;
  }
  for (const int P : {2, 4, 6, 8, 9})
    if (need <= P) return P;
  return -1;
}

// windows of kWin indices t' cover [-8, Lf - 1] (f is the shorter operand)
int64_t seed_slices(int64_t lf, int64_t lg, int C) {
  (void)C;
  const int64_t l = lf < lg ? lf : lg;
  return (l + 8 + kWin - 1) / kWin;
}

cudaError_t launch_seed_planes(const SeedArgs *d, const int64_t *prefix, int n, int64_t blocks,
                               cudaStream_t s) {
  if (n == 0 || blocks == 0) return cudaSuccess;
  (void)launch_k(seed_planes<Many<SeedArgs>>, dim3((unsigned)blocks), dim3(256), 0, s, Many<SeedArgs>{d, prefix, n});
  note_launches(1);
  return cudaGetLastError();
}

const int kSeedKindList[kSeedKinds] = {22, 24, 42, 44, 62, 64, 82, 84, 92, 94,
                                        102, 104, 108, 116, 132, 164};

int seed_kind_index(int kind) {
  for (int i = 0; i < kSeedKinds; i++)
    if (kSeedKindList[i] == kind) return i;
  return -1;
}

int make_seed_plan(const uint64_t *f, int64_t lf, int bf, const uint64_t *g, int64_t lg, int bg,
                   int sgn, int kb, int64_t k00, int64_t kstep, int64_t ncl, int C,
                   unsigned long long *acc, uint32_t *seeds, int seed_words, __half *planes,
                   int *status, SeedPlan &sp) {
  sp = SeedPlan{};
  sp.nvalues = ncl * C;
  if (sp.nvalues == 0) return 0;
  if (C != 2 && C != 4) return -1;
  SeedArgs &a = sp.a;
  const bool narrow = bf <= 64 && bg <= 64;
  if (narrow && lf > lg) {  // h_k is symmetric in f and g: let f be the shorter
    const uint64_t *tp = f;
    f = g;
    g = tp;
    const int64_t tl = lf;
    lf = lg;
    lg = tl;
    const int tb = bf;
    bf = bg;
    bg = tb;
  }
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
  a.status = status;
  if (narrow) {
    // the g copies' origin Z = k00 (mod 8) keeps every fragment read aligned,
    // which needs every cluster start k0 = k00 (mod 8); the staged rows keep
    // their bank offsets if kstep is a multiple of 64
    if (a.kb >= 192 || planes == nullptr || kstep % 64 != 0) return -1;
    a.P = seed_digits(bf, bg, sgn);
    if (a.P < 0) return -1;
    a.Z = lg - 1 + ((((k00 - (lg - 1)) % 8) + 8) % 8);
    a.planes = planes;
    // clusters per CTA: as many (4, 2 or 1) as keep the staged digits within
    // the budget (a group's g windows are kstep apart)
    a.G = 4;
    while (a.G > 1 && seed_smem(a.P, C, a.G, kstep) > kSeedSmemMax) a.G /= 2;
    if (seed_smem(a.P, C, a.G, kstep) > kSeedSmemMax) return -1;
    a.smem = (int)seed_smem(a.P, C, a.G, kstep);
    a.slices = seed_slices(lf, lg, C);
    // narrow kinds 10 P + C
    sp.kind = 10 * a.P + C;
    sp.blocks = (ncl + a.G - 1) / a.G * a.slices;
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

cudaError_t launch_seed_planes_one(const SeedPlan &sp, cudaStream_t s) {
  if (!sp.narrow() || sp.blocks == 0) return cudaSuccess;
  (void)launch_k(seed_planes<One<SeedArgs>>, dim3((unsigned)planes_blocks(sp.a)), dim3(256), 0, s,
                 One<SeedArgs>{sp.a});
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_seed_plan(const SeedPlan &sp, cudaStream_t s) {
  if (sp.kind == 0 || sp.blocks == 0) return cudaSuccess;
  const cudaError_t e = launch_kind(sp.kind, sp.blocks, sp.narrow() ? sp.a.smem : 0,
                                    One<SeedArgs>{sp.a}, s);
  if (e != cudaSuccess) return e;
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_seeds_batch(int kind, const SeedArgs *d, const int64_t *prefix, int n,
                               int64_t blocks, int smem, cudaStream_t s) {
  if (n == 0 || blocks == 0) return cudaSuccess;
  const cudaError_t e = launch_kind(kind, blocks, smem, Many<SeedArgs>{d, prefix, n}, s);
  if (e != cudaSuccess) return e;
  note_launches(1);
  return cudaGetLastError();
}

}  // namespace ks
