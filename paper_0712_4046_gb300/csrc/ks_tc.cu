// Tensor-core engine: exact column sums C_k = sum_i A_i B_(k-i) of signed
// 8-bit digit strings on the 5th-generation tensor cores (tcgen05.mma,
// kind::f16, fp16 operands, fp32 accumulation in tensor memory).
//
// Digits and exactness.  Each evaluation digit D_j (a signed sum of at most
// P <= 8 bit slices of 8 bits, Sec. 3) is recoded into the balanced form
//   D'_j = D_j - 256 c_j + c_(j-1),   c_j = floor((D_j + 128) / 256),
// which keeps the value of the digit string (one more top digit holds the
// last carry), needs no carry chain, and gives |D'_j| <= 128 + P <= 136
// (fp16 holds it exactly).  An accumulation chunk of ks <= 7 block offsets
// adds at most 7 * 128 products per output digit, so every partial sum stays
// below 896 * 136^2 = 16,572,416 < 2^24 and fp32 holds it exactly.  After
// each chunk the accumulator is read out of tensor memory, converted to int32
// (exact) and added to per-thread integer sums; after a work item the sums of
// four neighbouring digits are merged into one 32-bit-digit column sum and
// added to global memory with 64-bit reductions.
//
// Blocking (a product of digit strings is a Toeplitz matrix-vector product):
// write output digit k = 128 p + q.  For a block offset delta,
//   C[q, p] += sum_t' A[128 delta + q - 127 + t'] * B[128 (p - delta) + 127 - t'],
// t' = 0..127.  The A factor depends on q + t' only (a Hankel matrix), so its
// 8x8 core matrices depend on q/8 + t'/8 only: the A operand of a chunk is a
// strip of 16 ks + 15 core matrices G_s (G_s[q0][t0] = A[8 s + q0 + t0 - 127])
// and one shared memory descriptor with both core-matrix strides equal to 128
// bytes walks it -- no 128 x 128 Toeplitz tile is ever stored.  Row h of a
// core-matrix strip is the window of eight digits A[h - 127 .. h - 120]; the
// packing kernel writes every such window once (16 bytes per digit position),
// so the strip of a chunk is one contiguous bulk copy.  For B, the reversed
// digit string is cut into rows of 128 digits and stored as 16 K-planes (8
// digits = 16 bytes per row per plane); the N dimension of the MMA runs over
// rows (column n of the accumulator is block column p = P0 + 127 - n), so
// moving from delta to delta + 1 is a 16-byte shift of the B descriptor.
//
// Trimming.  For a block offset delta only block columns with
// 0 <= p - delta < R meet B; the MMA of that offset covers just those columns,
// rounded out to multiples of 16 (its N and its accumulator column offset),
// so the triangles at both ends of a tile cost almost nothing.  A chunk opens
// with one MMA of an all-zero A strip that clears the whole accumulator.  The
// B planes carry 16 zero rows on each side, enough for the rounding.
//
// Split.  An MMA costs about the same whatever its trimmed N, so the unit of
// work is one block offset of one tile (eight MMAs), and the CTAs take equal
// contiguous ranges of the offsets of all tiles.  A CTA's share may start and
// end inside a tile; its chunks are runs of up to kKS offsets from wherever
// that share starts.
//
// Pipeline (one CTA per SM, persistent over work items of (sub-product,
// output tile, run of block offsets)): warp 0 copies the operands of each
// chunk into a ring of kStages shared memory stages (cp.async.bulk completing
// on an mbarrier), warp 1 issues the MMAs of a chunk into one of kNumAcc
// tensor memory accumulators and commits them to the stage's "empty" and the
// accumulator's "full" barrier, and eight epilogue warps read each
// accumulator out while the tensor core fills the next one.  Every mbarrier wait is bounded (about
// one second of %globaltimer); on expiry the CTA records KS status 1, waits
// (bounded) for its own copies and MMAs, releases its tensor memory and
// returns.
#include <cuda_fp16.h>

#include <atomic>
#include <vector>

#include "ks_internal.cuh"
#include "ks_src.cuh"

namespace ks {

namespace {
constexpr int kTM = 128;                   // MMA M: digits per output block column
constexpr int kNT = 128;                   // MMA N (largest): block columns per tile
constexpr int kKS = 7;                     // largest number of delta steps per chunk
constexpr int kStages = 3;
constexpr int kCoreA = 16 * kKS + 15;      // A strip core matrices per chunk
constexpr int kBRows = kNT + kKS - 1;      // B rows per plane per chunk
constexpr int kStageA = kCoreA * 128;
constexpr int kPlaneB = kBRows * 16;
constexpr int kStageB = 16 * kPlaneB;
constexpr int kStage = kStageA + kStageB;
constexpr int kZeroA = 17 * 128;           // all-zero strip of the clearing MMA
constexpr int kSmem = kStages * kStage + kZeroA;
constexpr int kPadB = 16;                  // zero rows on each side of the B planes
constexpr int kEpiWarps = 8;
constexpr int kThreads = 64 + 32 * kEpiWarps;
constexpr int kNumAcc = 4;
constexpr int kTmemCols = kNT * kNumAcc;
constexpr int kMaxItemChunks = 128;        // int32 sums: 128 * 16,572,416 < 2^31
constexpr int kPackSeg = 2048;             // A window rows / reversed B digits per pack CTA
constexpr int kPackStageWords = 2048;       // coefficient words a pack CTA stages (16 KB)
// instruction descriptor, kind::f16: D = f32 (bits 4-5 = 1), A = B = f16
// (bits 7-9, 10-12 = 0), both K-major, N >> 3 at bit 17, M >> 4 at bit 24
constexpr uint32_t kIdescM = (1u << 4) | ((uint32_t)(kTM >> 4) << 24);
constexpr uint64_t kWaitNs = 1000000000ull;  // default bound of every wait (1 s)
static_assert(kSmem <= 227 * 1024, "shared memory");

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ uint64_t globaltimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// bounded wait (limit ns of %globaltimer) for the phase with the given
// parity; false on timeout
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, uint64_t limit) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = globaltimer();
  while (!mbar_try_wait(bar, parity))
    if (globaltimer() - t0 > limit) return false;
  return true;
}
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void tmem_alloc(uint32_t *dst, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                   smem_u32(dst)),
               "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
// one MMA (kind::f16, fp32 accumulate), issued by lane 0 of a warp that executes the
// call in uniform control flow
__device__ __forceinline__ void mma_f16_lane0(uint32_t dtmem, uint64_t adesc, uint64_t bdesc,
                                              uint32_t idesc, uint32_t accumulate, uint32_t lane) {
  asm volatile(
      "{\n\t.reg .pred p, e;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "setp.eq.u32 e, %5, 0;\n\t"
      "@e tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(dtmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate), "r"(lane)
      : "memory");
}
__device__ __forceinline__ void mma_commit_lane0(uint64_t *bar, uint32_t lane) {
  asm volatile(
      "{\n\t.reg .pred e;\n\t"
      "setp.eq.u32 e, %1, 0;\n\t"
      "@e tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n\t}" ::"r"(
          smem_u32(bar)), "r"(lane)
      : "memory");
}
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
        "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
        "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld() {
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}
// bulk reduction (add, u64) of `bytes` from shared to global memory, bulk async-group
// shared memory matrix descriptor, no swizzle: start, leading (K) and stride
// (M/N) byte offsets between 8x16-byte core matrices, version bits 46-48 = 1
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)(lbo >> 4) << 16) |
         ((uint64_t)(sbo >> 4) << 32) | (1ull << 46);
}
}  // namespace

// ------------------------------------------------------------------ pack
__device__ __forceinline__ int32_t carry8(int32_t d) { return (d + 128) >> 8; }
// balanced recoding of digit d whose lower neighbour is prev
__device__ __forceinline__ int32_t recode8(int32_t d, int32_t prev) {
  return d - (carry8(d) << 8) + carry8(prev);
}

// One CTA writes kPackSeg rows of an A window array or 16 storage rows of the
// 16 B planes of one sub-product: first the plain 8-bit digits of the segment
// (one more for the recoding carry) into shared memory, then the recoded
// fp16 digits in the operand layout, 16 bytes per thread, coalesced.
template <class Src>
__global__ void __launch_bounds__(256) tc_pack_kernel(Src src) {
  pdl_enter();
  __shared__ int32_t raw[kPackSeg + 8];
  __shared__ __align__(16) __half dig[kPackSeg + 8];
  __shared__ uint64_t cf[kPackStageWords];  // the segment's coefficients, when they fit
  int64_t local;
  const TcPackArgs &a = src.locate(blockIdx.x, local);
  const int64_t per = a.segA + a.segB;
  const int tid = threadIdx.x;
  if (local >= per * a.nprod) {  // the column sums the product kernel accumulates into
    const int64_t i0 = (local - per * a.nprod) * 2048;
    for (int i = tid; i < 2048; i += 256)
      if (i0 + i < a.nzero) a.zero[i0 + i] = 0;
    return;
  }
  const int q = (int)(local / per);
  const int64_t r = local - q * per;
  if (r < a.segA) {
    // window rows h in [h0, h0 + kPackSeg); row h = digits h - 127 .. h - 120
    const PackOp &op = a.op[2 * q];
    const int64_t h0 = r * kPackSeg;
    const int64_t x0 = h0 - 127;
    // digits x0 - 1 + i, i < kPackSeg + 8: runs of eight per thread (digits
    // at negative positions come out as zero)
    int64_t t_lo, t_hi, src0;
    field_range<8>(op, x0 - 1, x0 + kPackSeg + 6, a.N, a.ninv, op.b, t_lo, t_hi);
    const bool staged = stage_coeffs(op, t_lo, t_hi, op.il, cf, kPackStageWords, src0);
    __syncthreads();
    for (int i0 = 8 * tid; i0 < kPackSeg + 8; i0 += 8 * 256) {
      int32_t v[8];
      if (staged)
        digit_run<8, 8>(op, x0 - 1 + i0, a.N, a.ninv, op.b, op.il, a.flip, v, cf, src0);
      else
        digit_run<8, 8>(op, x0 - 1 + i0, a.N, a.ninv, op.b, op.il, a.flip, v);
#pragma unroll
      for (int m = 0; m < 8; m++) raw[i0 + m] = v[m];
    }
    __syncthreads();
    for (int i = tid; i < kPackSeg + 7; i += 256) dig[i] = __int2half_rn(recode8(raw[i + 1], raw[i]));
    __syncthreads();
    __half *E = a.E[q];
    for (int i = tid; i < kPackSeg; i += 256) {
      const int64_t h = h0 + i;
      if (h >= a.nE) break;
      uint32_t w[4];
#pragma unroll
      for (int u = 0; u < 4; u++)
        w[u] = (uint32_t)__half_as_ushort(dig[i + 2 * u]) |
               ((uint32_t)__half_as_ushort(dig[i + 2 * u + 1]) << 16);
      *reinterpret_cast<uint4 *>(E + h * 8) = make_uint4(w[0], w[1], w[2], w[3]);
    }
  } else {
    // storage rows s in [s0, s0 + 16) of every plane; storage row s is the
    // reversed row rho = s - kPadB, which holds reversed digits 128 rho .. + 127
    const PackOp &op = a.op[2 * q + 1];
    const int64_t s0 = (r - a.segA) * 16;
    const int64_t rho0 = s0 - kPadB;
    const int64_t top = 128 * a.R - 1;  // digit index of reversed position 0
    // reversed digits j = top - (128 rho0 + m), m <= kPackSeg: runs of eight
    // consecutive j per thread, zero outside [0, top]
    int64_t t_lo, t_hi, src0;
    field_range<8>(op, top - 128 * rho0 - kPackSeg - 7, top - 128 * rho0, a.N, a.ninv, op.b, t_lo,
                   t_hi);
    const bool staged = stage_coeffs(op, t_lo, t_hi, op.il, cf, kPackStageWords, src0);
    __syncthreads();
    for (int m0 = 8 * tid; m0 < kPackSeg + 1; m0 += 8 * 256) {
      const int64_t jhi = top - (128 * rho0 + m0);  // j of m0; j of m0 + 7 is jhi - 7
      int32_t v[8];
      if (staged)
        digit_run<8, 8>(op, jhi - 7, a.N, a.ninv, op.b, op.il, a.flip, v, cf, src0);
      else
        digit_run<8, 8>(op, jhi - 7, a.N, a.ninv, op.b, op.il, a.flip, v);
#pragma unroll
      for (int u = 0; u < 8; u++) {
        const int64_t j = jhi - u;
        if (m0 + u < kPackSeg + 1) raw[m0 + u] = (j < 0 || j > top) ? 0 : v[7 - u];
      }
    }
    __syncthreads();
    for (int m = tid; m < kPackSeg; m += 256) dig[m] = __int2half_rn(recode8(raw[m], raw[m + 1]));
    __syncthreads();
    const int t1 = tid >> 4, u = tid & 15;
    const int64_t s = s0 + u;
    if (s < a.rows) {
      const int64_t rho = rho0 + u;
      uint4 o = make_uint4(0u, 0u, 0u, 0u);
      if (rho >= 0 && rho < a.R) o = *reinterpret_cast<const uint4 *>(dig + 128 * u + 8 * t1);
      *reinterpret_cast<uint4 *>(a.BRT[q] + (t1 * a.rows + s) * 8) = o;
    }
  }
}

// ------------------------------------------------------------------ MMA
namespace {
// Output tile t (block columns 128 t .. 128 t + 127) meets the block offsets
// delta in [dlo, dhi]; they form nch chunks of kKS offsets.  Every tile
// t < T meets at least one offset.
__host__ __device__ __forceinline__ void tc_tile(int64_t dmax, int64_t R, int64_t t,
                                                 int64_t &dlo, int64_t &dhi, int64_t &nch) {
  dlo = 128 * t - R + 1 > 0 ? 128 * t - R + 1 : 0;
  dhi = 128 * t + 127 < dmax ? 128 * t + 127 : dmax;
  nch = (dhi - dlo) / kKS + 1;
}

// The unit of work is one block offset of one output tile (eight MMAs of
// N <= 128; their cost hardly depends on N).  Offsets of the tiles before tile
// t, in closed form: the sum over t' < t of
// min(dmax, 128 t' + 127) - max(0, 128 t' - R + 1) + 1, each bound linear in
// t' on one side of its clipping point.
__host__ __device__ __forceinline__ int64_t tc_offset_prefix(int64_t dmax, int64_t R, int64_t t) {
  const int64_t T = (dmax + R + kNT - 1) / kNT;
  if (t > T) t = T;
  if (t <= 0) return 0;
  const int64_t na = dmax >= kNT - 1 ? (dmax - (kNT - 1)) / kNT + 1 : 0;  // dhi unclipped
  const int64_t m = t < na ? t : na;
  const int64_t s_hi = (kNT / 2) * m * (m - 1) + (kNT - 1) * m + (t - m) * dmax;
  const int64_t n0 = (R - 1) / kNT + 1;  // dlo = 0
  const int64_t s_lo = t > n0 ? (kNT / 2) * (n0 + t - 1) * (t - n0) - (R - 1) * (t - n0) : 0;
  return s_hi - s_lo + t;
}

// one work item, as the producer hands it to the MMA issuer and the epilogue
struct __align__(16) TcSlot {
  const __half *E, *BRT;
  int64_t *C;
  int *status;
  int64_t nE, rows, R, ncols, P0, dlo, dhi;
  int c0, c1, pad, done;
};
constexpr int kItemSlots = 4;

// tc_decode gives the item that starts at offset position s: that offset and
// the ones after it in the same tile, up to position s_end and at most
// kMaxItemChunks chunks of kKS offsets; `next` is the position after the item.
// Requires s < s_end.  hdesc >= 0: the item lies in tile htile of sub-product
// hq of descriptor hdesc (the host's split says so for a CTA's first item),
// which saves the searches and their dependent loads.
template <class Src>
__device__ void tc_decode(const Src &src, int64_t s, int64_t s_end, TcSlot &it, int64_t &next,
                          int hdesc = -1, int hq = 0, int64_t htile = 0) {
  int64_t local;
  const TcArgs &a = hdesc >= 0 ? src.at(hdesc, s, local) : src.locate(s, local);
  int q = hq;
  if (hdesc < 0)
    while (q + 1 < a.nprod && local >= a.work_prefix[q + 1]) q++;
  const TcProduct &P = a.p[q];
  const int64_t L = local - a.work_prefix[q];
  int64_t tlo = htile, thi = P.T - 1;  // last tile whose prefix is <= L
  if (hdesc >= 0) thi = tlo;
  while (tlo < thi) {
    const int64_t mid = (tlo + thi + 1) >> 1;
    if (tc_offset_prefix(P.dmax, P.R, mid) <= L)
      tlo = mid;
    else
      thi = mid - 1;
  }
  int64_t dlo, dhi, nch;
  tc_tile(P.dmax, P.R, tlo, dlo, dhi, nch);
  const int64_t da = dlo + (L - tc_offset_prefix(P.dmax, P.R, tlo));
  int64_t db = da + (s_end - s) - 1;
  if (db > dhi) db = dhi;
  if (db > da + (int64_t)kKS * kMaxItemChunks - 1) db = da + (int64_t)kKS * kMaxItemChunks - 1;
  it.E = P.E;
  it.BRT = P.BRT;
  it.C = P.C;
  it.status = a.status;
  it.nE = P.nE;
  it.rows = P.rows;
  it.R = P.R;
  it.ncols = P.ncols;
  it.P0 = tlo * kNT;
  it.dlo = da;
  it.dhi = db;
  it.c0 = 0;
  it.c1 = (int)((db - da) / kKS + 1);
  it.pad = 0;
  it.done = 0;
  next = s + (db - da + 1);
}

__device__ __forceinline__ void slot_store(TcSlot *dst, const TcSlot &v) {
  const uint4 *s = reinterpret_cast<const uint4 *>(&v);
  uint4 *d = reinterpret_cast<uint4 *>(dst);
#pragma unroll
  for (int i = 0; i < (int)(sizeof(TcSlot) / 16); i++) d[i] = s[i];
}
__device__ __forceinline__ void slot_load(TcSlot &v, const TcSlot *src) {
  const uint4 *s = reinterpret_cast<const uint4 *>(src);
  uint4 *d = reinterpret_cast<uint4 *>(&v);
#pragma unroll
  for (int i = 0; i < (int)(sizeof(TcSlot) / 16); i++) d[i] = s[i];
}
}  // namespace

// wait_ns bounds every wait of the kernel; stall (a test hook) makes the copy
// warp wait, before its first copy, on a barrier that nothing completes, so the
// kernel's waits run out while no copy or MMA is in flight.
template <class Src>
__global__ void __launch_bounds__(kThreads, 1)
    tc_kernel(Src src, int64_t total, uint64_t wait_ns, int stall,
              const __grid_constant__ TcSplit split) {
  extern __shared__ __align__(1024) uint8_t smem[];
  __shared__ __align__(8) uint64_t bar_full[kStages];
  __shared__ __align__(8) uint64_t bar_empty[kStages];
  __shared__ __align__(8) uint64_t bar_tfull[kNumAcc];
  __shared__ __align__(8) uint64_t bar_tempty[kNumAcc];
  __shared__ __align__(8) uint64_t bar_ifull[kItemSlots];
  __shared__ __align__(8) uint64_t bar_iempty[kItemSlots];
  __shared__ __align__(8) uint64_t bar_drain;
  __shared__ __align__(8) uint64_t bar_never;  // the stall hook's: nothing arrives on it
  __shared__ TcSlot slots[kItemSlots];
  __shared__ uint32_t tmem_sh;
  __shared__ int abort_sh, bad_range_sh;
  __shared__ int *status_sh;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  volatile int *abort_v = &abort_sh;

  // this CTA's share of the offsets: the host's split, else an even one
  const bool hsplit = split.n == (int)gridDim.x;
  const int64_t s_beg = hsplit ? split.at[blockIdx.x] : total * blockIdx.x / gridDim.x;
  const int64_t s_end = hsplit ? split.at[blockIdx.x + 1] : total * (blockIdx.x + 1) / gridDim.x;
  // the producer decodes its first item (descriptor loads) while the other
  // warps set up shared and tensor memory
  TcSlot first_it;
  int64_t first_next = s_end;
  if (tid == 0 && s_beg < s_end) {
    if (hsplit)
      tc_decode(src, s_beg, s_end, first_it, first_next, split.desc[blockIdx.x],
                split.q[blockIdx.x], split.tile[blockIdx.x]);
    else
      tc_decode(src, s_beg, s_end, first_it, first_next);
  }
  // the B planes and the zero strip start as zeros: B rows a chunk does not
  // copy stay finite (the clearing MMA multiplies them by zero)
  if (warp > 0) {
    for (int st = 0; st < kStages; st++)
      for (int i = tid - 32; i < kStageB / 16; i += kThreads - 32)
        reinterpret_cast<uint4 *>(smem + st * kStage + kStageA)[i] = make_uint4(0u, 0u, 0u, 0u);
    for (int i = tid - 32; i < kZeroA / 16; i += kThreads - 32)
      reinterpret_cast<uint4 *>(smem + kStages * kStage)[i] = make_uint4(0u, 0u, 0u, 0u);
  }
  if (warp == 1) {  // allocates (and at the end releases) the tensor memory
    tmem_alloc(&tmem_sh, kTmemCols);
    tmem_relinquish();
  }
  if (tid == 64) {
    for (int s = 0; s < kStages; s++) {
      mbar_init(&bar_full[s], 1);
      mbar_init(&bar_empty[s], 1);
    }
    for (int b = 0; b < kNumAcc; b++) {
      mbar_init(&bar_tfull[b], 1);
      mbar_init(&bar_tempty[b], kEpiWarps);
    }
    for (int s = 0; s < kItemSlots; s++) {
      mbar_init(&bar_ifull[s], 1);
      mbar_init(&bar_iempty[s], 1 + kEpiWarps);
    }
    mbar_init(&bar_drain, 1);
    mbar_init(&bar_never, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    abort_sh = 0;
    bad_range_sh = 0;
    status_sh = nullptr;
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  // the setup above touched only shared and tensor memory and read the
  // host-written descriptors: it overlaps the previous kernel of the stream
  pdl_enter();
  const uint32_t tmem = tmem_sh;

  if (warp == 0) {
    // ---------------- producer: item sequence, operand copies into the stage ring
    if (lane == 0) {
      int stage = 0, islot = 0;
      uint32_t phase = 0, iphase = 0, armed = 0, armed_par = 0;
      bool aborted = false;
      for (int64_t s = s_beg;;) {
        TcSlot it;
        int64_t next = s_end;
        const bool have = s < s_end;
        if (have && s == s_beg) {
          it = first_it;
          next = first_next;
        } else if (have) {
          tc_decode(src, s, s_end, it, next);
        } else {
          it.done = 1;
        }
        if (!mbar_wait(&bar_iempty[islot], iphase ^ 1, wait_ns) || *abort_v) {
          aborted = true;
          break;
        }
        slot_store(&slots[islot], it);
        mbar_arrive(&bar_ifull[islot]);  // release: the slot is visible to the consumers
        if (++islot == kItemSlots) {
          islot = 0;
          iphase ^= 1;
        }
        if (!have) break;
        s = next;
        if (status_sh == nullptr) status_sh = it.status;
        for (int c = it.c0; c < it.c1; c++) {
          if (!mbar_wait(&bar_empty[stage], phase ^ 1, wait_ns) || *abort_v) {
            aborted = true;
            break;
          }
          if (stall && !mbar_wait(&bar_never, 0, wait_ns)) {  // the test hook: gives up
            aborted = true;
            break;
          }
          uint8_t *sA = smem + stage * kStage;
          uint8_t *sB = sA + kStageA;
          const int64_t d0 = it.dlo + (int64_t)c * kKS;
          const int64_t h0 = 128 * d0;
          const int64_t nrowsA = 128 * kKS + 120;
          const int64_t r0 = it.R - kNT - it.P0 + d0;  // reversed B row of stage row 0
          const int64_t lo = r0 > -kPadB ? r0 : -kPadB;
          const int64_t hi = r0 + kNT + kKS - 1 < it.R + kPadB ? r0 + kNT + kKS - 1 : it.R + kPadB;
          if (h0 < 0 || h0 + nrowsA > it.nE || lo >= hi || hi + kPadB > it.rows) {
            bad_range_sh = 1;
            mbar_arrive(&bar_full[stage]);  // complete the phase without copies
          } else {
            const uint32_t bbytes = (uint32_t)(hi - lo) * 16u;
            mbar_expect_tx(&bar_full[stage], (uint32_t)nrowsA * 16u + 16u * bbytes);
            bulk_g2s(sA, it.E + h0 * 8, (uint32_t)nrowsA * 16u, &bar_full[stage]);
            for (int t1 = 0; t1 < 16; t1++)
              bulk_g2s(sB + t1 * kPlaneB + (lo - r0) * 16,
                       it.BRT + (t1 * it.rows + lo + kPadB) * 8, bbytes, &bar_full[stage]);
          }
          armed |= 1u << stage;
          armed_par = (armed_par & ~(1u << stage)) | (phase << stage);
          if (++stage == kStages) {
            stage = 0;
            phase ^= 1;
          }
        }
        if (aborted) break;
      }
      if (aborted) {
        *abort_v = 1;
        for (int s = 0; s < kStages; s++)  // copies still in flight land before exit
          if (armed & (1u << s)) mbar_wait(&bar_full[s], (armed_par >> s) & 1, wait_ns);
      }
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer: one chunk = clearing MMA + trimmed MMAs.  The
    // whole warp walks the items and chunks, so the descriptors are computed in
    // warp-uniform control flow; lane 0 alone issues each MMA and commit (the
    // predicate sits inside the instruction's asm block).
    int stage = 0, acc = 0, islot = 0;
    uint32_t phase = 0, aphase = 0, iphase = 0;
    bool aborted = false, issued = false;
    const uint32_t lane_u = (uint32_t)lane;
    const uint64_t zdesc = sdesc(smem_u32(smem + kStages * kStage), 128u, 128u);
    for (;;) {
      const bool iok = mbar_wait(&bar_ifull[islot], iphase, wait_ns);
      if (__any_sync(0xffffffffu, !iok || *abort_v)) {
        aborted = true;
        break;
      }
      TcSlot it;
      slot_load(it, &slots[islot]);
      __syncwarp();
      if (lane == 0) mbar_arrive(&bar_iempty[islot]);
      if (++islot == kItemSlots) {
        islot = 0;
        iphase ^= 1;
      }
      if (it.done) break;
      for (int c = it.c0; c < it.c1; c++) {
        const bool ok = mbar_wait(&bar_full[stage], phase, wait_ns) &&
                        mbar_wait(&bar_tempty[acc], aphase ^ 1, wait_ns);
        if (__any_sync(0xffffffffu, !ok || *abort_v)) {
          aborted = true;
          break;
        }
        tc_fence_after();
        const uint32_t a0 = smem_u32(smem + stage * kStage), b0 = a0 + kStageA;
        const uint32_t dt = tmem + (uint32_t)(acc * kNT);
        const int64_t d0 = it.dlo + (int64_t)c * kKS;
        // block columns n' of offset delta: [P0 + 128 - delta - R, P0 + 128 - delta) clipped
        const int64_t top = it.P0 + kNT - d0;
        // when the chunk's first offset covers every block column, its first
        // MMA overwrites the accumulator; otherwise an MMA of the zero strip
        // clears it first
        const bool full0 = top - it.R <= 0 && top >= kNT;
        if (!full0)
          mma_f16_lane0(dt, zdesc, sdesc(b0, (uint32_t)kPlaneB, 128u),
                        kIdescM | ((uint32_t)(kNT >> 3) << 17), 0u, lane_u);
        int jmax = kKS;
        if (d0 + jmax - 1 > it.dhi) jmax = (int)(it.dhi - d0 + 1);
        for (int j = 0; j < jmax; j++) {
          int64_t lo = top - j - it.R;
          int64_t hi = top - j;
          if (lo < 0) lo = 0;
          if (hi > kNT) hi = kNT;
          const uint32_t lo16 = (uint32_t)lo & ~15u;
          const uint32_t hi16 = ((uint32_t)hi + 15u) & ~15u;
          const uint32_t idesc = kIdescM | (((hi16 - lo16) >> 3) << 17);
          // the K steps advance A by two core matrices (256 bytes) and B by two
          // planes; the start-address field of a descriptor is the address / 16
          const uint64_t ad = sdesc(a0 + (uint32_t)(16 * j) * 128u, 128u, 128u);
          const uint64_t bd = sdesc(b0 + ((uint32_t)j + lo16) * 16u, (uint32_t)kPlaneB, 128u);
#pragma unroll
          for (int k = 0; k < 8; k++)
            mma_f16_lane0(dt + lo16, ad + (uint64_t)(16 * k), bd + (uint64_t)((2 * k * kPlaneB) >> 4),
                          idesc, (j == 0 && k == 0 && full0) ? 0u : 1u, lane_u);
        }
        mma_commit_lane0(&bar_empty[stage], lane_u);
        mma_commit_lane0(&bar_tfull[acc], lane_u);
        issued = true;
        if (++stage == kStages) {
          stage = 0;
          phase ^= 1;
        }
        if (++acc == kNumAcc) {
          acc = 0;
          aphase ^= 1;
        }
      }
      if (aborted) break;
    }
    if (aborted) {
      if (lane == 0) *abort_v = 1;
      if (issued) {  // every MMA issued so far completes before the memory is released
        mma_commit_lane0(&bar_drain, lane_u);
        mbar_wait(&bar_drain, 0, wait_ns);
      }
    }
  } else {
    // ---------------- epilogue: tensor memory -> integer sums -> column atomics
    const int quad = warp & 3, half = (warp - 2) >> 2;
    const int u = lane & 3;
    int acc = 0, islot = 0;
    uint32_t aphase = 0, iphase = 0;
    bool aborted = false;
    for (;;) {
      const bool iok = mbar_wait(&bar_ifull[islot], iphase, wait_ns);
      if (__any_sync(0xffffffffu, !iok || *abort_v)) {
        aborted = true;
        break;
      }
      TcSlot it;
      slot_load(it, &slots[islot]);
      __syncwarp();
      if (lane == 0) mbar_arrive(&bar_iempty[islot]);
      if (++islot == kItemSlots) {
        islot = 0;
        iphase ^= 1;
      }
      if (it.done) break;
      int32_t sum[64];
#pragma unroll
      for (int i = 0; i < 64; i++) sum[i] = 0;
      for (int c = it.c0; c < it.c1; c++) {
        const bool ok = mbar_wait(&bar_tfull[acc], aphase, wait_ns);
        if (__any_sync(0xffffffffu, !ok || *abort_v)) {
          aborted = true;
          break;
        }
        tc_fence_after();
        const uint32_t taddr =
            tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(acc * kNT + half * 64);
        uint32_t r[32];
        tmem_ld32(taddr, r);
        tmem_wait_ld();
#pragma unroll
        for (int i = 0; i < 32; i++) sum[i] += __float2int_rn(__uint_as_float(r[i]));
        tmem_ld32(taddr + 32, r);
        tmem_wait_ld();
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&bar_tempty[acc]);
#pragma unroll
        for (int i = 0; i < 32; i++) sum[32 + i] += __float2int_rn(__uint_as_float(r[i]));
        if (++acc == kNumAcc) {
          acc = 0;
          aphase ^= 1;
        }
      }
      if (aborted) break;
      // Four neighbouring digits (lanes 4g .. 4g + 3, weights 256^w) form one
      // 32-bit-digit column sum.  A two-step butterfly over each group of
      // four block columns gives lane 4g + u the whole sum of column i + u:
      // step 1 (lanes u, u ^ 1) pairs the columns i + (u & 1) and
      // i + 2 + (u & 1), step 2 (lanes u, u ^ 2) completes column i + u.
      // The tile's 4096 column sums (block column p = P0 + row, 32 per row)
      // are contiguous in C; every thread adds its 16 with reductions that
      // return nothing (a warp's 32 touch four 64-byte runs), so no warp
      // waits for another and no staging buffer is needed.
      {
        const bool odd = (u & 1) != 0, up = (u & 2) != 0;
        const long long w_me = 1ll << (8 * u), w_x1 = 1ll << (8 * (u ^ 1));
        const int64_t k0 = 32 * it.P0;
        const int64_t n = it.ncols - k0 < 4096 ? it.ncols - k0 : 4096;
        unsigned long long *cb = reinterpret_cast<unsigned long long *>(it.C + k0);
        const int col = 8 * quad + (lane >> 2);
#pragma unroll
        for (int i = 0; i < 64; i += 4) {
          const int32_t m01 = odd ? sum[i + 1] : sum[i];
          const int32_t m23 = odd ? sum[i + 3] : sum[i + 2];
          const int32_t r01 = __shfl_xor_sync(0xffffffffu, odd ? sum[i] : sum[i + 1], 1);
          const int32_t r23 = __shfl_xor_sync(0xffffffffu, odd ? sum[i + 2] : sum[i + 3], 1);
          const long long p01 = (long long)m01 * w_me + (long long)r01 * w_x1;
          const long long p23 = (long long)m23 * w_me + (long long)r23 * w_x1;
          const long long v = (up ? p23 : p01) + __shfl_xor_sync(0xffffffffu, up ? p01 : p23, 2);
          const int idx = (kNT - 1 - half * 64 - i - u) * 32 + col;
          if (v != 0 && idx < n) atomicAdd(cb + idx, (unsigned long long)v);
        }
      }
    }
    if (aborted) *abort_v = 1;
  }

  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (tid == 0 && status_sh) {
    if (*abort_v) atomicCAS(status_sh, 0, 1);
    if (bad_range_sh) atomicCAS(status_sh, 0, 3);
  }
  if (warp == 1) tmem_dealloc(tmem, kTmemCols);
}

// ------------------------------------------------------------------ host
void tc_geometry(int64_t nA, int64_t nB, TcGeom &g) {
  g.nA = nA;
  g.nB = nB;
  g.dmax = (nA + 126) / 128;
  g.R = (nB + 127) / 128;
  g.Pcols = g.dmax + g.R;
  g.T = (g.Pcols + kNT - 1) / kNT;
  g.nE = 128 * (g.dmax + kKS) + 128;  // window rows read by the last chunk, padded
  g.rows = g.R + 2 * kPadB;
  g.ncols = ((nA + nB - 2) / 4 + 2) & ~(int64_t)1;  // even: 16-byte aligned column arrays
}

static size_t window_bytes(const TcGeom &g) { return ((size_t)g.nE * 16 + 255) & ~(size_t)255; }
size_t tc_operand_bytes(const TcGeom &g) { return window_bytes(g) + (size_t)16 * g.rows * 16; }

void make_tc_pack_args(const PackArgs &pa, const TcGeom &g, int nprod, char *base,
                       TcPackArgs &a, int64_t &blocks, int64_t *zero, int64_t nzero) {
  a = TcPackArgs{};
  for (int i = 0; i < 2 * nprod; i++) a.op[i] = pa.op[i];
  a.nprod = nprod;
  a.N = pa.N;
  a.b = pa.b;
  a.in_limbs = pa.in_limbs;
  a.flip = pa.flip;
  a.ninv = pa.ninv;
  const size_t per = tc_operand_bytes(g);
  for (int q = 0; q < nprod; q++) {
    a.E[q] = reinterpret_cast<__half *>(base + q * per);
    a.BRT[q] = reinterpret_cast<__half *>(base + q * per + window_bytes(g));
  }
  a.nE = g.nE;
  a.rows = g.rows;
  a.R = g.R;
  a.nA = g.nA;
  a.nB = g.nB;
  a.segA = (g.nE + kPackSeg - 1) / kPackSeg;
  a.segB = (g.rows + 15) / 16;
  a.zero = zero;
  a.nzero = zero ? nzero : 0;
  blocks = (a.segA + a.segB) * nprod + (a.nzero + 2047) / 2048;
}

cudaError_t launch_tc_pack(const PackArgs &pa, const TcGeom &g, int nprod, char *base,
                           int64_t *zero, int64_t nzero, cudaStream_t s) {
  TcPackArgs a;
  int64_t blocks;
  make_tc_pack_args(pa, g, nprod, base, a, blocks, zero, nzero);
  (void)launch_k(tc_pack_kernel<One<TcPackArgs>>, dim3((unsigned)blocks), dim3(256), 0, s, One<TcPackArgs>{a});
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_tc_pack_batch(const TcPackArgs *d, const int64_t *prefix, int n,
                                 int64_t blocks, cudaStream_t s) {
  if (n == 0 || blocks == 0) return cudaSuccess;
  (void)launch_k(tc_pack_kernel<Many<TcPackArgs>>, dim3((unsigned)blocks), dim3(256), 0, s, Many<TcPackArgs>{d, prefix, n});
  note_launches(1);
  return cudaGetLastError();
}

// per-device launch attributes and SM count (the grid: one CTA per SM)
static cudaError_t tc_attr(int *sms) {
  static bool attr_done[64] = {false};
  static int sm_count[64] = {0};
  int dev = 0;
  cudaError_t e0 = cudaGetDevice(&dev);
  if (e0 != cudaSuccess) return e0;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  if (!attr_done[dev]) {
    cudaError_t e = cudaFuncSetAttribute(tc_kernel<One<TcArgs>>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(tc_kernel<Many<TcArgs>>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             kSmem);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&sm_count[dev], cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    attr_done[dev] = true;
  }
  if (sms) *sms = sm_count[dev] > 0 ? sm_count[dev] : 1;
  return cudaSuccess;
}

int64_t tc_work(const TcGeom &g) { return tc_offset_prefix(g.dmax, g.R, g.T); }

int tc_grid(int64_t work) {
  int sms = 0;
  if (tc_attr(&sms) != cudaSuccess) return 0;
  return (int)(work < sms ? work : sms);
}

// Virtual positions: tile j (in order over all descriptors and sub-products)
// covers [b_j + c j, b_(j+1) + c j) with c = kTcSwitchCost, and the charge
// [b_j + c (j - 1), b_j + c j) before it maps to its start b_j.  Equal shares
// of the virtual length charge every share that runs into a next tile.
void tc_make_split(const TcArgs *args, const int64_t *prefix, int n, int grid, TcSplit &sp) {
  sp.n = 0;
  if (grid < 1 || grid > kTcMaxCtas || n < 1) return;
  struct Tile {
    int64_t b;
    int32_t desc, q, t;
  };
  std::vector<Tile> tiles;
  for (int i = 0; i < n; i++)
    for (int q = 0; q < args[i].nprod; q++) {
      const TcProduct &P = args[i].p[q];
      if ((int64_t)tiles.size() + P.T > (1 << 22)) return;  // too many to walk: even split
      for (int64_t t = 0; t < P.T; t++) {
        const int64_t b = prefix[i] + args[i].work_prefix[q] + tc_offset_prefix(P.dmax, P.R, t);
        if (b < prefix[i] + args[i].work_prefix[q + 1]) tiles.push_back(Tile{b, i, q, (int32_t)t});
      }
    }
  const int64_t total = prefix[n];
  if (tiles.empty() || total <= 0) return;
  const int64_t nt = (int64_t)tiles.size();
  const double V = (double)total + (double)kTcSwitchCost * (double)(nt - 1);
  size_t j = 0;  // tile of the current split point
  sp.at[0] = 0;
  for (int k = 1; k < grid; k++) {
    const double tau = V * k / grid;
    // the last tile whose virtual start is <= tau
    while (j + 1 < tiles.size() &&
           (double)tiles[j + 1].b + (double)kTcSwitchCost * (double)(j + 1) <= tau)
      j++;
    int64_t x;
    if (j + 1 < tiles.size() && tau >= (double)tiles[j + 1].b + (double)kTcSwitchCost * (double)j)
      x = tiles[j + 1].b;  // inside the charge before tile j + 1: snap to its start
    else
      x = (int64_t)(tau - (double)kTcSwitchCost * (double)j);
    if (x < sp.at[k - 1]) x = sp.at[k - 1];
    if (x > total) x = total;
    sp.at[k] = x;
  }
  sp.at[grid] = total;
  // each share's first tile
  size_t u = 0;
  for (int k = 0; k < grid; k++) {
    const int64_t s0 = sp.at[k] < total ? sp.at[k] : total - 1;
    while (u + 1 < tiles.size() && tiles[u + 1].b <= s0) u++;
    sp.desc[k] = tiles[u].desc;
    sp.q[k] = tiles[u].q;
    sp.tile[k] = tiles[u].t;
  }
  sp.n = grid;
}

// the wait bound and the stall hook of the kernel (a test hook; see ks.h)
static std::atomic<int> g_tc_stall{0};
static std::atomic<unsigned long long> g_tc_wait_ns{kWaitNs};

void make_tc_args(const TcGeom &g, int nprod, char *base, int64_t *const *C, int *status,
                  TcArgs &a) {
  a = TcArgs{};
  a.nprod = nprod;
  a.status = status;
  const size_t per = tc_operand_bytes(g);
  a.work_prefix[0] = 0;
  for (int q = 0; q < nprod; q++) {
    TcProduct &P = a.p[q];
    P.E = reinterpret_cast<const __half *>(base + q * per);
    P.nE = g.nE;
    P.BRT = reinterpret_cast<const __half *>(base + q * per + window_bytes(g));
    P.rows = g.rows;
    P.dmax = g.dmax;
    P.R = g.R;
    P.T = g.T;
    P.work = tc_work(g);
    P.C = C[q];
    P.ncols = g.ncols;
    a.work_prefix[q + 1] = a.work_prefix[q] + P.work;
  }
}

cudaError_t launch_tc_products(const TcGeom &g, int nprod, char *base, int64_t *const *C,
                               int *status, cudaStream_t s) {
  int sms = 0;
  cudaError_t e = tc_attr(&sms);
  if (e != cudaSuccess) return e;
  TcArgs a;
  make_tc_args(g, nprod, base, C, status, a);
  const int64_t work = a.work_prefix[nprod];
  if (work <= 0) return cudaSuccess;
  const int64_t grid = work < sms ? work : sms;
  const int64_t prefix[2] = {0, work};
  TcSplit split;
  tc_make_split(&a, prefix, 1, (int)grid, split);
  (void)launch_k(tc_kernel<One<TcArgs>>, dim3((unsigned)grid), dim3(kThreads), kSmem, s,
                 One<TcArgs>{a}, work, g_tc_wait_ns.load(), g_tc_stall.load(), split);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_tc_batch(const TcArgs *d, const int64_t *prefix, int n, int64_t work,
                            const TcSplit &split, cudaStream_t s) {
  if (n == 0 || work == 0) return cudaSuccess;
  int sms = 0;
  cudaError_t e = tc_attr(&sms);
  if (e != cudaSuccess) return e;
  const int64_t grid = work < sms ? work : sms;
  (void)launch_k(tc_kernel<Many<TcArgs>>, dim3((unsigned)grid), dim3(kThreads), kSmem, s,
                 Many<TcArgs>{d, prefix, n}, work, g_tc_wait_ns.load(), g_tc_stall.load(), split);
  note_launches(1);
  return cudaGetLastError();
}

}  // namespace ks

extern "C" void ks_debug_tc_stall(int on, int64_t wait_ns) {
  ks::g_tc_stall.store(on ? 1 : 0);
  ks::g_tc_wait_ns.store(wait_ns > 0 ? (unsigned long long)wait_ns : ks::kWaitNs);
  ks::bump_epoch();
}

// The host's split of one product's tensor-core work over `grid` CTAs (host
// only: plans it without touching the device).
extern "C" int ks_debug_tc_split(int64_t len_f, int64_t len_g, int coeff_bits, int is_signed,
                                 int variant, int grid, int64_t *at, int32_t *first_q,
                                 int32_t *first_tile, int64_t *total) {
  if (!at || !first_q || !first_tile || !total || grid < 1 || grid > ks::kTcMaxCtas)
    return KS_EINVAL;
  ks::Plan p;
  const int rc = ks::make_plan(p, len_f, len_g, coeff_bits, is_signed, variant, KS_ENGINE_TC);
  if (rc != KS_OK) return rc;
  // operand and column-sum addresses are only recorded here, never used
  char *base = reinterpret_cast<char *>(static_cast<uintptr_t>(1) << 20);
  int64_t *C[4];
  for (int q = 0; q < p.nprod; q++) C[q] = reinterpret_cast<int64_t *>(base);
  ks::TcArgs a;
  ks::make_tc_args(p.tg, p.nprod, base, C, nullptr, a);
  const int64_t prefix[2] = {0, a.work_prefix[p.nprod]};
  ks::TcSplit sp;
  ks::tc_make_split(&a, prefix, 1, grid, sp);
  if (sp.n != grid) return KS_ERANGE;
  for (int k = 0; k <= grid; k++) at[k] = sp.at[k];
  for (int k = 0; k < grid; k++) {
    first_q[k] = sp.q[k];
    first_tile[k] = sp.tile[k];
  }
  *total = prefix[1];
  return KS_OK;
}
