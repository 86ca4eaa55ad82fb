// Tensor-core engine: exact column sums C_k = sum_i A_i B_(k-i) of signed
// 7-bit digit strings on the 5th-generation tensor cores (tcgen05.mma,
// kind::f16, fp16 operands, fp32 accumulation in tensor memory).
//
// Exactness.  Digits are integers with |D| <= 127, exactly representable in
// fp16.  (A + evaluation whose fields overlap, N < b in the four-point
// variant, first has digits in [0, 254]; those are recoded locally as
// D'_j = D_j - 128 [D_j >= 64] + [D_(j-1) >= 64], which lies in [-64, 127],
// keeps the value, and needs no carry chain.)  One accumulation chunk adds at
// most 128 * 8 products per output digit, so every partial sum stays below
// 128 * 8 * 127^2 = 16,516,096 < 2^24, where fp32 holds every integer
// exactly.  After each chunk the accumulator
// is read out of tensor memory, converted to int32 (exact) and added to
// per-thread integer sums; after a work item the sums of four neighbouring
// digits are merged into one 28-bit-digit column sum and added to global
// memory with a 64-bit atomic.
//
// Blocking (a product of digit strings is a Toeplitz matrix-vector product):
// write output digit k = 128 p + q.  For a block offset delta,
//   C[q, p] += sum_t' A[128 delta + q - 127 + t'] * B[128 (p - delta) + 127 - t'],
// t' = 0..127.  The A factor depends on q + t' only (a Hankel matrix), so its
// 8x8 core matrices depend on q/8 + t'/8 only: the A operand is a strip of
// 8x8 core matrices G_s (G_s[q0][t0] = A[8 s + q0 + t0 - 127]) and one shared
// memory descriptor with both core-matrix strides equal to 128 bytes walks
// it -- no 128 x 128 Toeplitz tile is ever stored.  The strip of one chunk is
// expanded in shared memory from 128 * 8 + 144 consecutive raw digits (one
// bulk copy), so global memory holds 2 bytes per digit.  For B, the reversed digit
// string is cut into rows of 128 digits and stored as 16 K-planes (8 digits =
// 16 bytes per row per plane); the N dimension of the MMA runs over rows, so
// moving from delta to delta + 1 is a 16-byte shift of the B descriptor.
// Both operands are copied to shared memory with cp.async.bulk (one copy for
// the raw A digits, one per B plane) completing on an mbarrier.
//
// Work: a CTA (8 warps, two per SM) owns an output tile of 128 digits x 128
// block columns and a run of accumulation chunks; the tensor core of one CTA
// overlaps the copies and the tensor-memory read-out of the other.  Every
// mbarrier wait is bounded (about one second of %globaltimer); on expiry the
// kernel records KS status 1, waits (bounded) for its own copies and MMAs,
// releases its tensor memory and returns.
#include <cuda_fp16.h>

#include "ks_internal.cuh"
#include "ks_src.cuh"

namespace ks {

namespace {
constexpr int kTM = 128;                   // MMA M: digits per output block column
constexpr int kNT = 128;                   // MMA N: block columns per tile
constexpr int kKS = 8;                     // largest number of delta steps per chunk
constexpr int kThreads = 256;
constexpr int kCoreA = 16 * kKS + 15;      // A strip core matrices per chunk
constexpr int kBRows = kNT + kKS - 1;      // B rows per plane per chunk
constexpr int kStageA = kCoreA * 128;
constexpr int kPlaneB = kBRows * 16;
constexpr int kStageB = 16 * kPlaneB;
constexpr int kRawA = 2 * (128 * kKS + 144);  // raw A digits of one chunk (bytes)
constexpr int kSmem = kStageA + kStageB + kRawA;
constexpr int kPad = kNT + 3 * kKS;        // zero rows on each side of the B planes
constexpr int kMaxItemChunks = 64;
// instruction descriptor, kind::f16: D = f32 (bits 4-5 = 1), A = B = f16
// (bits 7-9, 10-12 = 0), both K-major, N >> 3 at bit 17, M >> 4 at bit 24
constexpr uint32_t kIdesc = (1u << 4) | ((uint32_t)(kNT >> 3) << 17) | ((uint32_t)(kTM >> 4) << 24);
constexpr uint64_t kWaitNs = 1000000000ull;

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
// bounded wait for the phase with the given parity; false on timeout
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = globaltimer();
  while (!mbar_try_wait(bar, parity))
    if (globaltimer() - t0 > kWaitNs) return false;
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
__device__ __forceinline__ void mma_f16(uint32_t dtmem, uint64_t adesc, uint64_t bdesc,
                                        uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(dtmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t *bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(bar))
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
// shared memory matrix descriptor, no swizzle: start, leading (K) and stride
// (M/N) byte offsets between 8x16-byte core matrices, version bits 46-48 = 1
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)(lbo >> 4) << 16) |
         ((uint64_t)(sbo >> 4) << 32) | (1ull << 46);
}
}  // namespace

// ------------------------------------------------------------------ pack
// digit j of an evaluation, recoded into [-127, 127] when its fields overlap
__device__ __forceinline__ int32_t tc_digit(const PackOp &op, int64_t j, int64_t n, int N, int b,
                                            int in_limbs, int flip) {
  if (j < 0 || j >= n) return 0;
  int32_t v = digit_at(op, j, N, b, 7, in_limbs, flip);
  if (op.sigma > 0 && N < b) {
    const int32_t prev = j > 0 ? digit_at(op, j - 1, N, b, 7, in_limbs, flip) : 0;
    v = v - (v >= 64 ? 128 : 0) + (prev >= 64 ? 1 : 0);
  }
  return v;
}

template <class Src>
__global__ void __launch_bounds__(256) tc_pack_kernel(Src src) {
  int64_t local;
  const TcPackArgs &a = src.locate(blockIdx.x, local);
  const int64_t perA = a.nAraw, perB = 16 * a.rows * 8, per = perA + perB;
  const int64_t total = per * a.nprod;
  {
    const int64_t e = local * 256 + threadIdx.x;
    if (e >= total) return;
    const int q = (int)(e / per);
    const int64_t r = e - q * per;
    if (r < perA) {
      const int32_t v = tc_digit(a.op[2 * q], r - 127, a.nA, a.N, a.b, a.in_limbs, a.flip);
      a.Araw[q][r] = __int2half_rn(v);
    } else {
      const int64_t r2 = r - perA;
      const int64_t t1 = r2 / (a.rows * 8);
      const int64_t rem = r2 - t1 * a.rows * 8;
      const int64_t rho = rem / 8 - kPad;
      const int t0 = (int)(rem & 7);
      int32_t v = 0;
      if (rho >= 0 && rho < a.R)
        v = tc_digit(a.op[2 * q + 1], 128 * a.R - 1 - (128 * rho + 8 * t1 + t0), a.nB, a.N, a.b,
                     a.in_limbs, a.flip);
      a.BRT[q][r2] = __int2half_rn(v);
    }
  }
}

// ------------------------------------------------------------------ MMA
template <class Src>
__global__ void __launch_bounds__(kThreads, 2) tc_kernel(Src src, int64_t total) {
  extern __shared__ __align__(1024) uint8_t smem[];
  __shared__ __align__(8) uint64_t bar_full;
  __shared__ __align__(8) uint64_t bar_mma;
  __shared__ uint32_t tmem_sh;
  __shared__ int bad_range;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  uint8_t *sA = smem;                       // expanded Hankel strip
  uint8_t *sB = smem + kStageA;             // 16 B planes
  uint8_t *sR = smem + kStageA + kStageB;   // raw A digits of the chunk

  if (warp == 0) {
    tmem_alloc(&tmem_sh, kNT);
    tmem_relinquish();
  }
  if (tid == 0) {
    mbar_init(&bar_full, 1);
    mbar_init(&bar_mma, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    bad_range = 0;
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_sh;
  uint32_t ph_full = 0, ph_mma = 0;
  bool aborted = false, load_pending = false, mma_pending = false;

  const int quad = warp & 3, half = warp >> 2;
  int *status = nullptr;
  const int qd = quad * 32 + lane;  // this thread's digit row (TMEM lane)

  for (int64_t gitem = blockIdx.x; gitem < total && !aborted; gitem += gridDim.x) {
    int64_t item;
    const TcArgs &a = src.locate(gitem, item);
    status = a.status;
    int qp = 0;
    while (qp + 1 < a.nprod && item >= a.item_prefix[qp + 1]) qp++;
    const TcProduct &P = a.p[qp];
    const int64_t local = item - a.item_prefix[qp];
    const int64_t t = local / P.items_per_tile;
    const int64_t g = local - t * P.items_per_tile;
    const int64_t P0 = t * kNT;
    const int64_t dlo = P0 - P.R + 1 > 0 ? P0 - P.R + 1 : 0;
    const int64_t dhi = P0 + kNT - 1 < P.dmax ? P0 + kNT - 1 : P.dmax;
    if (dlo > dhi) continue;
    const int ks = P.ks;
    const int64_t nchunks = (dhi - dlo + ks) / ks;
    const int64_t c0 = g * a.chunks_per_item;
    const int64_t c1 = c0 + a.chunks_per_item < nchunks ? c0 + a.chunks_per_item : nchunks;
    if (c0 >= c1) continue;

    // one chunk's operands: raw A digits and 16 B planes
    auto issue = [&](int64_t c) {
      const int64_t d0 = dlo + c * ks;
      const int64_t x0 = 128 * d0;
      const uint32_t abytes = (uint32_t)(2 * (128 * ks + 144));
      const int64_t rho0 = P.R - P0 - kNT + d0 + kPad;
      const uint32_t rbytes = (uint32_t)(kNT + ks - 1) * 16u;
      if (x0 < 0 || x0 + 128 * ks + 144 > P.nAraw || rho0 < 0 ||
          rho0 + kNT + ks - 1 > P.rows) {
        bad_range = 1;
        mbar_arrive(&bar_full);  // complete the phase without copies
        return;
      }
      mbar_expect_tx(&bar_full, abytes + 16u * rbytes);
      bulk_g2s(sR, P.Araw + x0, abytes, &bar_full);
      for (int t1 = 0; t1 < 16; t1++)
        bulk_g2s(sB + t1 * kPlaneB, P.BRT + (t1 * P.rows + rho0) * 8, rbytes, &bar_full);
    };

    int32_t acc[64];
#pragma unroll
    for (int i = 0; i < 64; i++) acc[i] = 0;
    if (tid == 0) issue(c0);
    load_pending = true;
    for (int64_t c = c0; c < c1; c++) {
      bool ok = mbar_wait(&bar_full, ph_full);
      ph_full ^= 1;
      if (__syncthreads_or(!ok)) {
        aborted = true;
        break;
      }
      load_pending = false;
      // expand the Hankel strip: core matrix s, row q0 = raw digits [8 s + q0, 8 s + q0 + 8)
      {
        const uint32_t *raw = reinterpret_cast<const uint32_t *>(sR);
        const int nrows = (16 * ks + 15) * 8;
        for (int rr = tid; rr < nrows; rr += kThreads) {
          const int h0 = rr;  // 8 * s + q0 == row index
          uint4 o;
          if ((h0 & 1) == 0) {
            const int w = h0 >> 1;
            o = make_uint4(raw[w], raw[w + 1], raw[w + 2], raw[w + 3]);
          } else {
            const int w = h0 >> 1;
            const uint32_t x0 = raw[w], x1 = raw[w + 1], x2 = raw[w + 2], x3 = raw[w + 3],
                           x4 = raw[w + 4];
            o = make_uint4(__funnelshift_r(x0, x1, 16), __funnelshift_r(x1, x2, 16),
                           __funnelshift_r(x2, x3, 16), __funnelshift_r(x3, x4, 16));
          }
          *reinterpret_cast<uint4 *>(sA + (size_t)rr * 16) = o;
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
      }
      if (tid == 0) {
        tc_fence_after();
        const uint32_t a0 = smem_u32(sA), b0 = smem_u32(sB);
        for (int j = 0; j < ks; j++)
#pragma unroll
          for (int k = 0; k < 8; k++) {
            const uint64_t ad = sdesc(a0 + (uint32_t)(16 * j + 2 * k) * 128u, 128u, 128u);
            const uint64_t bd = sdesc(b0 + (uint32_t)(2 * k) * kPlaneB + (uint32_t)j * 16u,
                                      (uint32_t)kPlaneB, 128u);
            mma_f16(tmem, ad, bd, kIdesc, (j | k) != 0 ? 1u : 0u);
          }
        mma_commit(&bar_mma);
      }
      mma_pending = true;
      ok = mbar_wait(&bar_mma, ph_mma);
      ph_mma ^= 1;
      if (__syncthreads_or(!ok)) {
        aborted = true;
        break;
      }
      mma_pending = false;
      if (c + 1 < c1) {
        if (tid == 0) issue(c + 1);  // the MMAs are done with the stage
        load_pending = true;
      }
      tc_fence_after();
      const uint32_t taddr = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(half * 64);
      uint32_t r[32];
      tmem_ld32(taddr, r);
      tmem_wait_ld();
#pragma unroll
      for (int i = 0; i < 32; i++) acc[i] += __float2int_rn(__uint_as_float(r[i]));
      tmem_ld32(taddr + 32, r);
      tmem_wait_ld();
#pragma unroll
      for (int i = 0; i < 32; i++) acc[32 + i] += __float2int_rn(__uint_as_float(r[i]));
      tc_fence_before();
      __syncthreads();
    }
    if (aborted) break;
    // four neighbouring digits (lanes) -> one 28-bit-digit column sum
#pragma unroll 4
    for (int i = 0; i < 64; i++) {
      const long long v0 = acc[i];
      const long long v1 = __shfl_down_sync(0xffffffffu, v0, 1);
      const long long v2 = __shfl_down_sync(0xffffffffu, v0, 2);
      const long long v3 = __shfl_down_sync(0xffffffffu, v0, 3);
      if ((lane & 3) == 0) {
        const long long v = v0 + v1 * 128 + v2 * 16384 + v3 * 2097152;
        const int64_t p = P0 + kNT - 1 - (half * 64 + i);
        const int64_t kappa = 32 * p + (qd >> 2);
        if (v != 0 && kappa < P.ncols)
          atomicAdd(reinterpret_cast<unsigned long long *>(P.C + kappa), (unsigned long long)v);
      }
    }
  }

  if (aborted) {
    if (tid == 0) {
      if (status) atomicExch(status, 1);
      if (load_pending) mbar_wait(&bar_full, ph_full ^ 1);
      if (mma_pending) mbar_wait(&bar_mma, ph_mma ^ 1);
    }
  }
  if (tid == 0 && bad_range && status) atomicExch(status, 3);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) tmem_dealloc(tmem, kNT);
}

// ------------------------------------------------------------------ host
void tc_geometry(int64_t nA, int64_t nB, TcGeom &g) {
  g.nA = nA;
  g.nB = nB;
  g.dmax = (nA + 126) / 128;
  g.R = (nB + 127) / 128;
  g.Pcols = g.dmax + g.R;
  g.T = (g.Pcols + kNT - 1) / kNT;
  g.nG = 128 * (g.dmax + 1 + kKS) + 288;  // raw A digits, offset by 127
  g.rows = g.R + 2 * kPad;
  g.ncols = (nA + nB - 2) / 4 + 1;
}

size_t tc_operand_bytes(const TcGeom &g) {
  return (((size_t)g.nG * 2 + 255) & ~(size_t)255) + (size_t)16 * g.rows * 16;
}
static size_t raw_bytes(const TcGeom &g) { return ((size_t)g.nG * 2 + 255) & ~(size_t)255; }

void make_tc_pack_args(const PackArgs &pa, const TcGeom &g, int nprod, char *base,
                       TcPackArgs &a, int64_t &blocks) {
  a = TcPackArgs{};
  for (int i = 0; i < 2 * nprod; i++) a.op[i] = pa.op[i];
  a.nprod = nprod;
  a.N = pa.N;
  a.b = pa.b;
  a.in_limbs = pa.in_limbs;
  a.flip = pa.flip;
  const size_t per = tc_operand_bytes(g);
  for (int q = 0; q < nprod; q++) {
    a.Araw[q] = reinterpret_cast<__half *>(base + q * per);
    a.BRT[q] = reinterpret_cast<__half *>(base + q * per + raw_bytes(g));
  }
  a.nAraw = g.nG;
  a.rows = g.rows;
  a.R = g.R;
  a.nA = g.nA;
  a.nB = g.nB;
  blocks = ((g.nG + 16 * g.rows * 8) * nprod + 255) / 256;
}

cudaError_t launch_tc_pack(const PackArgs &pa, const TcGeom &g, int nprod, char *base,
                           cudaStream_t s) {
  TcPackArgs a;
  int64_t blocks;
  make_tc_pack_args(pa, g, nprod, base, a, blocks);
  tc_pack_kernel<One<TcPackArgs>><<<(unsigned)blocks, 256, 0, s>>>(One<TcPackArgs>{a});
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_tc_pack_batch(const TcPackArgs *d, const int64_t *prefix, int n,
                                 int64_t blocks, cudaStream_t s) {
  if (n == 0 || blocks == 0) return cudaSuccess;
  tc_pack_kernel<Many<TcPackArgs>><<<(unsigned)blocks, 256, 0, s>>>(Many<TcPackArgs>{d, prefix, n});
  note_launches(1);
  return cudaGetLastError();
}

static cudaError_t tc_attr() {
  static bool attr_done[64] = {false};
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
    attr_done[dev] = true;
  }
  return cudaSuccess;
}

// chunks per item for a total chunk count: enough items for ~8 per CTA slot
static int chunks_per_item(int64_t total_chunks) {
  int64_t cpi = (total_chunks + 1215) / 1216;
  if (cpi < 1) cpi = 1;
  if (cpi > kMaxItemChunks) cpi = kMaxItemChunks;
  return (int)cpi;
}

int64_t tc_chunks(const TcGeom &g, int nprod, const int *ks) {
  int64_t total = 0;
  for (int q = 0; q < nprod; q++) {
    const int64_t span = g.dmax + 1 < g.R + kNT - 1 ? g.dmax + 1 : g.R + kNT - 1;
    total += (span + ks[q] - 1) / ks[q] * g.T;
  }
  return total;
}

void make_tc_args(const TcGeom &g, int nprod, const int *ks, char *base, int64_t *const *C,
                  int *status, int cpi, TcArgs &a) {
  a = TcArgs{};
  a.nprod = nprod;
  a.status = status;
  a.chunks_per_item = cpi;
  const size_t per = tc_operand_bytes(g);
  a.item_prefix[0] = 0;
  for (int q = 0; q < nprod; q++) {
    const int64_t span = g.dmax + 1 < g.R + kNT - 1 ? g.dmax + 1 : g.R + kNT - 1;
    const int64_t cmax = (span + ks[q] - 1) / ks[q];
    TcProduct &P = a.p[q];
    P.Araw = reinterpret_cast<const __half *>(base + q * per);
    P.nAraw = g.nG;
    P.BRT = reinterpret_cast<const __half *>(base + q * per + raw_bytes(g));
    P.rows = g.rows;
    P.dmax = g.dmax;
    P.R = g.R;
    P.T = g.T;
    P.items_per_tile = (cmax + cpi - 1) / cpi;
    P.ks = ks[q];
    P.C = C[q];
    P.ncols = g.ncols;
    a.item_prefix[q + 1] = a.item_prefix[q] + g.T * P.items_per_tile;
  }
}

cudaError_t launch_tc_products(const TcGeom &g, int nprod, const int *ks, char *base,
                               int64_t *const *C, int *status, cudaStream_t s) {
  cudaError_t e = tc_attr();
  if (e != cudaSuccess) return e;
  TcArgs a;
  make_tc_args(g, nprod, ks, base, C, status, chunks_per_item(tc_chunks(g, nprod, ks)), a);
  const int64_t items = a.item_prefix[nprod];
  if (items <= 0) return cudaSuccess;
  const int64_t grid = items < 2 * 152 ? items : 2 * 152;
  tc_kernel<One<TcArgs>><<<(unsigned)grid, kThreads, kSmem, s>>>(One<TcArgs>{a}, items);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_tc_batch(const TcArgs *d, const int64_t *prefix, int n, int64_t items,
                            cudaStream_t s) {
  if (n == 0 || items == 0) return cudaSuccess;
  cudaError_t e = tc_attr();
  if (e != cudaSuccess) return e;
  const int64_t grid = items < 2 * 152 ? items : 2 * 152;
  tc_kernel<Many<TcArgs>><<<(unsigned)grid, kThreads, kSmem, s>>>(Many<TcArgs>{d, prefix, n}, items);
  note_launches(1);
  return cudaGetLastError();
}

int tc_batch_chunks_per_item(int64_t total_chunks) { return chunks_per_item(total_chunks); }

}  // namespace ks
