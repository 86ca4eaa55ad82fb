// Schoolbook engine: exact column sums C_k = sum_i A_i B_(k-i) of signed-digit
// operands on the INT32 pipe (each term one 32x32->64-bit multiply-add).
//
// This is the classical integer product the paper's analysis starts from
// (Sec. 1: M(b) ~ b^alpha with alpha = 2 in the classical regime), written
// for the GPU as a 2-D tiling of the (i, j) product plane:
//
//   * a CTA owns output columns [k0, k0 + 2048) and a chunk of 1024 indices i;
//   * thread t owns the aligned 8x8 blocks (i, j) of the plane whose corner
//     satisfies i + j = k0 + 8t, walking along that anti-diagonal: each step
//     loads 8 digits of A (a shared-memory broadcast) and 8 of B (contiguous
//     across the warp) and does 64 multiply-adds into 15 int64 column
//     accumulators -- four 16-byte loads per 64 MACs;
//   * neighbouring threads' 15-column windows overlap by 7 columns; those
//     partial sums are handed to the next thread through shared memory, and
//     each column is added once to global memory with a 64-bit atomic.
//
// Split over i (split-K) supplies the parallelism; the atomics make the
// partial sums of different CTAs meet without a separate reduction pass.
#include "ks_internal.cuh"
#include "ks_src.cuh"

namespace ks {

namespace {
constexpr int kThreads = 256;
constexpr int kR = 8;
constexpr int kTK = kThreads * kR;  // output columns per CTA
constexpr int kTI = 1024;           // i-chunk per CTA
}  // namespace

template <class Src>
__global__ void __launch_bounds__(kThreads) schoolbook_kernel(Src src) {
  pdl_enter();
  __shared__ __align__(16) int32_t sA[kTI];
  __shared__ __align__(16) int32_t sB[kTK + kTI];
  __shared__ long long sHi[kThreads][7];

  int64_t bid;
  const SchoolArgs &a = src.locate(blockIdx.x, bid);
  int p = 0;
  while (p + 1 < a.nprod && bid >= a.block_prefix[p + 1]) p++;
  const Product P = a.p[p];
  const int64_t local = bid - a.block_prefix[p];
  const int64_t ct = local / a.ichunks[p];
  const int64_t ic = local % a.ichunks[p];
  const int64_t k0 = ct * kTK;
  const int64_t i0 = ic * kTI;
  const int64_t ncols = P.nA + P.nB - 1;
  const int64_t i_end = (i0 + kTI < P.nA) ? i0 + kTI : P.nA;
  // any (i, j) with i in [i0, i_end), j in [0, nB), i + j in [k0, k0 + kTK + 7)?
  if (i0 >= P.nA || k0 + kTK + 6 - i0 < 0 || k0 - (i_end - 1) >= P.nB) return;

  const int t = threadIdx.x;
  const int64_t jlo = k0 - i0 - kTI + 8;
  for (int y = t; y < kTI; y += kThreads) {
    int64_t i = i0 + y;
    sA[y] = (i < P.nA) ? P.A[i] : 0;
  }
  for (int x = t; x < kTK + kTI; x += kThreads) {
    int64_t jj = jlo + x;
    sB[x] = (jj >= 0 && jj < P.nB) ? P.B[jj] : 0;
  }
  __syncthreads();

  long long acc[2 * kR - 1];
#pragma unroll
  for (int r = 0; r < 2 * kR - 1; r++) acc[r] = 0;

  const int ib_end = (int)(i_end - i0);
  for (int ib = 0; ib < ib_end; ib += kR) {
    const int4 a0 = *reinterpret_cast<const int4 *>(&sA[ib]);
    const int4 a1 = *reinterpret_cast<const int4 *>(&sA[ib + 4]);
    const int jb = kR * t + kTI - kR - ib;
    const int4 b0 = *reinterpret_cast<const int4 *>(&sB[jb]);
    const int4 b1 = *reinterpret_cast<const int4 *>(&sB[jb + 4]);
    const int av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
    const int bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
    for (int ii = 0; ii < kR; ii++)
#pragma unroll
      for (int jj = 0; jj < kR; jj++) acc[ii + jj] += (long long)av[ii] * bv[jj];
  }

#pragma unroll
  for (int r = 0; r < kR - 1; r++) sHi[t][r] = acc[kR + r];
  __syncthreads();
  const int64_t kb = k0 + (int64_t)kR * t;
#pragma unroll
  for (int r = 0; r < kR; r++) {
    long long v = acc[r];
    if (t > 0 && r < kR - 1) v += sHi[t - 1][r];
    const int64_t k = kb + r;
    if (v != 0 && k < ncols)
      atomicAdd(reinterpret_cast<unsigned long long *>(P.C + k), (unsigned long long)v);
  }
  if (t == kThreads - 1) {
#pragma unroll
    for (int r = 0; r < kR - 1; r++) {
      const long long v = acc[kR + r];
      const int64_t k = kb + kR + r;
      if (v != 0 && k < ncols)
        atomicAdd(reinterpret_cast<unsigned long long *>(P.C + k), (unsigned long long)v);
    }
  }
}

int make_school_args(const Product *prods, int nprod, SchoolArgs &a) {
  if (nprod < 1 || nprod > 4) return -1;
  a = SchoolArgs{};
  a.nprod = nprod;
  a.block_prefix[0] = 0;
  for (int p = 0; p < nprod; p++) {
    a.p[p] = prods[p];
    const int64_t ncols = prods[p].nA + prods[p].nB - 1;
    const int64_t ctiles = (ncols + kTK - 1) / kTK;
    a.ichunks[p] = (prods[p].nA + kTI - 1) / kTI;
    a.block_prefix[p + 1] = a.block_prefix[p] + ctiles * a.ichunks[p];
  }
  return 0;
}

cudaError_t launch_schoolbook(const Product *prods, int nprod, cudaStream_t s) {
  SchoolArgs a;
  if (make_school_args(prods, nprod, a) != 0) return cudaErrorInvalidValue;
  const int64_t blocks = a.block_prefix[nprod];
  if (blocks <= 0) return cudaSuccess;
  if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
  (void)launch_k(schoolbook_kernel<One<SchoolArgs>>, dim3((unsigned)blocks), dim3(kThreads), 0, s, One<SchoolArgs>{a});
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_schoolbook_batch(const SchoolArgs *d, const int64_t *prefix, int n,
                                    int64_t blocks, cudaStream_t s) {
  if (blocks <= 0) return cudaSuccess;
  if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
  (void)launch_k(schoolbook_kernel<Many<SchoolArgs>>, dim3((unsigned)blocks), dim3(kThreads), 0, s,
                 Many<SchoolArgs>{d, prefix, n});
  note_launches(1);
  return cudaGetLastError();
}

}  // namespace ks
