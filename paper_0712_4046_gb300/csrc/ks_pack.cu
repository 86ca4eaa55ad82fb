// Pack: the evaluations of Sec. 3.1-3.4 as signed digit strings.
//
// An evaluation  F = sum_t s_t c_t 2^(tN)  (c_t the t-th coefficient of the
// polynomial or of its reversal, s_t = -1 for odd t at the point -2^N, else
// +1) is written as digits D_j, j = 0.., with  F = sum_j D_j 2^(d j)  and
//
//   D_j = sum over the coefficients t whose bit field [tN, tN + b) meets
//         [jd, jd + d) of  s_t * (the bits of c_t that fall in that window).
//
// Each digit is a plain sum of at most a few shifted bit slices, so no carry
// or borrow crosses digit positions: negative evaluations (Sec. 3.3: "one-
// padding" alternating with zero-padding) and the overlapping fields of the
// four-point variant (Sec. 3.4, N < b) cost nothing extra here.  The
// sub-product engines take these signed digits as they are, and the single
// carry normalization after the products resolves every carry at once.
//
// Signed inputs are biased to unsigned b-bit values by flipping bit b-1
// (c + 2^(b-1)); the exact correction is applied after unpacking.
#include "ks_internal.cuh"
#include "ks_src.cuh"

namespace ks {

namespace {
constexpr int kPackThreads = 256;
constexpr int kRun = 8;                             // digits per thread
constexpr int kCtaDigits = kPackThreads * kRun;     // digits per CTA
__device__ __forceinline__ int pad8(int i) { return i + (i >> 3); }
__host__ __device__ __forceinline__ int64_t ctas_for(int64_t ndig) {
  return (ndig + kCtaDigits - 1) / kCtaDigits;
}
}  // namespace

// One CTA makes 2048 consecutive digits of one operand: it copies the
// coefficients they read into shared memory (when they fit), each thread
// makes a run of eight (digit_run), and the digits are stored coalesced
// through shared memory.
constexpr int kStageWords = 3072;  // coefficient words staged per CTA (24 KB)

template <class Src>
__global__ void __launch_bounds__(kPackThreads) pack_kernel(Src src) {
  __shared__ int32_t st[kCtaDigits + kCtaDigits / 8];
  __shared__ uint64_t cf[kStageWords];
  int64_t local;
  const PackArgs &a = src.locate(blockIdx.x, local);
  int o = 0;
  while (o < a.nops && local >= ctas_for(a.op[o].ndig)) {
    local -= ctas_for(a.op[o].ndig);
    o++;
  }
  if (o >= a.nops) return;
  const PackOp &op = a.op[o];
  const int tid = threadIdx.x;
  const int64_t jc = local * kCtaDigits;
  // the coefficients this CTA's digits read, staged once (coalesced)
  int64_t t_lo, t_hi, src0;
  field_range<16>(op, jc, jc + kCtaDigits - 1, a.N, a.ninv, a.b, t_lo, t_hi);
  const bool staged = stage_coeffs(op, t_lo, t_hi, a.in_limbs, cf, kStageWords, src0);
  __syncthreads();
  int32_t v[kRun];
  // two call sites, so that the staged one reads shared memory as such
  if (staged)
    digit_run<16, kRun>(op, jc + (int64_t)kRun * tid, a.N, a.ninv, a.b, a.in_limbs, a.flip, v,
                        cf, src0);
  else
    digit_run<16, kRun>(op, jc + (int64_t)kRun * tid, a.N, a.ninv, a.b, a.in_limbs, a.flip, v);
#pragma unroll
  for (int m = 0; m < kRun; m++) st[pad8(kRun * tid + m)] = v[m];
  __syncthreads();
  for (int i = tid; i < kCtaDigits; i += kPackThreads) {
    const int64_t j = jc + i;
    if (j < op.ndig) op.out[j] = st[pad8(i)];
  }
}

void squaring_pack(PackArgs &a, Product *prods, int nprod) {
  for (int q = 0; q < nprod; q++) {
    a.op[q] = a.op[2 * q];
    prods[q].B = prods[q].A;
  }
  a.nops = nprod;
}

void pack_finish(PackArgs &a) {
  a.ninv = a.N > 1 ? (uint64_t)(((unsigned __int128)1 << 64) / (unsigned)a.N) + 1 : 0;
  for (int o = 0; o < a.nops; o++) {
    PackOp &op = a.op[o];
    // largest bit position a digit run or a field reaches (with a margin for
    // the runs past the last digit: the tensor-core window rows reach about
    // 2300 digits beyond it)
    const int64_t top_digit = (op.ndig + 8192) * (int64_t)a.d;
    const int64_t top_field = op.L * (int64_t)a.N + a.b;
    op.narrow = (top_digit < ((int64_t)1 << 31) && top_field < ((int64_t)1 << 31)) ? 1 : 0;
  }
}

int64_t pack_blocks(const PackArgs &a) {
  int64_t total = 0;
  for (int o = 0; o < a.nops; o++) total += ctas_for(a.op[o].ndig);
  return total;
}

cudaError_t launch_pack(const PackArgs &a, cudaStream_t s) {
  if (a.d != 16) return cudaErrorInvalidValue;  // the int32-digit engines use 16-bit digits
  const int64_t blocks = pack_blocks(a);
  if (blocks == 0) return cudaSuccess;
  pack_kernel<One<PackArgs>><<<(unsigned)blocks, kPackThreads, 0, s>>>(One<PackArgs>{a});
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_pack_batch(const PackArgs *d, const int64_t *prefix, int n, int64_t blocks,
                              cudaStream_t s) {
  if (blocks == 0) return cudaSuccess;
  pack_kernel<Many<PackArgs>><<<(unsigned)blocks, kPackThreads, 0, s>>>(
      Many<PackArgs>{d, prefix, n});
  note_launches(1);
  return cudaGetLastError();
}

}  // namespace ks
