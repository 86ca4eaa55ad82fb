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

namespace ks {

__global__ void __launch_bounds__(256) pack_kernel(PackArgs a) {
  int64_t total = 0;
  for (int o = 0; o < a.nops; o++) total += a.op[o].ndig;
  const int64_t N = a.N;
  const int b = a.b, d = a.d;
  for (int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; gid < total;
       gid += (int64_t)gridDim.x * blockDim.x) {
    int o = 0;
    int64_t j = gid;
    while (j >= a.op[o].ndig) {
      j -= a.op[o].ndig;
      o++;
    }
    const PackOp &op = a.op[o];
    const int32_t val = digit_at(op, j, N, b, d, a.in_limbs, a.flip);
    op.out[j] = val;
  }
}

cudaError_t launch_pack(const PackArgs &a, cudaStream_t s) {
  int64_t total = 0;
  for (int o = 0; o < a.nops; o++) total += a.op[o].ndig;
  if (total == 0) return cudaSuccess;
  int64_t blocks = (total + 255) / 256;
  if (blocks > 152 * 64) blocks = 152 * 64;
  pack_kernel<<<(unsigned)blocks, 256, 0, s>>>(a);
  note_launches(1);
  return cudaGetLastError();
}

}  // namespace ks
