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

template <class Src>
__global__ void __launch_bounds__(256) pack_kernel(Src src) {
  int64_t local;
  const PackArgs &a = src.locate(blockIdx.x, local);
  int64_t j = local * 256 + threadIdx.x;
  int o = 0;
  while (o < a.nops && j >= a.op[o].ndig) {
    j -= a.op[o].ndig;
    o++;
  }
  if (o >= a.nops) return;
  a.op[o].out[j] = digit_at(a.op[o], j, a.N, a.b, a.d, a.in_limbs, a.flip);
}

int64_t pack_blocks(const PackArgs &a) {
  int64_t total = 0;
  for (int o = 0; o < a.nops; o++) total += a.op[o].ndig;
  return (total + 255) / 256;
}

cudaError_t launch_pack(const PackArgs &a, cudaStream_t s) {
  const int64_t blocks = pack_blocks(a);
  if (blocks == 0) return cudaSuccess;
  pack_kernel<One<PackArgs>><<<(unsigned)blocks, 256, 0, s>>>(One<PackArgs>{a});
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_pack_batch(const PackArgs *d, const int64_t *prefix, int n, int64_t blocks,
                              cudaStream_t s) {
  if (blocks == 0) return cudaSuccess;
  pack_kernel<Many<PackArgs>><<<(unsigned)blocks, 256, 0, s>>>(Many<PackArgs>{d, prefix, n});
  note_launches(1);
  return cudaGetLastError();
}

}  // namespace ks
