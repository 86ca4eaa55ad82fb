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
// Signed inputs are two's complement b-bit values: bit b-1 of a coefficient
// weighs -2^(b-1).  The pieces are taken from c + 2^(b-1) (bit b-1 flipped,
// non-negative) and the digit holding the field's top bit takes 2^(b-1) back,
// so the digits evaluate the signed polynomial itself.
#include "ks_internal.cuh"
#include "ks_src.cuh"

namespace ks {

namespace {
constexpr int kPackThreads = 256;
constexpr int kRun = 8;                             // digits per thread
constexpr int kCtaDigits = kPackThreads * kRun;     // digits per CTA
constexpr int kStageWords = 3072;                   // coefficient words staged per CTA (24 KB)
constexpr int kFieldDigits = 6144;                  // digits of a field-centric CTA (24 KB)
__device__ __forceinline__ int pad8(int i) { return i + (i >> 3); }
__host__ __device__ __forceinline__ int64_t ctas_for(int64_t ndig) {
  return (ndig + kCtaDigits - 1) / kCtaDigits;
}
__host__ __device__ __forceinline__ int64_t op_ctas(const PackArgs &a, const PackOp &op) {
  return a.fields > 0 ? (op.L + a.fields - 1) / a.fields : ctas_for(op.ndig);
}
}  // namespace

// Two ways to a CTA's digits, chosen per plan (block-uniform):
//
//  * digit-centric (any N): a CTA makes 2048 consecutive digits; it copies the
//    coefficients they read into shared memory (when they fit), each thread
//    makes a run of eight (digit_run), and the digits are stored coalesced
//    through shared memory.
//  * field-centric (N >= b, the fields do not overlap): a CTA takes `fields`
//    consecutive coefficient fields and owns the digits from the first one's
//    start to the next CTA's; it stages those coefficients (and the earlier
//    ones whose tails reach its first digit), each thread adds the
//    16-bit pieces of one field into shared digit accumulators (+- by the sign
//    of the evaluation point), and the CTA stores its digit range coalesced.
//    Digits between fields cost nothing but their store.
template <class Src>
__global__ void __launch_bounds__(kPackThreads) pack_kernel(Src src) {
  pdl_enter();
  __shared__ __align__(16) uint64_t raw[kStageWords + kFieldDigits / 2];
  int64_t local;
  const PackArgs &a = src.locate(blockIdx.x, local);
  int o = 0;
  while (o < a.nops && local >= op_ctas(a, a.op[o])) {
    local -= op_ctas(a, a.op[o]);
    o++;
  }
  if (o >= a.nops) return;
  const PackOp &op = a.op[o];
  const int tid = threadIdx.x;
  uint64_t *cf = raw;
  if (a.fields > 0) {
    int32_t *sd = reinterpret_cast<int32_t *>(raw + kStageWords);
    const int64_t N = a.N;
    const int64_t c0 = local * a.fields;
    const int64_t c1 = c0 + a.fields < op.L ? c0 + a.fields : op.L;  // one past the last field
    const int64_t D0 = (c0 * N) >> 4;
    const int64_t D1 = c1 < op.L ? (c1 * N) >> 4 : op.ndig;
    const int nd = (int)(D1 - D0);
    for (int i = tid; i < nd; i += kPackThreads) sd[i] = 0;
    // every field that meets digit D0: the earlier ones only with their tails
    // (more than one when N < 16)
    int64_t src0;
    const int64_t e0 = 16 * D0 - op.b;
    const int64_t t_lo = e0 < 0 ? 0 : e0 / N + 1;
    const bool staged = stage_coeffs(op, t_lo, c1 - 1, op.il, cf, kStageWords, src0);
    __syncthreads();
    const int b = op.b, il = op.il, flip = a.flip;
    const int64_t t = t_lo + tid;  // this thread's field
    if (t < c1) {
      const int64_t pos = t * N;
      const int64_t src = op.reversed ? (op.L - 1 - t) : t;
      const uint64_t *c = staged ? cf + (src - src0) * il : op.poly + src * il;
      const bool neg = op.sigma < 0 && (t & 1);
      int64_t d = pos >> 4;
      int64_t dend = (pos + b - 1) >> 4;
      if (d < D0) d = D0;
      if (dend > D1 - 1) dend = D1 - 1;
      for (; d <= dend; d++) {
        const int x = (int)(16 * d - pos);  // the coefficient's bit at the digit's bit 0
        uint32_t piece;
        if (x >= 0) {
          const int li = x >> 6, sh = x & 63;
          const uint64_t w0 = coeff_limb(c, li, il, b, flip);
          const uint64_t w1 = sh + 16 > 64 ? coeff_limb(c, li + 1, il, b, flip) : 0ull;
          piece = (uint32_t)(((w0 >> sh) | (sh ? w1 << (64 - sh) : 0ull)) & 0xFFFFull);
        } else {
          piece = (uint32_t)((coeff_limb(c, 0, il, b, flip) << (-x)) & 0xFFFFull);
        }
        int32_t val = (int32_t)piece;
        if (flip) {  // the bias of a signed coefficient leaves at its top bit
          const int top = (int)(pos + b - 1 - 16 * d);
          if (top >= 0 && top < 16) val -= (int32_t)1 << top;
        }
        if (val) atomicAdd(&sd[d - D0], neg ? -val : val);
      }
    }
    __syncthreads();
    for (int i = tid; i < nd; i += kPackThreads) op.out[D0 + i] = sd[i];
    return;
  }
  int32_t *st = reinterpret_cast<int32_t *>(raw + kStageWords);
  const int64_t jc = local * kCtaDigits;
  // the coefficients this CTA's digits read, staged once (coalesced)
  int64_t t_lo, t_hi, src0;
  field_range<16>(op, jc, jc + kCtaDigits - 1, a.N, a.ninv, op.b, t_lo, t_hi);
  const bool staged = stage_coeffs(op, t_lo, t_hi, op.il, cf, kStageWords, src0);
  __syncthreads();
  int32_t v[kRun];
  // two call sites, so that the staged one reads shared memory as such
  if (staged)
    digit_run<16, kRun>(op, jc + (int64_t)kRun * tid, a.N, a.ninv, op.b, op.il, a.flip, v,
                        cf, src0);
  else
    digit_run<16, kRun>(op, jc + (int64_t)kRun * tid, a.N, a.ninv, op.b, op.il, a.flip, v);
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
  // field-centric CTAs when the fields do not overlap: as many fields as keep
  // the CTA's digits (about fields N / 16 + 2) and its staged coefficients
  // (fields + 1 of them) in shared memory, at most one per thread but one
  a.fields = 0;
  if (a.d == 16 && a.N >= a.b) {
    // fields before a CTA's first that can still reach its first digit
    const int64_t extra = (16 + a.b - 1) / a.N + 1;
    int64_t c = (int64_t)(kFieldDigits - 2) * 16 / a.N;
    const int64_t cw = kStageWords / a.in_limbs - extra;
    if (cw < c) c = cw;
    if (c > kPackThreads - extra) c = kPackThreads - extra;
    if (c >= 16) a.fields = (int)c;
  }
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
  for (int o = 0; o < a.nops; o++) total += op_ctas(a, a.op[o]);
  return total;
}

cudaError_t launch_pack(const PackArgs &a, cudaStream_t s) {
  if (a.d != 16) return cudaErrorInvalidValue;  // the int32-digit engines use 16-bit digits
  const int64_t blocks = pack_blocks(a);
  if (blocks == 0) return cudaSuccess;
  (void)launch_k(pack_kernel<One<PackArgs>>, dim3((unsigned)blocks), dim3(kPackThreads), 0, s, One<PackArgs>{a});
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_pack_batch(const PackArgs *d, const int64_t *prefix, int n, int64_t blocks,
                              cudaStream_t s) {
  if (blocks == 0) return cudaSuccess;
  (void)launch_k(pack_kernel<Many<PackArgs>>, dim3((unsigned)blocks), dim3(kPackThreads), 0, s, 
      Many<PackArgs>{d, prefix, n});
  note_launches(1);
  return cudaGetLastError();
}

}  // namespace ks
