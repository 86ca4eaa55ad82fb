// Products in (Z/pZ)[x, y] by the polynomial-ring substitutions of Sec. 2:
// f, g (ly rows of lx residues, row i = the coefficient f_i(x) of y^i) are
// evaluated at y = +-x^N or +-x^-N into univariate polynomials of (Z/pZ)[x],
// the univariate products run through the library's (Z/pZ)[x] product, and
// the rows h_k of h are read off or recovered:
//
//   KS_1  Sec. 2.1: y = x^N, N = 2 lx - 1; the h_k do not overlap.
//   KS_2  Sec. 2.3: y = +-x^N, N = lx; (P+ + P-)/2 holds the even h_k,
//         (P+ - P-)/2 the odd ones, at spacing 2N, without overlap.
//   KS_3  Sec. 2.2: y = x^N and x^-N, N = lx; consecutive h_k overlap by
//         N - 1 terms, and the low half of h_k comes from the forward product,
//         the high half from the reversed one, each after subtracting the
//         neighbouring half of h_(k-1) (the subtraction Sec. 2.2 describes).
//   KS_4  Sec. 2.4: all four points, N = ceil(lx / 2); the rows of f overlap
//         already in the evaluations; the even and the odd h_k are recovered
//         as in KS_3 at spacing 2N.
//   KS_C  Sec. 2.5: y = x^M, -x^M, i x^M, M = ceil(lx / 2), in R[i]; the
//         complex product as three real ones; the rows k = r (mod 4) are read
//         off a quarter of a combination of the five products.
//
// All arithmetic is on residues in [0, p), p < 2^63 (no overflow in a + b);
// halving (KS_2, KS_4) needs p odd.
#include "ks_internal.cuh"

namespace ks {

namespace {
__device__ __forceinline__ uint64_t add_p(uint64_t a, uint64_t b, uint64_t p) {
  const uint64_t s = a + b;
  return s >= p ? s - p : s;
}
__device__ __forceinline__ uint64_t sub_p(uint64_t a, uint64_t b, uint64_t p) {
  return a >= b ? a - b : a + (p - b);
}
// a / 2 mod p for odd p
__device__ __forceinline__ uint64_t half_p(uint64_t a, uint64_t p) {
  return (a & 1) ? (a >> 1) + (p >> 1) + 1 : a >> 1;
}

// E[m] = sum over the rows i whose chunk [i N, i N + lx) holds m of
// s_i f_(pi(i))[m - i N] mod p, with pi the identity or the reversal of the
// rows and s_i = -1 for odd i at a negated point.
__global__ void __launch_bounds__(256) biv_eval(const __grid_constant__ BivEvalArgs a) {
  pdl_enter();
  const BivEval &e = a.e[blockIdx.y];
  for (int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; m < e.len;
       m += (int64_t)gridDim.x * blockDim.x) {
    int64_t i_hi = m / e.N;
    if (i_hi > e.ly - 1) i_hi = e.ly - 1;
    const int64_t lo = m - (e.lx - 1);
    const int64_t i_lo = lo > 0 ? (lo + e.N - 1) / e.N : 0;
    uint64_t acc = 0;
    for (int64_t i = i_lo; i <= i_hi; i++) {
      if ((e.part == 1 && (i & 1)) || (e.part == 2 && !(i & 1))) continue;
      const int64_t row = e.reversed ? e.ly - 1 - i : i;
      const uint64_t v = e.f[row * e.lx + (m - i * e.N)];
      const bool neg = e.part ? ((i >> 1) & 1) != 0 : (e.alternate && (i & 1));
      acc = neg ? sub_p(acc, v, e.p) : add_p(acc, v, e.p);
    }
    e.out[m] = acc;
  }
}

// KS_1 / KS_2: h[k][j] = P1[k N + j] (KS_1), or (P1 + (-1)^k P2)[k N + j] / 2
// (KS_2: the even rows from the sum, the odd ones from the difference).
__global__ void __launch_bounds__(256) biv_readoff(BivReadArgs a) {
  pdl_enter();
  const int64_t hx = 2 * a.lx - 1, total = (2 * a.ly - 1) * hx;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t k = idx / hx, j = idx - k * hx;
    const int64_t src = k * a.N + j;
    uint64_t v = a.P1[src];
    if (a.P2 != nullptr) {
      const uint64_t w = a.P2[src];
      v = half_p((k & 1) ? sub_p(v, w, a.p) : add_p(v, w, a.p), a.p);
    }
    a.h[idx] = v;
  }
}

// KS_C (Sec. 2.5): at q = k M + j, with s = P1 + P2, d = P1 - P2 (the points
// +-x^M), Re = P3 - P4, Im = P5 - P3 - P4 (the point i x^M):
//   h[k][j] = (s + 2 Re) / 4, (d + 2 Im) / 4, (s - 2 Re) / 4, (d - 2 Im) / 4
// for k = 0, 1, 2, 3 (mod 4).
__global__ void __launch_bounds__(256) biv_readoff_complex(BivComplexArgs a) {
  pdl_enter();
  const uint64_t p = a.p;
  const int64_t hx = 2 * a.lx - 1, total = (2 * a.ly - 1) * hx;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t k = idx / hx, j = idx - k * hx;
    const int64_t q = k * a.M + j;
    const uint64_t p1 = a.P[0][q], p2 = a.P[1][q], p3 = a.P[2][q], p4 = a.P[3][q],
                   p5 = a.P[4][q];
    uint64_t v, w;
    if (k & 1) {
      v = sub_p(p1, p2, p);                                // d
      w = sub_p(sub_p(p5, p3, p), p4, p);                  // Im
    } else {
      v = add_p(p1, p2, p);                                // s
      w = sub_p(p3, p4, p);                                // Re
    }
    const uint64_t w2 = add_p(w, w, p);
    const uint64_t t = (k & 2) ? sub_p(v, w2, p) : add_p(v, w2, p);
    a.h[idx] = half_p(half_p(t, p), p);
  }
}

// A(m) = P1[m], or (P1 +- P2)[m + shift] / 2 (the combinations of Sec. 2.4).
__device__ __forceinline__ uint64_t comb(const BivSeq &q, int64_t m, uint64_t p) {
  const int64_t i = m + q.shift;
  if (m < 0 || i >= q.len) return 0;
  const uint64_t v = q.P1[i];
  if (q.P2 == nullptr) return v;
  const uint64_t w = q.P2[i];
  return half_p(q.sign > 0 ? add_p(v, w, p) : sub_p(v, w, p), p);
}

// Reciprocal recovery (Sec. 2.2): blocks c_0 .. c_(n-1) of length ell <= 2M - 1
// at spacing M, from A = sum c_k x^(kM) and B = sum c_(n-1-k) x^(kM):
//   c_k[j]     = A[k M + j]       - c_(k-1)[M + j]    (0 <= j < M)
//   c_k[M + j] = B[(n - k) M + j] - c_(k-1)[j]        (M + j < ell)
// Thread j carries c_(k-1)[j] and c_(k-1)[M + j] from block to block; block
// k is row row0 + rstep k of h.
__global__ void __launch_bounds__(128) biv_recover(BivRecoverArgs a) {
  pdl_enter();
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= a.M) return;
  const int64_t hx = 2 * a.lx - 1;
  const bool has_hi = a.M + j < a.ell;
  uint64_t lo_prev = 0, hi_prev = 0;
  for (int64_t k = 0; k < a.n; k++) {
    const uint64_t lo = sub_p(comb(a.A, k * a.M + j, a.p), hi_prev, a.p);
    const uint64_t hi = has_hi ? sub_p(comb(a.B, (a.n - k) * a.M + j, a.p), lo_prev, a.p) : 0;
    uint64_t *row = a.h + (a.row0 + a.rstep * k) * hx;
    if (j < a.ell) row[j] = lo;
    if (has_hi) row[a.M + j] = hi;
    lo_prev = lo;
    hi_prev = hi;
  }
}

unsigned grid1(int64_t n, int threads) {
  int64_t b = (n + threads - 1) / threads;
  if (b < 1) b = 1;
  if (b > 152 * 16) b = 152 * 16;
  return (unsigned)b;
}
}  // namespace

cudaError_t launch_biv_eval(const BivEvalArgs &a, int64_t maxlen, cudaStream_t s) {
  if (a.n < 1 || a.n > kMaxBivEvals) return cudaErrorInvalidValue;
  (void)launch_k(biv_eval, dim3(dim3(grid1(maxlen, 256), (unsigned)a.n)), dim3(256), 0, s, a);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_biv_readoff(const BivReadArgs &a, cudaStream_t s) {
  (void)launch_k(biv_readoff, dim3(grid1((2 * a.ly - 1) * (2 * a.lx - 1), 256)), dim3(256), 0, s, a);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_biv_readoff_complex(const BivComplexArgs &a, cudaStream_t s) {
  (void)launch_k(biv_readoff_complex, dim3(grid1((2 * a.ly - 1) * (2 * a.lx - 1), 256)),
                 dim3(256), 0, s, a);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_biv_recover(const BivRecoverArgs &a, cudaStream_t s) {
  if (a.n < 1) return cudaSuccess;
  (void)launch_k(biv_recover, dim3((unsigned)((a.M + 127) / 128)), dim3(128), 0, s, a);
  note_launches(1);
  return cudaGetLastError();
}

}  // namespace ks
