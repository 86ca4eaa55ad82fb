// Number-theoretic-transform engine: exact column sums C_k = sum_i A_i B_(k-i)
// of signed 16-bit digit strings by cyclic convolution modulo two primes and
// the Chinese remainder theorem (the quasi-linear M(b) regime of Sec. 1, where
// the variants converge, Sec. 4).
//
//   p1 = 15 * 2^27 + 1 = 2013265921 (primitive root 31)
//   p2 = 17 * 2^27 + 1 = 2281701377 (primitive root 3)
//
// Both have 2^27 | p - 1, so transforms of length n = 2^L, L <= 27, exist.
// |C_k| <= min(nA, nB) * (2^17)^2 < P / 2 with P = p1 p2 > 2^61.9 (checked by
// the planner), so the residues identify C_k, signed, exactly.
//
// Arithmetic: Montgomery multiplication with R = 2^32 in the form
// u = hi(a b) - hi(m p), m = lo(a b) p^-1 mod 2^32 (no 64-bit overflow for
// p < 2^32).  Data stay plain residues; twiddles are in Montgomery form.
// Forward transforms are decimation in frequency (natural order in,
// bit-reversed out), the pointwise product keeps the bit-reversed order, and
// the inverse is decimation in time (bit-reversed in, natural out), so no
// permutation pass exists.  A pass takes 4096 elements of one transform and
// runs up to 12 radix-2 stages on them, three at a time in registers (radix
// 8) with shared memory between: the last pass takes contiguous blocks,
// earlier passes take 2^k strided elements for 4096 / 2^k consecutive offsets
// (coalesced).  Twiddles w^e come from two tables per prime and direction,
// w^e = T1[e mod 2^13] * T2[e >> 13], one lookup per unit of eight elements;
// the unit's other twiddles are products with fixed roots of unity.
#include <mutex>

#include "ks_internal.cuh"

namespace ks {

namespace {
constexpr int kMaxLog = 27;
constexpr int kT1 = 1 << 13;
constexpr int kT2 = 1 << 14;
constexpr int kTile = 4096;
constexpr int kTileLog = 12;
constexpr int kPassThreads = 512;
constexpr uint32_t kP[2] = {2013265921u, 2281701377u};
constexpr uint32_t kG[2] = {31u, 3u};

struct PrimeC {
  uint32_t p, pinv;  // pinv = p^-1 mod 2^32
};

__device__ uint32_t g_tw[2][2][kT1 + kT2];  // [prime][forward, inverse][T1 | T2], Montgomery form

__device__ __forceinline__ uint32_t mont_mul(uint32_t a, uint32_t b, uint32_t p, uint32_t pinv) {
  const uint64_t t = (uint64_t)a * b;
  const uint32_t m = (uint32_t)t * pinv;
  const uint32_t th = (uint32_t)(t >> 32);
  const uint32_t mh = __umulhi(m, p);
  return th >= mh ? th - mh : th - mh + p;
}
__device__ __forceinline__ uint32_t add_mod(uint32_t a, uint32_t b, uint32_t p) {
  const uint32_t s = a + b;
  return (s < a || s >= p) ? s - p : s;
}
__device__ __forceinline__ uint32_t sub_mod(uint32_t a, uint32_t b, uint32_t p) {
  return a >= b ? a - b : a - b + p;
}
__device__ __forceinline__ uint32_t twiddle(int prime, int dir, uint32_t e, uint32_t p,
                                            uint32_t pinv) {
  const uint32_t *T = g_tw[prime][dir];
  return mont_mul(__ldg(T + (e & (kT1 - 1))), __ldg(T + kT1 + (e >> 13)), p, pinv);
}

struct NttArgs {
  uint32_t *data;      // arrays of n elements, array id a at data + a * n
  int L;
  int s0, k;           // stages s0 .. s0 + k - 1 in this pass
  int astride;         // the y-th array of this launch is a = y * astride + aoff
  int aoff;
  PrimeC pc[2];
};

// array id -> prime: arrays are laid out [product][prime][side]
__device__ __forceinline__ int prime_of(int a) { return (a >> 1) & 1; }

// zeta[prime][dir][m] = W^(m 2^24) (Montgomery form), W the order-2^27 root of
// the direction: the 8th roots of unity the radix-8 rounds need
__constant__ uint32_t c_zeta[2][2][4];

// One pass: stages s0 .. s0 + k - 1 of one transform on a tile of 2^k rows x
// Wc consecutive offsets (4096 elements when the transform is large enough).
// The stages go in rounds of up to three: a thread takes a unit of 2^g
// elements (rows v0 + m 2^pp, one offset) and runs the round's g radix-2
// stages on them in registers.  Within a unit every twiddle follows from one,
// t = w^(J 2^s) (J the unit's offset in its half-block, s its first stage):
// the first stage multiplies by t zeta_8^m, the second by t^2 zeta_4^m', the
// third by t^4 (for g = 2: t zeta_4^m, then t^2; g = 1: t).  The first
// round reads the transform in global memory, the last writes it back; the
// rounds between exchange through shared memory (one padding word per 32).
__device__ __forceinline__ int sidx(int i) { return i + (i >> 5); }

template <bool kForward>
__global__ void __launch_bounds__(kPassThreads) ntt_pass(NttArgs g) {
  pdl_enter();
  __shared__ uint32_t S[kTile + kTile / 32];
  const int a = blockIdx.y * g.astride + g.aoff;
  const int r = prime_of(a);
  const int dir = kForward ? 0 : 1;
  const uint32_t p = g.pc[r].p, pinv = g.pc[r].pinv;
  uint32_t *X = g.data + ((int64_t)a << g.L);
  const int k = g.k;
  // every extent is a power of two: F = 2^lf rows apart, Wc = 2^lw offsets
  const int lf = g.L - g.s0 - k;
  const int lw = lf < kTileLog - k ? lf : kTileLog - k;
  const int wmask = (1 << lw) - 1;
  const int64_t u = (int64_t)blockIdx.x >> (lf - lw);
  const int64_t w0 = ((int64_t)blockIdx.x & ((((int64_t)1) << (lf - lw)) - 1)) << lw;
  const int64_t gbase = (u << (g.L - g.s0)) + w0;
  const int shift = kMaxLog - g.L;  // exponents in units of the order-2^27 root
  const uint32_t z1 = c_zeta[r][dir][1], z2 = c_zeta[r][dir][2], z3 = c_zeta[r][dir][3];
  const int nr = (k + 2) / 3;
  for (int ri = 0; ri < nr; ri++) {
    const int rr = kForward ? ri : nr - 1 - ri;
    const int r0 = 3 * rr;                       // first stage of the round (in the pass)
    const int gs = (k - r0) < 3 ? (k - r0) : 3;  // stages in the round
    const int pp = k - r0 - gs;                  // rows between a unit's elements: 2^pp
    const int nunits = 1 << (k - gs + lw);
    const bool first = ri == 0, last = ri == nr - 1;
    const int s = g.s0 + r0;                     // global stage of the round's first stage
    for (int un = threadIdx.x; un < nunits; un += kPassThreads) {
      const int wi = un & wmask;
      const int vr = un >> lw;
      const int vlow = vr & ((1 << pp) - 1);
      const int v0 = ((vr >> pp) << (pp + gs)) | vlow;
      const int ne = 1 << gs;
      uint32_t x[8];
#pragma unroll
      for (int m = 0; m < 8; m++) {
        if (m < ne) {
          const int v = v0 + (m << pp);
          x[m] = first ? X[gbase + ((int64_t)v << lf) + wi] : S[sidx((v << lw) | wi)];
        }
      }
      const uint32_t J = (uint32_t)(((int64_t)vlow << lf) + w0 + wi);
      const uint32_t t = twiddle(r, dir, (J << s) << shift, p, pinv);
      if (gs == 3) {
        const uint32_t t2 = mont_mul(t, t, p, pinv), t4 = mont_mul(t2, t2, p, pinv);
        const uint32_t tA[4] = {t, mont_mul(t, z1, p, pinv), mont_mul(t, z2, p, pinv),
                                mont_mul(t, z3, p, pinv)};
        const uint32_t tB[2] = {t2, mont_mul(t2, z2, p, pinv)};
        if (kForward) {
#pragma unroll
          for (int m = 0; m < 4; m++) {
            const uint32_t x0 = x[m], x1 = x[m + 4];
            x[m] = add_mod(x0, x1, p);
            x[m + 4] = mont_mul(sub_mod(x0, x1, p), tA[m], p, pinv);
          }
#pragma unroll
          for (int m = 0; m < 8; m++) {
            if ((m & 2) == 0) {
              const uint32_t x0 = x[m], x1 = x[m + 2];
              x[m] = add_mod(x0, x1, p);
              x[m + 2] = mont_mul(sub_mod(x0, x1, p), tB[m & 1], p, pinv);
            }
          }
#pragma unroll
          for (int m = 0; m < 8; m += 2) {
            const uint32_t x0 = x[m], x1 = x[m + 1];
            x[m] = add_mod(x0, x1, p);
            x[m + 1] = mont_mul(sub_mod(x0, x1, p), t4, p, pinv);
          }
        } else {
#pragma unroll
          for (int m = 0; m < 8; m += 2) {
            const uint32_t x0 = x[m], y = mont_mul(x[m + 1], t4, p, pinv);
            x[m] = add_mod(x0, y, p);
            x[m + 1] = sub_mod(x0, y, p);
          }
#pragma unroll
          for (int m = 0; m < 8; m++) {
            if ((m & 2) == 0) {
              const uint32_t x0 = x[m], y = mont_mul(x[m + 2], tB[m & 1], p, pinv);
              x[m] = add_mod(x0, y, p);
              x[m + 2] = sub_mod(x0, y, p);
            }
          }
#pragma unroll
          for (int m = 0; m < 4; m++) {
            const uint32_t x0 = x[m], y = mont_mul(x[m + 4], tA[m], p, pinv);
            x[m] = add_mod(x0, y, p);
            x[m + 4] = sub_mod(x0, y, p);
          }
        }
      } else if (gs == 2) {
        const uint32_t t2 = mont_mul(t, t, p, pinv);
        const uint32_t tA[2] = {t, mont_mul(t, z2, p, pinv)};
        if (kForward) {
#pragma unroll
          for (int m = 0; m < 2; m++) {
            const uint32_t x0 = x[m], x1 = x[m + 2];
            x[m] = add_mod(x0, x1, p);
            x[m + 2] = mont_mul(sub_mod(x0, x1, p), tA[m], p, pinv);
          }
#pragma unroll
          for (int m = 0; m < 4; m += 2) {
            const uint32_t x0 = x[m], x1 = x[m + 1];
            x[m] = add_mod(x0, x1, p);
            x[m + 1] = mont_mul(sub_mod(x0, x1, p), t2, p, pinv);
          }
        } else {
#pragma unroll
          for (int m = 0; m < 4; m += 2) {
            const uint32_t x0 = x[m], y = mont_mul(x[m + 1], t2, p, pinv);
            x[m] = add_mod(x0, y, p);
            x[m + 1] = sub_mod(x0, y, p);
          }
#pragma unroll
          for (int m = 0; m < 2; m++) {
            const uint32_t x0 = x[m], y = mont_mul(x[m + 2], tA[m], p, pinv);
            x[m] = add_mod(x0, y, p);
            x[m + 2] = sub_mod(x0, y, p);
          }
        }
      } else {
        if (kForward) {
          const uint32_t x0 = x[0], x1 = x[1];
          x[0] = add_mod(x0, x1, p);
          x[1] = mont_mul(sub_mod(x0, x1, p), t, p, pinv);
        } else {
          const uint32_t x0 = x[0], y = mont_mul(x[1], t, p, pinv);
          x[0] = add_mod(x0, y, p);
          x[1] = sub_mod(x0, y, p);
        }
      }
#pragma unroll
      for (int m = 0; m < 8; m++) {
        if (m < ne) {
          const int v = v0 + (m << pp);
          if (last)
            X[gbase + ((int64_t)v << lf) + wi] = x[m];
          else
            S[sidx((v << lw) | wi)] = x[m];
        }
      }
    }
    if (!last) __syncthreads();
  }
}

// The sub-products of one launch: up to four in the kernel's parameters (a
// direct call), or a device array of any number (a plan's batch of equal
// transform lengths).
using NttProd = Product;
struct InlineProds {
  NttProd p[4];
  __device__ __forceinline__ const NttProd &get(int q) const { return p[q]; }
};
struct DeviceProds {
  const NttProd *p;
  __device__ __forceinline__ const NttProd &get(int q) const { return p[q]; }
};

template <class Prods>
struct LoadArgs {
  Prods prods;
  uint32_t *data;
  int L;
  int nprod;
  int square;  // A = B: only the first side is loaded and transformed
  PrimeC pc[2];
};

template <class Prods>
__global__ void __launch_bounds__(256) ntt_load(const __grid_constant__ LoadArgs<Prods> g) {
  pdl_enter();
  const int64_t n = (int64_t)1 << g.L;
  const int64_t total = n * 4 * g.nprod;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int a = (int)(idx >> g.L);
    const int64_t i = idx & (n - 1);
    const int q = a >> 2, r = (a >> 1) & 1, side = a & 1;
    if (g.square && side == 1) continue;
    const uint32_t p = g.pc[r].p;
    const NttProd &pq = g.prods.get(q);
    int32_t d = 0;
    if (side == 0) {
      if (i < pq.nA) d = pq.A[i];
    } else {
      if (i < pq.nB) d = pq.B[i];
    }
    g.data[idx] = d >= 0 ? (uint32_t)d : (uint32_t)((int64_t)d + p);
  }
}

__global__ void __launch_bounds__(256) ntt_pointwise(uint32_t *data, int L, int nprod, PrimeC p0,
                                                     PrimeC p1, int square) {
  pdl_enter();
  const int64_t n = (int64_t)1 << L;
  const int64_t total = n * 2 * nprod;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int qr = (int)(idx >> L);  // product * 2 + prime
    const int64_t i = idx & (n - 1);
    const PrimeC pc = (qr & 1) ? p1 : p0;
    uint32_t *X = data + (int64_t)(2 * qr) * n;
    const uint32_t x = X[i];
    X[i] = mont_mul(x, square ? x : X[n + i], pc.p, pc.pinv);
  }
}

template <class Prods>
struct CrtArgs {
  Prods prods;
  const uint32_t *data;
  int L;
  int nprod;
  PrimeC pc[2];
  uint32_t K[2];      // n^-1 R^2 mod p (Montgomery scale after the inverse transform)
  uint32_t M;         // p1^-1 R mod p2
};

template <class Prods>
__global__ void __launch_bounds__(256) ntt_crt(const __grid_constant__ CrtArgs<Prods> g) {
  pdl_enter();
  const int64_t n = (int64_t)1 << g.L;
  const uint64_t P = (uint64_t)g.pc[0].p * g.pc[1].p;
  const int q = blockIdx.y;  // product
  const NttProd &pq = g.prods.get(q);
  const int64_t ncols = pq.nA + pq.nB - 1;
  int64_t *C = pq.C;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < ncols;
       k += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t z1 = g.data[(int64_t)(4 * q + 0) * n + k];
    const uint32_t z2 = g.data[(int64_t)(4 * q + 2) * n + k];
    const uint32_t c1 = mont_mul(z1, g.K[0], g.pc[0].p, g.pc[0].pinv);
    const uint32_t c2 = mont_mul(z2, g.K[1], g.pc[1].p, g.pc[1].pinv);
    const uint32_t d = sub_mod(c2, c1, g.pc[1].p);  // c1 < p1 < p2
    const uint32_t t = mont_mul(d, g.M, g.pc[1].p, g.pc[1].pinv);
    const uint64_t x = (uint64_t)c1 + (uint64_t)g.pc[0].p * t;  // in [0, P)
    const int64_t v = x > P / 2 ? (int64_t)(x - P) : (int64_t)x;
    C[k] = v;
  }
}

// ---------------------------------------------------------------- host side
uint64_t powmod(uint64_t a, uint64_t e, uint64_t m) {
  uint64_t r = 1 % m;
  a %= m;
  while (e) {
    if (e & 1) r = (unsigned __int128)r * a % m;
    a = (unsigned __int128)a * a % m;
    e >>= 1;
  }
  return r;
}
uint32_t inv_mod_2_32(uint32_t p) {  // Newton iteration for p^-1 mod 2^32 (p odd)
  uint32_t x = p;
  for (int i = 0; i < 5; i++) x *= 2u - p * x;
  return x;
}
PrimeC prime_c(int r) { return PrimeC{kP[r], inv_mod_2_32(kP[r])}; }
uint32_t to_mont(uint64_t x, uint32_t p) { return (uint32_t)(((unsigned __int128)x << 32) % p); }

// The twiddle tables of the current device, loaded once per device by
// blocking copies.  Those copies cannot run inside a stream capture: a first
// use on a capturing stream returns -2 and leaves the capture intact (every
// entry point loads the tables on its first call per device, so a call made
// before the capture is enough).
int init_tables(cudaStream_t s) {
  static std::mutex mu;
  static bool done[64] = {false};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return -1;
  std::lock_guard<std::mutex> lk(mu);
  if (done[dev]) return 0;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (s != nullptr && cudaStreamIsCapturing(s, &cs) != cudaSuccess) return -1;
  if (cs != cudaStreamCaptureStatusNone) return -2;
  static uint32_t host[2][2][kT1 + kT2];
  static bool host_ready = false;
  if (!host_ready) {
    for (int r = 0; r < 2; r++) {
      const uint64_t p = kP[r];
      const uint64_t w = powmod(kG[r], (p - 1) >> kMaxLog, p);  // order 2^27
      const uint64_t wi = powmod(w, p - 2, p);
      for (int dir = 0; dir < 2; dir++) {
        const uint64_t base = dir == 0 ? w : wi;
        uint64_t x = 1;
        for (int i = 0; i < kT1; i++) {
          host[r][dir][i] = to_mont(x, (uint32_t)p);
          x = (unsigned __int128)x * base % p;
        }
        const uint64_t step = powmod(base, kT1, p);
        x = 1;
        for (int i = 0; i < kT2; i++) {
          host[r][dir][kT1 + i] = to_mont(x, (uint32_t)p);
          x = (unsigned __int128)x * step % p;
        }
      }
    }
    host_ready = true;
  }
  if (cudaMemcpyToSymbol(g_tw, host, sizeof(host)) != cudaSuccess) return -1;
  // the 8th roots of unity W^(m 2^24), m < 4, per prime and direction
  uint32_t zeta[2][2][4];
  for (int r = 0; r < 2; r++) {
    const uint64_t p = kP[r];
    const uint64_t w = powmod(kG[r], (p - 1) >> kMaxLog, p);
    const uint64_t wi = powmod(w, p - 2, p);
    for (int dir = 0; dir < 2; dir++) {
      const uint64_t z = powmod(dir == 0 ? w : wi, (uint64_t)1 << 24, p);
      uint64_t x = 1;
      for (int m = 0; m < 4; m++) {
        zeta[r][dir][m] = to_mont(x, (uint32_t)p);
        x = (unsigned __int128)x * z % p;
      }
    }
  }
  if (cudaMemcpyToSymbol(c_zeta, zeta, sizeof(zeta)) != cudaSuccess) return -1;
  done[dev] = true;
  return 0;
}

// passes: earlier ones of <= 8 stages (>= 16 consecutive offsets per CTA), the
// last one of up to 12 stages on contiguous blocks
int plan_passes(int L, int *s0, int *kk) {
  int np = 0;
  const int last = L < 12 ? L : 12;
  int rest = L - last, s = 0;
  while (rest > 0) {
    const int k = rest < 8 ? rest : 8;
    s0[np] = s;
    kk[np] = k;
    np++;
    s += k;
    rest -= k;
  }
  s0[np] = s;
  kk[np] = last;
  np++;
  return np;
}
}  // namespace

int ntt_init_tables() { return init_tables(nullptr); }

size_t ntt_workspace_bytes(int log_n, int nprod) {
  return ((size_t)4 * nprod << log_n) * sizeof(uint32_t);
}

namespace {
// The transform products of one launch sequence: nprod sub-products of one
// transform length 2^log_n (all squarings or none), their arrays at scratch.
template <class Prods>
cudaError_t launch_ntt_core(const Prods &prods, int nprod, int64_t max_ncols, int square,
                            int log_n, void *scratch, cudaStream_t s) {
  const int tr = init_tables(s);
  if (tr == -2) return cudaErrorStreamCaptureUnsupported;
  if (tr != 0) return cudaErrorInitializationError;
  const int64_t n = (int64_t)1 << log_n;
  uint32_t *data = static_cast<uint32_t *>(scratch);
  const PrimeC pc0 = prime_c(0), pc1 = prime_c(1);

  LoadArgs<Prods> la{};
  la.prods = prods;
  la.square = square;
  la.data = data;
  la.L = log_n;
  la.nprod = nprod;
  la.pc[0] = pc0;
  la.pc[1] = pc1;
  int64_t tot = n * 4 * nprod;
  int64_t blocks = (tot + 255) / 256;
  if (blocks > 152 * 32) blocks = 152 * 32;
  (void)launch_k(ntt_load<Prods>, dim3((unsigned)blocks), dim3(256), 0, s, la);

  int s0[8], kk[8];
  const int np = plan_passes(log_n, s0, kk);
  NttArgs g{};
  g.data = data;
  g.L = log_n;
  g.pc[0] = pc0;
  g.pc[1] = pc1;
  for (int i = 0; i < np; i++) {  // forward: all 4 * nprod arrays (squaring: the first sides)
    g.s0 = s0[i];
    g.k = kk[i];
    g.astride = square ? 2 : 1;
    g.aoff = 0;
    const int64_t F = n >> (s0[i] + kk[i]);
    const int64_t Wc = F < (kTile >> kk[i]) ? F : (kTile >> kk[i]);
    const int64_t ctas = ((int64_t)1 << s0[i]) * (F / Wc);
    (void)launch_k(ntt_pass<true>, dim3((unsigned)ctas, (unsigned)((square ? 2 : 4) * nprod)),
                   dim3(kPassThreads), 0, s, g);
  }
  tot = n * 2 * nprod;
  blocks = (tot + 255) / 256;
  if (blocks > 152 * 32) blocks = 152 * 32;
  (void)launch_k(ntt_pointwise, dim3((unsigned)blocks), dim3(256), 0, s, data, log_n, nprod, pc0,
                 pc1, square);
  for (int i = np - 1; i >= 0; i--) {  // inverse: the product arrays (side 0)
    g.s0 = s0[i];
    g.k = kk[i];
    g.astride = 2;
    g.aoff = 0;
    const int64_t F = n >> (s0[i] + kk[i]);
    const int64_t Wc = F < (kTile >> kk[i]) ? F : (kTile >> kk[i]);
    const int64_t ctas = ((int64_t)1 << s0[i]) * (F / Wc);
    (void)launch_k(ntt_pass<false>, dim3((unsigned)ctas, (unsigned)(2 * nprod)),
                   dim3(kPassThreads), 0, s, g);
  }
  CrtArgs<Prods> c{};
  c.prods = prods;
  c.data = data;
  c.L = log_n;
  c.nprod = nprod;
  c.pc[0] = pc0;
  c.pc[1] = pc1;
  for (int r = 0; r < 2; r++) {
    const uint64_t p = kP[r];
    const uint64_t ninv = powmod((uint64_t)n % p, p - 2, p);
    // K = n^-1 R^2 mod p
    const uint64_t R2 = (uint64_t)(((unsigned __int128)1 << 64) % p);
    c.K[r] = (uint32_t)((unsigned __int128)ninv * R2 % p);
  }
  const uint64_t p1inv = powmod(kP[0] % kP[1], kP[1] - 2, kP[1]);
  c.M = to_mont(p1inv, kP[1]);
  blocks = (max_ncols + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  if (blocks < 1) blocks = 1;
  (void)launch_k(ntt_crt<Prods>, dim3((unsigned)blocks, (unsigned)nprod), dim3(256), 0, s, c);
  note_launches(3 + 2 * np);
  return cudaGetLastError();
}
}  // namespace

cudaError_t launch_ntt_products(const Product *prods, int nprod, int log_n, int d, void *scratch,
                                cudaStream_t s) {
  (void)d;
  if (log_n > kMaxLog || nprod < 1 || nprod > 4) return cudaErrorInvalidValue;
  if (log_n < 1) log_n = 1;
  InlineProds ip{};
  for (int q = 0; q < nprod; q++) ip.p[q] = prods[q];
  // squaring: both operands are the same digits
  const int square = (prods[0].A == prods[0].B && prods[0].nA == prods[0].nB) ? 1 : 0;
  return launch_ntt_core(ip, nprod, prods[0].nA + prods[0].nB - 1, square, log_n, scratch, s);
}

cudaError_t launch_ntt_batch(const Product *dprods, int nprod, int64_t max_ncols, int square,
                             int log_n, void *scratch, cudaStream_t s) {
  if (log_n > kMaxLog || nprod < 1 || nprod > kMaxNttBatch) return cudaErrorInvalidValue;
  if (log_n < 1) log_n = 1;
  return launch_ntt_core(DeviceProds{dprods}, nprod, max_ncols, square, log_n, scratch, s);
}

}  // namespace ks
