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
// permutation pass exists.  A pass loads 4096 elements of one transform into
// shared memory and runs up to 12 radix-2 stages there: the last pass takes
// contiguous blocks, earlier passes take 2^k strided elements for 4096 / 2^k
// consecutive offsets (coalesced).  Twiddles w^e come from two tables per
// prime and direction, w^e = T1[e mod 2^13] * T2[e >> 13].
#include <mutex>

#include "ks_internal.cuh"

namespace ks {

namespace {
constexpr int kMaxLog = 27;
constexpr int kT1 = 1 << 13;
constexpr int kT2 = 1 << 14;
constexpr int kTile = 4096;
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

template <bool kForward>
__global__ void __launch_bounds__(kPassThreads) ntt_pass(NttArgs g) {
  __shared__ uint32_t S[kTile];
  const int a = blockIdx.y * g.astride + g.aoff;
  const int r = prime_of(a);
  const uint32_t p = g.pc[r].p, pinv = g.pc[r].pinv;
  const int64_t n = (int64_t)1 << g.L;
  uint32_t *X = g.data + (int64_t)a * n;
  const int k = g.k;
  const int64_t F = n >> (g.s0 + k);        // finest block width of this pass
  const int Wc = (int)(F < (kTile >> k) ? F : (kTile >> k));  // consecutive offsets per CTA
  const int V = 1 << k;
  const int64_t wblocks = F / Wc;
  const int64_t u = blockIdx.x / wblocks;
  const int64_t w0 = (blockIdx.x % wblocks) * Wc;
  const int64_t ubase = u * (n >> g.s0);
  const int tot = V * Wc;
  for (int i = threadIdx.x; i < tot; i += kPassThreads) {
    const int v = i / Wc, wi = i % Wc;
    S[v * Wc + wi] = X[ubase + v * F + w0 + wi];
  }
  __syncthreads();
  const int shift = kMaxLog - g.L;  // exponents in units of the order-2^27 root
  for (int rr = 0; rr < k; rr++) {
    const int r_st = kForward ? rr : (k - 1 - rr);  // stage within the pass
    const int s = g.s0 + r_st;
    const int h = 1 << (k - 1 - r_st);
    for (int b = threadIdx.x; b < tot / 2; b += kPassThreads) {
      const int wi = b % Wc, vp = b / Wc;
      const int vlo = ((vp >> (k - 1 - r_st)) << (k - r_st)) | (vp & (h - 1));
      const int ilo = vlo * Wc + wi, ihi = (vlo + h) * Wc + wi;
      const uint32_t j = (uint32_t)((vlo & (h - 1)) * F + w0 + wi);
      const uint32_t e = (j << s) << shift;
      const uint32_t tw = twiddle(r, kForward ? 0 : 1, e, p, pinv);
      const uint32_t x = S[ilo], y = S[ihi];
      if (kForward) {
        S[ilo] = add_mod(x, y, p);
        S[ihi] = mont_mul(sub_mod(x, y, p), tw, p, pinv);
      } else {
        const uint32_t yt = mont_mul(y, tw, p, pinv);
        S[ilo] = add_mod(x, yt, p);
        S[ihi] = sub_mod(x, yt, p);
      }
    }
    __syncthreads();
  }
  for (int i = threadIdx.x; i < tot; i += kPassThreads) {
    const int v = i / Wc, wi = i % Wc;
    X[ubase + v * F + w0 + wi] = S[v * Wc + wi];
  }
}

struct LoadArgs {
  const int32_t *A[4];
  const int32_t *B[4];
  int64_t nA, nB;
  uint32_t *data;
  int L;
  int nprod;
  PrimeC pc[2];
};

__global__ void __launch_bounds__(256) ntt_load(LoadArgs g) {
  const int64_t n = (int64_t)1 << g.L;
  const int64_t total = n * 4 * g.nprod;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int a = (int)(idx >> g.L);
    const int64_t i = idx & (n - 1);
    const int q = a >> 2, r = (a >> 1) & 1, side = a & 1;
    const uint32_t p = g.pc[r].p;
    int32_t d = 0;
    if (side == 0) {
      if (i < g.nA) d = g.A[q][i];
    } else {
      if (i < g.nB) d = g.B[q][i];
    }
    g.data[idx] = d >= 0 ? (uint32_t)d : (uint32_t)((int64_t)d + p);
  }
}

__global__ void __launch_bounds__(256) ntt_pointwise(uint32_t *data, int L, int nprod, PrimeC p0,
                                                     PrimeC p1) {
  const int64_t n = (int64_t)1 << L;
  const int64_t total = n * 2 * nprod;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int qr = (int)(idx >> L);  // product * 2 + prime
    const int64_t i = idx & (n - 1);
    const PrimeC pc = (qr & 1) ? p1 : p0;
    uint32_t *X = data + (int64_t)(2 * qr) * n;
    X[i] = mont_mul(X[i], X[n + i], pc.p, pc.pinv);
  }
}

struct CrtArgs {
  const uint32_t *data;
  int L;
  int nprod;
  int64_t *C[4];
  int64_t ncols;
  PrimeC pc[2];
  uint32_t K[2];      // n^-1 R^2 mod p (Montgomery scale after the inverse transform)
  uint32_t M;         // p1^-1 R mod p2
};

__global__ void __launch_bounds__(256) ntt_crt(CrtArgs g) {
  const int64_t n = (int64_t)1 << g.L;
  const int64_t total = g.ncols * g.nprod;
  const uint64_t P = (uint64_t)g.pc[0].p * g.pc[1].p;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int q = (int)(idx / g.ncols);
    const int64_t k = idx - q * g.ncols;
    const uint32_t z1 = g.data[(int64_t)(4 * q + 0) * n + k];
    const uint32_t z2 = g.data[(int64_t)(4 * q + 2) * n + k];
    const uint32_t c1 = mont_mul(z1, g.K[0], g.pc[0].p, g.pc[0].pinv);
    const uint32_t c2 = mont_mul(z2, g.K[1], g.pc[1].p, g.pc[1].pinv);
    const uint32_t d = sub_mod(c2, c1, g.pc[1].p);  // c1 < p1 < p2
    const uint32_t t = mont_mul(d, g.M, g.pc[1].p, g.pc[1].pinv);
    const uint64_t x = (uint64_t)c1 + (uint64_t)g.pc[0].p * t;  // in [0, P)
    const int64_t v = x > P / 2 ? (int64_t)(x - P) : (int64_t)x;
    g.C[q][k] = v;
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

int init_tables() {
  static std::mutex mu;
  static bool done[64] = {false};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return -1;
  std::lock_guard<std::mutex> lk(mu);
  if (done[dev]) return 0;
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

size_t ntt_workspace_bytes(int log_n, int nprod) {
  return ((size_t)4 * nprod << log_n) * sizeof(uint32_t);
}

cudaError_t launch_ntt_products(const Product *prods, int nprod, int log_n, int d, void *scratch,
                                cudaStream_t s) {
  (void)d;
  if (log_n > kMaxLog || nprod < 1 || nprod > 4) return cudaErrorInvalidValue;
  if (log_n < 1) log_n = 1;
  if (init_tables() != 0) return cudaErrorInitializationError;
  const int64_t n = (int64_t)1 << log_n;
  uint32_t *data = static_cast<uint32_t *>(scratch);
  const PrimeC pc0 = prime_c(0), pc1 = prime_c(1);

  LoadArgs la{};
  for (int q = 0; q < nprod; q++) {
    la.A[q] = prods[q].A;
    la.B[q] = prods[q].B;
  }
  la.nA = prods[0].nA;
  la.nB = prods[0].nB;
  la.data = data;
  la.L = log_n;
  la.nprod = nprod;
  la.pc[0] = pc0;
  la.pc[1] = pc1;
  int64_t tot = n * 4 * nprod;
  int64_t blocks = (tot + 255) / 256;
  if (blocks > 152 * 32) blocks = 152 * 32;
  ntt_load<<<(unsigned)blocks, 256, 0, s>>>(la);

  int s0[8], kk[8];
  const int np = plan_passes(log_n, s0, kk);
  NttArgs g{};
  g.data = data;
  g.L = log_n;
  g.pc[0] = pc0;
  g.pc[1] = pc1;
  for (int i = 0; i < np; i++) {  // forward: all 4 * nprod arrays
    g.s0 = s0[i];
    g.k = kk[i];
    g.astride = 1;
    g.aoff = 0;
    const int64_t F = n >> (s0[i] + kk[i]);
    const int64_t Wc = F < (kTile >> kk[i]) ? F : (kTile >> kk[i]);
    const int64_t ctas = ((int64_t)1 << s0[i]) * (F / Wc);
    ntt_pass<true><<<dim3((unsigned)ctas, (unsigned)(4 * nprod)), kPassThreads, 0, s>>>(g);
  }
  tot = n * 2 * nprod;
  blocks = (tot + 255) / 256;
  if (blocks > 152 * 32) blocks = 152 * 32;
  ntt_pointwise<<<(unsigned)blocks, 256, 0, s>>>(data, log_n, nprod, pc0, pc1);
  for (int i = np - 1; i >= 0; i--) {  // inverse: the product arrays (side 0)
    g.s0 = s0[i];
    g.k = kk[i];
    g.astride = 2;
    g.aoff = 0;
    const int64_t F = n >> (s0[i] + kk[i]);
    const int64_t Wc = F < (kTile >> kk[i]) ? F : (kTile >> kk[i]);
    const int64_t ctas = ((int64_t)1 << s0[i]) * (F / Wc);
    ntt_pass<false><<<dim3((unsigned)ctas, (unsigned)(2 * nprod)), kPassThreads, 0, s>>>(g);
  }
  CrtArgs c{};
  c.data = data;
  c.L = log_n;
  c.nprod = nprod;
  for (int q = 0; q < nprod; q++) c.C[q] = prods[q].C;
  c.ncols = prods[0].nA + prods[0].nB - 1;
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
  tot = c.ncols * nprod;
  blocks = (tot + 255) / 256;
  if (blocks > 152 * 32) blocks = 152 * 32;
  ntt_crt<<<(unsigned)blocks, 256, 0, s>>>(c);
  note_launches(3 + 2 * np);
  return cudaGetLastError();
}

}  // namespace ks
