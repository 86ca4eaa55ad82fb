// Learned dispatch: a small MLP cost model, trained and evaluated by the
// library's own CUDA kernels, and the autotuned dispatch table it falls back
// to.  (The paper chooses variants by hand per experiment, Sec. 4, and notes
// that small degrees favour the standard substitution; nothing here affects
// correctness -- every choice is an exact path.)
//
// Model: features x (5) -> 32 ReLU -> 32 ReLU -> 12 outputs, the predicted
// log2 of the time per product (microseconds) of each (variant, engine):
// output j = 3 (variant - 1) + e, e = 0 INT32 schoolbook, 1 NTT, 2 tensor
// cores.  Features: log2 len_f / 20, log2 len_g / 20, log2 bits / 11, signed,
// log2 batch / 12.  Loss: masked mean squared error over measured outputs.
// Training: full-batch Adam, every step on the GPU (forward, loss gradient,
// backward, update kernels below).  Parameters are one float array:
// W1 [32 x 5], b1 [32], W2 [32 x 32], b2 [32], W3 [12 x 32], b3 [12].
#include <math.h>
#include <mutex>
#include <string.h>
#include <vector>

#include "ks_internal.cuh"

namespace ks {

namespace {
constexpr int IN = KS_MLP_IN, H = KS_MLP_HIDDEN, OUT = KS_MLP_OUT;
constexpr int64_t NPARAM = (int64_t)H * IN + H + H * H + H + (int64_t)OUT * H + OUT;
constexpr double kBatchBitsSat = 26.0;  // log2 of the operand bits that fill the GPU
struct Layout {
  int64_t w1 = 0, b1 = w1 + H * IN, w2 = b1 + H, b2 = w2 + H * H, w3 = b2 + H,
          b3 = w3 + OUT * H;
};

__global__ void dense_forward(const float *W, const float *b, const float *X, float *Y, int64_t n,
                              int din, int dout, int relu) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n * dout) return;
  const int64_t s = idx / dout;
  const int o = (int)(idx - s * dout);
  float acc = b[o];
  for (int i = 0; i < din; i++) acc += W[o * din + i] * X[s * din + i];
  Y[idx] = relu ? fmaxf(acc, 0.f) : acc;
}

// dY = 2 m (Y - T) / sum(m)
__global__ void loss_grad(const float *Y, const float *T, const float *M, float *dY, int64_t n,
                          float inv_count) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n * OUT) return;
  dY[idx] = 2.f * M[idx] * (Y[idx] - T[idx]) * inv_count;
}

// dX[s, i] = sum_o dOut[s, o] W[o, i], masked by the ReLU of X when relu_in
__global__ void dense_backward_input(const float *W, const float *dOut, const float *X, float *dX,
                                     int64_t n, int din, int dout, int relu_in) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n * din) return;
  const int64_t s = idx / din;
  const int i = (int)(idx - s * din);
  float acc = 0.f;
  for (int o = 0; o < dout; o++) acc += dOut[s * dout + o] * W[o * din + i];
  dX[idx] = (relu_in && X[idx] <= 0.f) ? 0.f : acc;
}

// dW[o, i] = sum_s dOut[s, o] X[s, i]; db[o] = sum_s dOut[s, o] (fixed order: deterministic)
__global__ void dense_backward_weight(const float *dOut, const float *X, float *dW, float *db,
                                      int64_t n, int din, int dout) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx < dout * din) {
    const int o = idx / din, i = idx - (idx / din) * din;
    float acc = 0.f;
    for (int64_t s = 0; s < n; s++) acc += dOut[s * dout + o] * X[s * din + i];
    dW[idx] = acc;
  } else if (idx < dout * din + dout) {
    const int o = idx - dout * din;
    float acc = 0.f;
    for (int64_t s = 0; s < n; s++) acc += dOut[s * dout + o];
    db[o] = acc;
  }
}

__global__ void loss_value(const float *Y, const float *T, const float *M, int64_t n,
                           float inv_count, float *out) {
  __shared__ float part[256];
  float acc = 0.f;
  for (int64_t idx = threadIdx.x; idx < n * OUT; idx += 256) {
    const float d = Y[idx] - T[idx];
    acc += M[idx] * d * d;
  }
  part[threadIdx.x] = acc;
  __syncthreads();
  for (int off = 128; off > 0; off >>= 1) {
    if (threadIdx.x < off) part[threadIdx.x] += part[threadIdx.x + off];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = part[0] * inv_count;
}

__global__ void adam_update(float *P, const float *G, float *m, float *v, int64_t np, float lr,
                            float c1, float c2) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= np) return;
  const float g = G[i];
  m[i] = 0.9f * m[i] + 0.1f * g;
  v[i] = 0.999f * v[i] + 0.001f * g * g;
  const float mh = m[i] / c1, vh = v[i] / c2;
  P[i] -= lr * mh / (sqrtf(vh) + 1e-8f);
}

unsigned nb(int64_t n) { return (unsigned)((n + 255) / 256); }

struct Buffers {
  float *P, *G, *m, *v, *X, *T, *M, *h1, *h2, *y, *d3, *d2, *d1, *dx, *loss;
};

// forward pass for n samples; activations into the buffers
void forward(const Buffers &B, int64_t n, cudaStream_t s) {
  Layout L;
  dense_forward<<<nb(n * H), 256, 0, s>>>(B.P + L.w1, B.P + L.b1, B.X, B.h1, n, IN, H, 1);
  dense_forward<<<nb(n * H), 256, 0, s>>>(B.P + L.w2, B.P + L.b2, B.h1, B.h2, n, H, H, 1);
  dense_forward<<<nb(n * OUT), 256, 0, s>>>(B.P + L.w3, B.P + L.b3, B.h2, B.y, n, H, OUT, 0);
}

void backward(const Buffers &B, int64_t n, float inv_count, cudaStream_t s) {
  Layout L;
  loss_grad<<<nb(n * OUT), 256, 0, s>>>(B.y, B.T, B.M, B.d3, n, inv_count);
  dense_backward_weight<<<nb(OUT * H + OUT), 256, 0, s>>>(B.d3, B.h2, B.G + L.w3, B.G + L.b3, n,
                                                          H, OUT);
  dense_backward_input<<<nb(n * H), 256, 0, s>>>(B.P + L.w3, B.d3, B.h2, B.d2, n, H, OUT, 1);
  dense_backward_weight<<<nb(H * H + H), 256, 0, s>>>(B.d2, B.h1, B.G + L.w2, B.G + L.b2, n, H,
                                                      H);
  dense_backward_input<<<nb(n * H), 256, 0, s>>>(B.P + L.w2, B.d2, B.h1, B.d1, n, H, H, 1);
  dense_backward_weight<<<nb(H * IN + H), 256, 0, s>>>(B.d1, B.X, B.G + L.w1, B.G + L.b1, n, IN,
                                                       H);
}

float inv_mask_count(const float *mask, int64_t n) {
  double c = 0;
  for (int64_t i = 0; i < n * OUT; i++) c += mask[i];
  return c > 0 ? (float)(1.0 / c) : 0.f;
}

// device buffers for n samples (freed by free_buffers)
int alloc_buffers(Buffers &B, int64_t n) {
  memset(&B, 0, sizeof(B));
  // per sample: X, dx (IN); T, M, y, d3 (OUT); h1, h2, d2, d1 (H)
  const size_t total = (size_t)(4 * NPARAM + n * (2 * IN + 4 * OUT + 4 * H) + 1);
  float *base = nullptr;
  if (cudaMalloc(&base, total * sizeof(float)) != cudaSuccess) return KS_ENOMEM;
  cudaMemset(base, 0, total * sizeof(float));
  float *p = base;
  auto take = [&](int64_t k) {
    float *r = p;
    p += k;
    return r;
  };
  B.P = take(NPARAM);
  B.G = take(NPARAM);
  B.m = take(NPARAM);
  B.v = take(NPARAM);
  B.X = take(n * IN);
  B.T = take(n * OUT);
  B.M = take(n * OUT);
  B.h1 = take(n * H);
  B.h2 = take(n * H);
  B.y = take(n * OUT);
  B.d3 = take(n * OUT);
  B.d2 = take(n * H);
  B.d1 = take(n * H);
  B.dx = take(n * IN);
  B.loss = take(1);
  return KS_OK;
}
void free_buffers(Buffers &B) {
  if (B.P) cudaFree(B.P);
  memset(&B, 0, sizeof(B));
}

// ---- installed dispatch state (per process)
std::mutex g_mu;
bool g_have_mlp = false;
float g_params[NPARAM];
struct TableEntry {
  int32_t lf, lg, bits, sgn, variant, engine;
};
std::vector<TableEntry> g_table;
}  // namespace

// Features of one product: its lengths and size, its sign, and the operand
// bits of the whole batch it runs in (sum of (Lf + Lg) b over the batch),
// log-scaled and saturating at 2^26: beyond that the batch fills the GPU and
// a product's cost is its share of the work, not its latency.
void mlp_features(int64_t lf, int64_t lg, int b, int is_signed, double batch_bits, float *x) {
  x[0] = (float)(log2((double)lf) / 20.0);
  x[1] = (float)(log2((double)lg) / 20.0);
  x[2] = (float)(log2((double)b) / 11.0);
  x[3] = is_signed ? 1.f : 0.f;
  const double w = log2(batch_bits < 1.0 ? 1.0 : batch_bits);
  x[4] = (float)((w < kBatchBitsSat ? w : kBatchBitsSat) / kBatchBitsSat);
}

bool mlp_installed() {
  std::lock_guard<std::mutex> lk(g_mu);
  return g_have_mlp;
}

// GPU inference for n feature rows (host in, host out): one forward launch set
int mlp_predict_host(const float *x, int64_t n, float *y) {
  float params[NPARAM];
  {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_have_mlp) return KS_EINVAL;
    memcpy(params, g_params, sizeof(params));
  }
  Buffers B;
  int rc = alloc_buffers(B, n);
  if (rc != KS_OK) return rc;
  cudaMemcpy(B.P, params, sizeof(params), cudaMemcpyHostToDevice);
  cudaMemcpy(B.X, x, n * IN * sizeof(float), cudaMemcpyHostToDevice);
  forward(B, n, nullptr);
  note_launches(3);
  cudaError_t e = cudaMemcpy(y, B.y, n * OUT * sizeof(float), cudaMemcpyDeviceToHost);
  free_buffers(B);
  return e == cudaSuccess ? KS_OK : KS_ECUDA;
}

// the nearest measured bucket of the table (log-space distance)
bool table_lookup(int64_t lf, int64_t lg, int b, int is_signed, int *variant, int *engine) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (g_table.empty()) return false;
  const double x0 = log2((double)lf), x1 = log2((double)lg), x2 = log2((double)b);
  double best = 1e300;
  const TableEntry *pick = nullptr;
  for (const auto &t : g_table) {
    if (t.sgn != (is_signed ? 1 : 0)) continue;
    const double d0 = log2((double)t.lf) - x0, d1 = log2((double)t.lg) - x1,
                 d2 = log2((double)t.bits) - x2;
    const double d = d0 * d0 + d1 * d1 + 2.0 * d2 * d2;
    if (d < best) {
      best = d;
      pick = &t;
    }
  }
  if (pick == nullptr) return false;
  *variant = pick->variant;
  *engine = pick->engine;
  return true;
}

}  // namespace ks

using namespace ks;

extern "C" {

int64_t ks_mlp_param_count(void) { return NPARAM; }

int ks_mlp_set_params(const float *params) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (params == nullptr) {
    g_have_mlp = false;
    return KS_OK;
  }
  for (int64_t i = 0; i < NPARAM; i++)
    if (!isfinite(params[i])) return KS_EINVAL;
  memcpy(g_params, params, sizeof(g_params));
  g_have_mlp = true;
  return KS_OK;
}

int ks_dispatch_set_table(int64_t n, const int32_t *rows) {
  if (n < 0 || (n > 0 && rows == nullptr)) return KS_EINVAL;
  std::vector<TableEntry> t;
  for (int64_t i = 0; i < n; i++) {
    const int32_t *r = rows + 6 * i;
    if (r[0] < 1 || r[1] < 1 || r[2] < 1 || r[4] < KS_1 || r[4] > KS_4 || r[5] < 1 || r[5] > 3)
      return KS_EINVAL;
    t.push_back(TableEntry{r[0], r[1], r[2], r[3] ? 1 : 0, r[4], r[5]});
  }
  std::lock_guard<std::mutex> lk(g_mu);
  g_table.swap(t);
  return KS_OK;
}

int ks_mlp_predict(const float *x, int64_t n, float *y) {
  if (n < 1 || !x || !y) return KS_EINVAL;
  return mlp_predict_host(x, n, y);
}

// One forward + backward pass on the GPU; gradient (NPARAM floats) and loss to the host.
int ks_mlp_grad(const float *params, const float *x, const float *t, const float *mask, int64_t n,
                float *grad, float *loss) {
  if (n < 1 || !params || !x || !t || !mask || !grad) return KS_EINVAL;
  Buffers B;
  int rc = alloc_buffers(B, n);
  if (rc != KS_OK) return rc;
  const float inv = inv_mask_count(mask, n);
  cudaMemcpy(B.P, params, NPARAM * sizeof(float), cudaMemcpyHostToDevice);
  cudaMemcpy(B.X, x, n * IN * sizeof(float), cudaMemcpyHostToDevice);
  cudaMemcpy(B.T, t, n * OUT * sizeof(float), cudaMemcpyHostToDevice);
  cudaMemcpy(B.M, mask, n * OUT * sizeof(float), cudaMemcpyHostToDevice);
  forward(B, n, nullptr);
  backward(B, n, inv, nullptr);
  loss_value<<<1, 256>>>(B.y, B.T, B.M, n, inv, B.loss);
  note_launches(10);
  cudaError_t e = cudaMemcpy(grad, B.G, NPARAM * sizeof(float), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && loss) e = cudaMemcpy(loss, B.loss, sizeof(float), cudaMemcpyDeviceToHost);
  free_buffers(B);
  return e == cudaSuccess ? KS_OK : KS_ECUDA;
}

// Full-batch Adam for `steps` steps on the GPU; params updated in place (host).
int ks_mlp_train(float *params, const float *x, const float *t, const float *mask, int64_t n,
                 int steps, float lr, float *loss_out) {
  if (n < 1 || steps < 0 || !params || !x || !t || !mask) return KS_EINVAL;
  Buffers B;
  int rc = alloc_buffers(B, n);
  if (rc != KS_OK) return rc;
  const float inv = inv_mask_count(mask, n);
  cudaMemcpy(B.P, params, NPARAM * sizeof(float), cudaMemcpyHostToDevice);
  cudaMemcpy(B.X, x, n * IN * sizeof(float), cudaMemcpyHostToDevice);
  cudaMemcpy(B.T, t, n * OUT * sizeof(float), cudaMemcpyHostToDevice);
  cudaMemcpy(B.M, mask, n * OUT * sizeof(float), cudaMemcpyHostToDevice);
  double c1 = 1.0, c2 = 1.0;
  for (int step = 0; step < steps; step++) {
    forward(B, n, nullptr);
    backward(B, n, inv, nullptr);
    c1 *= 0.9;
    c2 *= 0.999;
    const float lr_t = (float)(lr * (step < steps / 2 ? 1.0 : 0.3));
    adam_update<<<nb(NPARAM), 256>>>(B.P, B.G, B.m, B.v, NPARAM, lr_t, (float)(1.0 - c1),
                                     (float)(1.0 - c2));
  }
  forward(B, n, nullptr);
  loss_value<<<1, 256>>>(B.y, B.T, B.M, n, inv, B.loss);
  note_launches(10 * steps + 4);
  cudaError_t e = cudaMemcpy(params, B.P, NPARAM * sizeof(float), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && loss_out)
    e = cudaMemcpy(loss_out, B.loss, sizeof(float), cudaMemcpyDeviceToHost);
  free_buffers(B);
  return e == cudaSuccess ? KS_OK : KS_ECUDA;
}

}  // extern "C"
