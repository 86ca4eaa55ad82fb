// Autotuning support: time one (variant, engine) configuration of the
// library on synthetic inputs, for one product or a batched plan of `batch`
// equal-shaped products.  The tuner (the Python driver in the package) sweeps
// problem shapes with it and builds the dispatch table and the training set
// of the cost model.  (No counterpart in the paper, which picks variants per
// experiment, Sec. 4.)
#include <vector>

#include "ks_internal.cuh"

namespace ks {

// coefficients of `bits` bits from a counter-based mix of (seed, index)
__global__ void fill_random(uint64_t *x, int64_t L, int limbs, int bits, int is_signed,
                            uint64_t seed) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= L * limbs) return;
  uint64_t z = seed + (uint64_t)(i + 1) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z ^= z >> 31;
  const int l = (int)(i % limbs);
  const int top = bits - 64 * (limbs - 1);
  if (l == limbs - 1 && top < 64) {
    z &= (1ull << top) - 1ull;
    if (is_signed && ((z >> (top - 1)) & 1ull)) z |= ~((1ull << top) - 1ull);
  }
  x[i] = z;
}

}  // namespace ks

using namespace ks;

extern "C" int ks_tune_time(int64_t len_f, int64_t len_g, int coeff_bits, int is_signed,
                            int variant, int engine, int batch, int reps, double *ms_per_product) {
  if (!ms_per_product || batch < 1 || reps < 1 || variant < KS_1 || variant > KS_4 ||
      engine < 1 || engine > 3)
    return KS_EINVAL;
  Plan p;
  int rc = make_plan(p, len_f, len_g, coeff_bits, is_signed, variant, engine);
  if (rc != KS_OK) return rc;
  const int il = p.in_limbs, ol = p.out_limbs;
  const size_t fb = (size_t)len_f * il * 8, gb = (size_t)len_g * il * 8,
               hb = (size_t)p.lh * ol * 8;
  char *buf = nullptr;
  const size_t per = ((fb + 255) & ~(size_t)255) + ((gb + 255) & ~(size_t)255) +
                     ((hb + 255) & ~(size_t)255);
  if (cudaMalloc(&buf, per * batch + 256) != cudaSuccess) return KS_ENOMEM;
  std::vector<ks_problem> probs(batch);
  for (int i = 0; i < batch; i++) {
    char *b0 = buf + per * i;
    uint64_t *f = reinterpret_cast<uint64_t *>(b0);
    uint64_t *g = reinterpret_cast<uint64_t *>(b0 + ((fb + 255) & ~(size_t)255));
    uint64_t *h = reinterpret_cast<uint64_t *>(b0 + ((fb + 255) & ~(size_t)255) +
                                               ((gb + 255) & ~(size_t)255));
    fill_random<<<(unsigned)((len_f * il + 255) / 256), 256>>>(f, len_f, il, coeff_bits,
                                                                is_signed, 17 + 2 * i);
    fill_random<<<(unsigned)((len_g * il + 255) / 256), 256>>>(g, len_g, il, coeff_bits,
                                                                is_signed, 18 + 2 * i);
    probs[i] = ks_problem{h, f, g, len_f, len_g, coeff_bits, is_signed, variant, engine};
  }
  cudaStream_t s = nullptr;
  if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
    cudaFree(buf);
    return KS_ECUDA;
  }
  ks_plan *plan = nullptr;
  rc = ks_plan_create(&plan, probs.data(), batch, KS_DISPATCH_AUTO);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (rc == KS_OK) {
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    for (int w = 0; w < 2 && rc == KS_OK; w++) rc = ks_plan_execute(plan, s);
    if (rc == KS_OK) {
      cudaEventRecord(e0, s);
      for (int r = 0; r < reps && rc == KS_OK; r++) rc = ks_plan_execute(plan, s);
      cudaEventRecord(e1, s);
    }
    if (cudaStreamSynchronize(s) != cudaSuccess) rc = KS_ECUDA;
    float ms = 0.f;
    if (rc == KS_OK && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess)
      *ms_per_product = (double)ms / reps / batch;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
  }
  ks_plan_destroy(plan);
  cudaStreamDestroy(s);
  cudaFree(buf);
  if (rc == KS_OK) rc = ks_status_sync(nullptr);
  return rc;
}
