/*
 * CPU oracle for products in Z[x] -- TEST INFRASTRUCTURE ONLY.
 *
 * Only the tests, the smoke check and the benchmark's CPU-baseline leg may
 * load this library.  The product path never calls it and shares no code
 * with it.
 *
 * What it computes is the plain definition of the product (Harvey, Sec. 3,
 * the product h = f g of two polynomials in Z[x]):
 *
 *     h_k = sum_{i + j = k} f_i g_j ,      0 <= k < Lf + Lg - 1,
 *
 * as an exact integer, by the schoolbook double loop over multi-limb
 * integers, one coefficient at a time.  No blocking, no reordering, no
 * substitution.  The modular entry point follows the paper's application
 * (Sec. 4): h_k mod p for residues in [0, p).  The bivariate entry point is
 * the plain product in (Z/pZ)[x, y], the setting of Sec. 2.
 *
 * Encoding: coefficient i of f is fl = ceil(b/64) little-endian uint64 limbs;
 * signed values are two's complement sign-extended over the limbs.  Each
 * output coefficient is written as out_limbs limbs of two's complement (the
 * caller chooses out_limbs wide enough for the exact value; the accumulator
 * is wider and wraps, so the low out_limbs limbs are exact whenever the value
 * fits).
 */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef unsigned __int128 u128;

#define MAX_LIMBS 64 /* 4096-bit coefficients at most */

/* |x| of a two's complement n-limb integer into mag; returns 1 if x < 0. */
static int magnitude(uint64_t *mag, const uint64_t *x, int n, int is_signed) {
  int neg = is_signed && (x[n - 1] >> 63);
  if (!neg) {
    memcpy(mag, x, (size_t)n * 8);
    return 0;
  }
  uint64_t carry = 1;
  for (int l = 0; l < n; l++) {
    uint64_t v = ~x[l] + carry;
    carry = (carry && v == 0) ? 1 : 0;
    mag[l] = v;
  }
  return 1;
}

/* acc (w limbs, wrapping) += sign * a * b, with a and b n-limb magnitudes. */
static void acc_product(uint64_t *acc, int w, const uint64_t *a,
                        const uint64_t *b, int n, int negative) {
  uint64_t prod[2 * MAX_LIMBS];
  memset(prod, 0, sizeof(uint64_t) * 2 * n);
  for (int i = 0; i < n; i++) {
    uint64_t carry = 0;
    for (int j = 0; j < n; j++) {
      u128 t = (u128)a[i] * b[j] + prod[i + j] + carry;
      prod[i + j] = (uint64_t)t;
      carry = (uint64_t)(t >> 64);
    }
    prod[i + n] = carry;
  }
  if (!negative) {
    uint64_t carry = 0;
    for (int l = 0; l < w; l++) {
      uint64_t p = l < 2 * n ? prod[l] : 0;
      u128 t = (u128)acc[l] + p + carry;
      acc[l] = (uint64_t)t;
      carry = (uint64_t)(t >> 64);
    }
  } else {
    uint64_t borrow = 0;
    for (int l = 0; l < w; l++) {
      uint64_t p = l < 2 * n ? prod[l] : 0;
      u128 t = (u128)acc[l] - p - borrow;
      acc[l] = (uint64_t)t;
      borrow = (uint64_t)(t >> 64) ? 1 : 0;
    }
  }
}

typedef struct {
  uint64_t *h;
  const uint64_t *f, *g;
  int64_t lf, lg;
  int limbs, is_signed, out_limbs;
  const int64_t *ks; /* NULL: all coefficients 0..Lh-1 */
  int64_t nk;
  int64_t begin, stride; /* this worker owns begin, begin+stride, ... < nk */
} job_t;

/* h_k = sum_{i+j=k} f_i g_j, written as out_limbs two's complement limbs. */
static void one_coeff(uint64_t *out, const job_t *J, int64_t k) {
  const int n = J->limbs;
  int w = 2 * n + 2;
  if (w < J->out_limbs) w = J->out_limbs;
  uint64_t acc[2 * MAX_LIMBS + 2];
  uint64_t ma[MAX_LIMBS], mb[MAX_LIMBS];
  memset(acc, 0, sizeof(uint64_t) * (size_t)w);
  int64_t i_lo = k - (J->lg - 1);
  if (i_lo < 0) i_lo = 0;
  int64_t i_hi = k < J->lf - 1 ? k : J->lf - 1;
  for (int64_t i = i_lo; i <= i_hi; i++) {
    int sa = magnitude(ma, J->f + i * n, n, J->is_signed);
    int sb = magnitude(mb, J->g + (k - i) * n, n, J->is_signed);
    acc_product(acc, w, ma, mb, n, sa ^ sb);
  }
  memcpy(out, acc, sizeof(uint64_t) * (size_t)J->out_limbs);
}

static void *worker(void *arg) {
  job_t *J = (job_t *)arg;
  for (int64_t t = J->begin; t < J->nk; t += J->stride) {
    int64_t k = J->ks ? J->ks[t] : t;
    one_coeff(J->h + t * J->out_limbs, J, k);
  }
  return NULL;
}

static int run_jobs(job_t base, int nthreads) {
  if (nthreads < 1) nthreads = 1;
  if (nthreads > 256) nthreads = 256;
  if (base.nk < nthreads) nthreads = base.nk > 0 ? (int)base.nk : 1;
  pthread_t th[256];
  job_t jobs[256];
  /* interleaved ownership balances the triangular cost of the coefficients */
  for (int t = 0; t < nthreads; t++) {
    jobs[t] = base;
    jobs[t].begin = t;
    jobs[t].stride = nthreads;
  }
  int started = 1, rc = 0;
  for (int t = 1; t < nthreads; t++, started++)
    if (pthread_create(&th[t], NULL, worker, &jobs[t]) != 0) { rc = -3; break; }
  if (rc == 0) worker(&jobs[0]);
  for (int t = 1; t < started; t++) pthread_join(th[t], NULL);
  return rc;
}

/* Full product: h holds (lf + lg - 1) * out_limbs limbs. */
int oracle_mul(uint64_t *h, const uint64_t *f, int64_t lf, const uint64_t *g,
               int64_t lg, int coeff_bits, int is_signed, int out_limbs,
               int nthreads) {
  if (lf < 1 || lg < 1 || coeff_bits < 1) return -1;
  int n = (coeff_bits + 63) / 64;
  if (n > MAX_LIMBS || out_limbs < 1 || out_limbs > 2 * MAX_LIMBS + 2) return -1;
  job_t J = {h, f, g, lf, lg, n, is_signed, out_limbs, NULL, lf + lg - 1, 0, 0};
  return run_jobs(J, nthreads);
}

/* Selected coefficients: out[t] = h_{ks[t]}. */
int oracle_coeffs(uint64_t *out, const int64_t *ks, int64_t nk,
                  const uint64_t *f, int64_t lf, const uint64_t *g, int64_t lg,
                  int coeff_bits, int is_signed, int out_limbs, int nthreads) {
  if (lf < 1 || lg < 1 || coeff_bits < 1) return -1;
  int n = (coeff_bits + 63) / 64;
  if (n > MAX_LIMBS || out_limbs < 1 || out_limbs > 2 * MAX_LIMBS + 2) return -1;
  for (int64_t t = 0; t < nk; t++)
    if (ks[t] < 0 || ks[t] >= lf + lg - 1) return -1;
  job_t J = {out, f, g, lf, lg, n, is_signed, out_limbs, ks, nk, 0, 0};
  return run_jobs(J, nthreads);
}

/* ---- (Z/pZ)[x]: h_k = sum f_i g_j mod p, residues in [0, p), one limb ---- */

typedef struct {
  uint64_t *h;
  const uint64_t *f, *g;
  int64_t lf, lg;
  uint64_t p;
  int64_t begin, stride;
} mjob_t;

static void *mworker(void *arg) {
  mjob_t *J = (mjob_t *)arg;
  int64_t nk = J->lf + J->lg - 1;
  for (int64_t k = J->begin; k < nk; k += J->stride) {
    int64_t i_lo = k - (J->lg - 1);
    if (i_lo < 0) i_lo = 0;
    int64_t i_hi = k < J->lf - 1 ? k : J->lf - 1;
    uint64_t acc = 0;
    for (int64_t i = i_lo; i <= i_hi; i++) {
      uint64_t t = (uint64_t)(((u128)J->f[i] * J->g[k - i]) % J->p);
      acc = (uint64_t)(((u128)acc + t) % J->p);
    }
    J->h[k] = acc;
  }
  return NULL;
}

int oracle_mul_mod(uint64_t *h, const uint64_t *f, int64_t lf,
                   const uint64_t *g, int64_t lg, uint64_t p, int nthreads) {
  if (lf < 1 || lg < 1 || p < 2) return -1;
  for (int64_t i = 0; i < lf; i++) if (f[i] >= p) return -1;
  for (int64_t i = 0; i < lg; i++) if (g[i] >= p) return -1;
  int64_t nk = lf + lg - 1;
  if (nthreads < 1) nthreads = 1;
  if (nthreads > 256) nthreads = 256;
  if (nk < nthreads) nthreads = (int)nk;
  pthread_t th[256];
  mjob_t jobs[256];
  for (int t = 0; t < nthreads; t++) {
    mjob_t J = {h, f, g, lf, lg, p, t, nthreads};
    jobs[t] = J;
  }
  int started = 1, rc = 0;
  for (int t = 1; t < nthreads; t++, started++)
    if (pthread_create(&th[t], NULL, mworker, &jobs[t]) != 0) { rc = -3; break; }
  if (rc == 0) mworker(&jobs[0]);
  for (int t = 1; t < started; t++) pthread_join(th[t], NULL);
  return rc;
}

/* ---- (Z/pZ)[x, y]: the plain bivariate product (Harvey, Sec. 2) ----
 *
 * f and g have ly rows of lx residues in [0, p): row i holds the coefficients
 * of f_i(x), the coefficient of y^i.  h has 2 ly - 1 rows of 2 lx - 1:
 *
 *     h[k][m] = sum_{i + i' = k} sum_{j + j' = m} f[i][j] g[i'][j']  mod p,
 *
 * one term at a time, each reduced mod p through a 128-bit product.
 * Multithreaded over the rows k of h. */

typedef struct {
  uint64_t *h;
  const uint64_t *f, *g;
  int64_t lx, ly;
  uint64_t p;
  int64_t begin, stride;
} bjob_t;

static void *bworker(void *arg) {
  bjob_t *J = (bjob_t *)arg;
  const int64_t hy = 2 * J->ly - 1, hx = 2 * J->lx - 1;
  for (int64_t k = J->begin; k < hy; k += J->stride) {
    for (int64_t m = 0; m < hx; m++) {
      uint64_t acc = 0;
      for (int64_t i = 0; i < J->ly; i++) {
        const int64_t i2 = k - i;
        if (i2 < 0 || i2 >= J->ly) continue;
        for (int64_t j = 0; j < J->lx; j++) {
          const int64_t j2 = m - j;
          if (j2 < 0 || j2 >= J->lx) continue;
          const uint64_t t =
              (uint64_t)(((u128)J->f[i * J->lx + j] * J->g[i2 * J->lx + j2]) % J->p);
          acc = (uint64_t)(((u128)acc + t) % J->p);
        }
      }
      J->h[k * hx + m] = acc;
    }
  }
  return NULL;
}

int oracle_mul_biv_mod(uint64_t *h, const uint64_t *f, const uint64_t *g, int64_t lx, int64_t ly,
                       uint64_t p, int nthreads) {
  if (lx < 1 || ly < 1 || p < 2) return -1;
  for (int64_t i = 0; i < lx * ly; i++)
    if (f[i] >= p || g[i] >= p) return -1;
  const int64_t hy = 2 * ly - 1;
  if (nthreads < 1) nthreads = 1;
  if (nthreads > 256) nthreads = 256;
  if (hy < nthreads) nthreads = (int)hy;
  pthread_t th[256];
  bjob_t jobs[256];
  for (int t = 0; t < nthreads; t++) {
    bjob_t J = {h, f, g, lx, ly, p, t, nthreads};
    jobs[t] = J;
  }
  int started = 1, rc = 0;
  for (int t = 1; t < nthreads; t++, started++)
    if (pthread_create(&th[t], NULL, bworker, &jobs[t]) != 0) { rc = -3; break; }
  if (rc == 0) bworker(&jobs[0]);
  for (int t = 1; t < started; t++) pthread_join(th[t], NULL);
  return rc;
}
