/*
 * ks.h -- C ABI of the GB300 multipoint Kronecker-substitution library.
 *
 * Computes h = f * g in Z[x] for dense polynomials with multi-word integer
 * coefficients, by the Kronecker substitution of Harvey, "Faster polynomial
 * multiplication via multipoint Kronecker substitution" (arXiv:0712.4046):
 *
 *   KS_1  evaluate at 2^N, N = 2b + e                      (Sec. 3.1)
 *   KS_2  evaluate at +2^N and -2^N, N = b + ceil(e/2)     (Sec. 3.3)
 *   KS_3  evaluate at 2^N and 2^-N,  N = b + ceil(e/2)     (Sec. 3.2)
 *   KS_4  all four points, N = ceil((2b + e) / 4)          (Sec. 3.4)
 *
 * with b the coefficient bit bound and e = ceil(log2 min(len_f, len_g))
 * (Sec. 3 states the method for equal lengths L; unequal lengths use the
 * shorter one, which bounds the number of terms of each h_k).  Every variant
 * returns the same, exact product.
 *
 * Coefficient layout (inputs and outputs):
 *   - coefficient i occupies `limbs` consecutive little-endian uint64 words;
 *     inputs use in_limbs = ceil(coeff_bits / 64), outputs use
 *     ks_out_limbs(...) limbs;
 *   - unsigned coefficients lie in [0, 2^b); signed ones in
 *     [-2^(b-1), 2^(b-1)), two's complement, sign-extended over the limbs
 *     (Sec. 3 treats non-negative coefficients; for signed ones the variants
 *     evaluate the signed coefficients as they are -- Sec. 3.3's evaluations
 *     are signed anyway -- and read every coefficient shifted by
 *     K = 2^(2b-2+e) >= |h_k|, which puts it in the non-negative range the
 *     read-off and the reconstruction of Sec. 3 need; K is subtracted on
 *     output);
 *   - h holds len_f + len_g - 1 coefficients in the same encoding.
 *
 * Pointers: "device" means memory the current CUDA device can address
 * (cudaMalloc or torch CUDA tensors); "host" means ordinary or pinned host
 * memory.  All device work is issued on `stream` (a cudaStream_t passed as
 * void*, NULL = the legacy default stream) and is asynchronous unless stated.
 *
 * Errors: every call returns a ks_status; nothing is thrown across the ABI.
 * Asynchronous device-side failures (a bounded wait that gave up, a failed
 * range check of the reconstruction) are reported by ks_status_sync() for
 * the single-product calls and by ks_plan_status() for a plan.  On any error
 * the output is unspecified.
 */
#ifndef KS_H
#define KS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef void *ks_stream_t; /* a cudaStream_t */

/* Variant selector (Sec. 3.1-3.4).  KS_AUTO lets the library choose.  KS_C,
 * the complex evaluation points of Sec. 2.5, exists for ks_mul_bivariate_mod
 * only. */
enum { KS_AUTO = 0, KS_1 = 1, KS_2 = 2, KS_3 = 3, KS_4 = 4, KS_C = 5 };

/* Engine for the independent big-integer sub-products. */
enum {
  KS_ENGINE_AUTO = 0,
  KS_ENGINE_SCHOOLBOOK = 1, /* exact digit contraction on the INT32 pipe */
  KS_ENGINE_NTT = 2,        /* multi-prime number-theoretic transform + CRT */
  KS_ENGINE_TC = 3          /* exact digit contraction on the tensor cores */
};

typedef enum {
  KS_OK = 0,
  KS_EINVAL = -1,   /* bad length, bit size, variant, engine, pointer or aliasing */
  KS_ERANGE = -2,   /* size beyond a documented maximum */
  KS_ENOMEM = -3,   /* a device or host allocation failed */
  KS_ECUDA = -4,    /* a CUDA runtime call failed (see ks_last_cuda_error) */
  KS_ETIMEOUT = -5, /* a bounded device-side wait gave up */
  KS_ENOTSUP = -6   /* engine or mode not available for these sizes */
} ks_status;

/* Largest supported coefficient bound b (bits). */
#define KS_MAX_COEFF_BITS 2048

/*
 * Limbs per output coefficient: ceil((2b + e + is_signed) / 64), where
 * e = ceil(log2 min(len_f, len_g)).  Sec. 3, eq. (h-inequality):
 * 0 <= h_i <= L (2^b - 1)^2 < 2^(2b+e) for unsigned inputs; a signed result
 * needs one more bit for its sign.  Returns a negative ks_status on bad input.
 */
int ks_out_limbs(int64_t len_f, int64_t len_g, int coeff_bits, int is_signed);

/*
 * Limbs per output coefficient for bits_f-bit coefficients in f and
 * bits_g-bit ones in g: ceil((bits_f + bits_g + e + is_signed) / 64), since
 * |h_i| <= L 2^bits_f 2^bits_g (the same inequality with bits_f + bits_g in
 * place of 2b).  ks_out_limbs(.., b, ..) is ks_out_limbs_bits(.., b, b, ..).
 */
int ks_out_limbs_bits(int64_t len_f, int64_t len_g, int bits_f, int bits_g, int is_signed);

/* Evaluation exponent N the given variant uses (Sec. 3.1-3.4); < 0 on error. */
int ks_eval_bits(int64_t len_f, int64_t len_g, int coeff_bits, int variant);

/*
 * Bytes of device workspace ks_mul_ex needs for this problem, variant and
 * engine (KS_AUTO / KS_ENGINE_AUTO resolve as ks_mul would).  < 0 on error.
 */
int64_t ks_workspace_bytes(int64_t len_f, int64_t len_g, int coeff_bits,
                           int is_signed, int variant, int engine);

/*
 * h = f * g (device pointers), exactly.  f has len_f coefficients, g has
 * len_g, both with coeff_bits-bit coefficients (signed if is_signed); h
 * receives len_f + len_g - 1 coefficients of ks_out_limbs() limbs.
 * h must not overlap f or g; f may equal g.  Workspace comes from a cache
 * the library keeps per (device, stream) and grows on demand (so the first
 * call for a size allocates; later ones do not).  Asynchronous on `stream`.
 * The phase that reads only f and g (the exact seeds of Sec. 3.2's
 * reconstruction) runs on a helper stream the library creates on the first
 * call per (device, stream),
 * forked from and joined back into `stream` with events; as seen from
 * `stream` the call is ordered like any other work on it, and it can be
 * captured into a CUDA graph (the helper stream becomes a parallel branch)
 * once a call of the same size has run outside the capture.  The first call
 * on each device (of any entry point) also loads the transform engine's
 * twiddle tables with blocking copies; a transform product whose first use
 * on a device is inside a capture returns KS_ECUDA and leaves the capture
 * intact.
 */
int ks_mul(uint64_t *h, const uint64_t *f, int64_t len_f, const uint64_t *g,
           int64_t len_g, int coeff_bits, int is_signed, int variant,
           ks_stream_t stream);

/*
 * As ks_mul, with an explicit engine and caller-owned device workspace of at
 * least ks_workspace_bytes() bytes (256-byte aligned).  Allocates no device
 * memory (it shares ks_mul's helper stream, created on first use).
 */
int ks_mul_ex(uint64_t *h, const uint64_t *f, int64_t len_f, const uint64_t *g,
              int64_t len_g, int coeff_bits, int is_signed, int variant,
              int engine, void *workspace, int64_t workspace_bytes,
              ks_stream_t stream);

/*
 * As ks_mul but with HOST buffers: copies f and g to the device, multiplies,
 * copies h back, and returns when h is complete (synchronous).  Device
 * buffers are cached per (device, stream).  On a stream other than the legacy
 * default streams, the product's launches are captured into a CUDA graph on
 * the first call of a problem (size, variant, engine) and replayed by the
 * following calls of the same problem on that stream; another problem, a
 * change of ks_set_pdl or ks_release_cache captures afresh.  Returns the
 * device status word's error (as ks_status_sync would) with the result.
 */
int ks_mul_host(uint64_t *h, const uint64_t *f, int64_t len_f,
                const uint64_t *g, int64_t len_g, int coeff_bits,
                int is_signed, int variant, int engine, ks_stream_t stream);

/*
 * (Z/pZ)[x] product (Sec. 4): residues in [0, p) as one uint64 limb each,
 * 2 <= p < 2^63; h receives (h_k mod p), one limb each.  The polynomials are
 * lifted to Z[x] with b = bitlength(p - 1), multiplied exactly by the chosen
 * variant, and reduced.  Device pointers, asynchronous.
 */
int ks_mul_mod(uint64_t *h, const uint64_t *f, int64_t len_f, const uint64_t *g,
               int64_t len_g, uint64_t p, int variant, ks_stream_t stream);

/*
 * h = f * g for coefficients of different sizes: f has bits_f-bit
 * coefficients (ceil(bits_f / 64) limbs each), g has bits_g-bit ones
 * (ceil(bits_g / 64) limbs; signed or unsigned as for ks_mul, both the same).
 * Every size bound of Sec. 3.1-3.4 holds with bits_f + bits_g in place of
 * 2b, so the evaluation exponents are N = bits_f + bits_g + e (KS_1),
 * ceil((bits_f + bits_g + e) / 2) (KS_2, KS_3; signed KS_3 at most 2 below
 * that sum: 2) and ceil((bits_f + bits_g + e) / 4) (KS_4); each operand is
 * packed from its own limbs with its own field width, and signed results are
 * read shifted by K = 2^(bits_f + bits_g - 2 + e).  h has
 * ks_out_limbs_bits(len_f, len_g, bits_f, bits_g, is_signed) limbs per
 * coefficient.  KS_AUTO chooses as ks_mul does for ceil((bits_f + bits_g) / 2)
 * bits.  Workspace is cached per (device, stream).  Asynchronous.
 */
int ks_mul_bits(uint64_t *h, const uint64_t *f, int64_t len_f, int bits_f,
                const uint64_t *g, int64_t len_g, int bits_g, int is_signed,
                int variant, ks_stream_t stream);

/*
 * Bivariate product in (Z/pZ)[x, y] (Sec. 2): f and g are device arrays of
 * ly rows of lx residues in [0, p) (row i, entry j: the coefficient of
 * x^j y^i); h receives 2 ly - 1 rows of 2 lx - 1 residues.  2 <= p < 2^63.
 * The variant is the polynomial-ring substitution of the paper:
 *   KS_1  y = x^N, N = 2 lx - 1, one product of length (ly - 1) N + lx (Sec. 2.1)
 *   KS_2  y = +-x^N, N = lx, two products of length lx ly (Sec. 2.3; p odd)
 *   KS_3  y = x^N and x^-N, N = lx, two products of length lx ly (Sec. 2.2)
 *   KS_4  y = +-x^N, +-x^-N, N = ceil(lx / 2), four products of length
 *         N (ly - 1) + lx (Sec. 2.4; p odd)
 *   KS_C  y = x^M, -x^M and i x^M, M = ceil(lx / 2), in R[i] = R[t]/(t^2 + 1)
 *         (Sec. 2.5; p odd): f(x, i x^M) = F_re + i F_im, and the complex
 *         product by three real ones (F_re G_re, F_im G_im,
 *         (F_re + F_im)(G_re + G_im)): five products of length M (ly - 1) + lx.
 *         With A_r the part of h(x, x^M) whose rows k are r mod 4,
 *         h(x, +-x^M) = A0 +- A1 + A2 +- A3, Re = A0 - A2, Im = A1 - A3, and
 *         every A_r is a quarter of a sum of those; its rows lie 4M >= 2 lx - 1
 *         apart, so they are read off.
 *   KS_AUTO  KS_2 for odd p, else KS_1.
 * Each univariate product runs through ks_mul_mod (whose own substitution
 * is chosen as for KS_AUTO).  Workspace is cached per (device, stream).
 * KS_EINVAL for bad arguments (KS_2 / KS_4 / KS_C with even p); KS_ERANGE beyond
 * lx, ly <= 2^26 and lx ly <= 2^28.  Asynchronous on `stream`.
 */
int ks_mul_bivariate_mod(uint64_t *h, const uint64_t *f, const uint64_t *g, int64_t lx,
                         int64_t ly, uint64_t p, int variant, ks_stream_t stream);

/*
 * ks_mul_static -- ks_mul without any allocation.  (The paper has no
 * counterpart; this entry point is a deployment convenience.)
 *
 * For callers that cannot allocate device memory when they multiply: code
 * whose device memory is owned and budgeted by another allocator (a
 * framework's caching pool, a fixed-size serving arena), code that must not
 * trigger cudaMalloc / cudaFree because those calls can synchronize the whole
 * device and stall unrelated work, and plugin hosts that forbid allocation
 * after start-up.  ks_mul grows a cached workspace on demand and ks_mul_ex
 * needs the caller to provide one; this call needs neither.
 *
 * Scratch lives in one file-scope device array of KS_STATIC_SCRATCH_BYTES
 * inside the library, which every GPU that loads the library keeps until the
 * process exits.  Problems whose workspace (ks_workspace_bytes with
 * KS_ENGINE_AUTO) is larger are refused with KS_ERANGE before anything runs.
 * The caller still passes f, g and h as device memory, exactly as for
 * ks_mul; the call makes no cudaMalloc, cudaFree or other allocating call.
 *
 * The first call on each device looks up the array's device address
 * (cudaGetSymbolAddress, with that device current) and loads the transform
 * engine's tables (blocking copies); make that first call before any stream
 * capture begins.  All calls, from any thread or stream,
 * share the one array and it keeps the last call's contents; the parts that
 * must start at zero are cleared on `stream` by every call.  Calls that
 * overlap on the GPU race on the array: order them (one stream, or events).
 */
#define KS_STATIC_SCRATCH_BYTES (16 << 20)
int ks_mul_static(uint64_t *h, const uint64_t *f, int64_t len_f,
                  const uint64_t *g, int64_t len_g, int coeff_bits,
                  int is_signed, int variant, ks_stream_t stream);

/*
 * One product of a batch (device pointers, layout as for ks_mul).
 * coeff_bits_g = 0: g has coeff_bits-bit coefficients like f; otherwise g's
 * size, and the product is ks_mul_bits's (h with ks_out_limbs_bits limbs).
 */
typedef struct {
  uint64_t *h;
  const uint64_t *f;
  const uint64_t *g;
  int64_t len_f, len_g;
  int32_t coeff_bits, is_signed, variant, engine;
  int32_t coeff_bits_g;
} ks_problem;

/*
 * Runs n independent products on `stream` as one batched launch sequence and
 * returns when they are done (synchronous; it plans, allocates and frees a
 * plan -- use the plan API below to reuse one).  probs is a HOST array of
 * descriptors with DEVICE pointers.  Each product's variant and engine may
 * be KS_AUTO.
 */
int ks_mul_batch(const ks_problem *probs, int64_t n, ks_stream_t stream);

/*
 * Batched plans (no counterpart in the paper; its Sec. 1 remark that the
 * sub-products are independent is what they exploit).  ks_plan_create plans
 * n products (problem array on the HOST, device pointers inside), allocates
 * one device workspace for all of them and uploads the per-kernel work
 * descriptors.  ks_plan_execute issues one launch per phase for the whole
 * batch on `stream` (asynchronous); the four sub-products of every four-point
 * product are independent work items of one persistent tensor-core kernel.
 * ks_plan_capture runs the plan once, then records its launches into a CUDA
 * graph on `stream` (a non-default stream); later ks_plan_execute calls on
 * that stream replay the graph.  The plan keeps the pointers it was created
 * with: the inputs may change between executes, the buffers may not move.
 * Dispatch modes choose variant and engine where a problem says KS_AUTO:
 *   KS_DISPATCH_AUTO  the library's choice (cost table, then learned model)
 *   KS_DISPATCH_KS1   always KS_1 (the standard substitution), engine auto
 *   KS_DISPATCH_TABLE the autotuned table only
 *   KS_DISPATCH_MLP   the learned cost model only
 */
typedef struct ks_plan ks_plan;
enum { KS_DISPATCH_AUTO = 0, KS_DISPATCH_KS1 = 1, KS_DISPATCH_TABLE = 2, KS_DISPATCH_MLP = 3 };
int ks_plan_create(ks_plan **plan, const ks_problem *probs, int64_t n, int dispatch_mode);
int ks_plan_execute(ks_plan *plan, ks_stream_t stream);
int ks_plan_capture(ks_plan *plan, ks_stream_t stream);
/*
 * The plan's own device status word (Sec. 3.2's reconstruction checks its
 * carries delta, epsilon in {0, 1}; every device wait of the plan's kernels is
 * bounded): waits for the stream of the plan's last execute, reads the word,
 * clears it and returns KS_OK, KS_ETIMEOUT (a bounded wait gave up) or
 * KS_ERANGE (a range check failed).  KS_EINVAL for NULL; KS_ECUDA if the
 * wait or the copy fails.  Other plans and single calls do not touch it.
 */
int ks_plan_status(ks_plan *plan);
/* Kernel launches of the last non-graph execute; device bytes the plan holds. */
long long ks_plan_launches(const ks_plan *plan);
int64_t ks_plan_workspace_bytes(const ks_plan *plan);
/* The variant and engine the plan chose for product i. */
int ks_plan_choice(const ks_plan *plan, int64_t i, int *variant, int *engine);
/* Waits for the device, then frees the plan (NULL is ignored). */
void ks_plan_destroy(ks_plan *plan);

/*
 * Dispatch: the autotuned table and the learned cost model (no counterpart
 * in the paper, which picks the variant by hand per experiment; Sec. 4 notes
 * that small degrees favour the standard substitution).  Neither affects the
 * result -- every choice is an exact path -- only which path runs where a
 * problem says KS_AUTO.
 *
 * ks_tune_time: mean device time per product (ms) of one (variant, engine)
 * on `batch` equal-shaped products with synthetic coefficients, over `reps`
 * executions of a batched plan, after two warm-up executions (synchronous).
 *
 * ks_dispatch_set_table: installs the autotuned table, n rows of 6 int32:
 * (len_f, len_g, coeff_bits, is_signed, best variant, best engine).  KS_AUTO
 * then takes the nearest row in log2 space (n = 0 clears it).
 *
 * The cost model is an MLP 5 -> 32 -> 32 -> 12 (ReLU) whose output
 * 3 (variant - 1) + e (e = 0 schoolbook, 1 NTT, 2 tensor cores) predicts
 * log2 of the time per product in microseconds from the features
 * (log2 len_f / 20, log2 len_g / 20, log2 bits / 11, signed, min(log2 W, 26) / 26),
 * W the operand bits of the whole batch, sum of (len_f + len_g) bits over its
 * products (a batch beyond 2^26 bits fills the GPU, and a product's cost is
 * then its share of the work rather than its latency).
 * Parameters: KS_MLP_PARAMS floats, W1 [32x5], b1, W2 [32x32], b2, W3 [12x32],
 * b3.  ks_mlp_train: full-batch Adam on the GPU (the library's forward,
 * backward and update kernels), masked mean squared error; params updated in
 * place.  ks_mlp_grad: one forward and backward pass on the GPU, the gradient
 * and loss returned to the host.  ks_mlp_predict: inference kernel for n
 * feature rows (requires installed parameters).  ks_mlp_set_params installs
 * parameters for dispatch (NULL uninstalls).  All arrays here are HOST arrays;
 * x is n x 5, t and mask are n x 12.
 */
#define KS_MLP_IN 5
#define KS_MLP_HIDDEN 32
#define KS_MLP_OUT 12
int ks_tune_time(int64_t len_f, int64_t len_g, int coeff_bits, int is_signed,
                 int variant, int engine, int batch, int reps,
                 double *ms_per_product);
int ks_dispatch_set_table(int64_t n, const int32_t *rows);
int64_t ks_mlp_param_count(void);
int ks_mlp_set_params(const float *params);
int ks_mlp_train(float *params, const float *x, const float *t,
                 const float *mask, int64_t n, int steps, float lr,
                 float *loss);
int ks_mlp_grad(const float *params, const float *x, const float *t,
                const float *mask, int64_t n, float *grad, float *loss);
int ks_mlp_predict(const float *x, int64_t n, float *y);

/* Waits for `stream`, then reports a pending device-side error (or KS_OK). */
int ks_status_sync(ks_stream_t stream);

/* The variant and engine KS_AUTO / KS_ENGINE_AUTO resolve to for a problem. */
int ks_choose(int64_t len_f, int64_t len_g, int coeff_bits, int is_signed,
              int *variant, int *engine);

/* Message for a ks_status; the last CUDA error string for KS_ECUDA. */
const char *ks_strerror(int status);
const char *ks_last_cuda_error(void);

/*
 * Instrumentation.  ks_launch_count: kernels the library has launched so far
 * (a host-side counter).  ks_profile_enable(1) makes every later call record
 * a pair of CUDA events around each phase on its stream; ks_profile_collect
 * waits for those events and returns, per phase id (0 .. n-1, names from
 * ks_phase_name), the summed milliseconds and the number of records, then
 * clears them.  Phases: 0 pack, 1 product, 2 normalize, 3 unpack, 4 seeds,
 * 5 recover, 6 reduce_mod.  Seeds read only f and g and run on a helper
 * stream concurrently with the normalization (their events are recorded on
 * that stream).
 */
long long ks_launch_count(void);

/*
 * Launch overlap (no counterpart in the paper).  With enabled != 0 the
 * library launches its kernels with programmatic dependent launch: a kernel
 * may be scheduled while the previous kernel of its stream is still running
 * and waits on the device, before touching memory, until that kernel has
 * finished.  enabled = 0 (the default) launches every kernel after the
 * previous one has finished.  Results are identical either way.  Calls and
 * plans captured afterwards use the setting; plans captured earlier keep
 * theirs.
 */
void ks_set_pdl(int enabled);

/*
 * Host-side fault injection for tests (no counterpart in the paper): the next
 * n device allocations the library makes (cached workspaces, plans) fail as
 * if the device were out of memory, so the calls return KS_ENOMEM.  No device
 * is touched by the failure.  n <= 0 clears it.
 */
void ks_debug_fail_allocs(int n);

/*
 * Test hook for the device-side failure path (no counterpart in the paper):
 * with on != 0, later launches of the tensor-core product kernel wait, before
 * their first operand copy, on a barrier that nothing completes, and every
 * wait of that kernel is bounded by wait_ns (> 0; else the default of one
 * second).  The wait runs out while no copy or MMA is in flight; the kernel
 * records the timeout in the status word, releases its tensor memory and
 * returns, and ks_status_sync / ks_plan_status report KS_ETIMEOUT.  on = 0
 * restores the normal kernel (wait_ns <= 0: the default bound).  Plans keep the
 * setting in force when they were created or captured.
 */
void ks_debug_tc_stall(int on, int64_t wait_ns);

/*
 * Test hook: which form the carry normalization takes (no counterpart in the
 * paper).  0: by size (one single-pass launch up to 2048 tile CTAs, else a
 * tile pass and a carry pass), 1: always the single pass, 2: always the two
 * passes.  Both give the same words; a captured plan keeps the form it was
 * captured with.
 */
void ks_debug_norm_form(int form);

/*
 * Test hook, host only: how the tensor-core engine would split the work of
 * one product (this variant, engine KS_ENGINE_TC) over `grid` <= 160 CTAs.
 * The work is the sequence of (sub-product, output tile, block offset), total
 * entries in all; CTA k takes [at[k], at[k + 1]) (at: grid + 1 entries) and
 * its first item lies in tile first_tile[k] of sub-product first_q[k].
 * (The paper has no counterpart: this is the engine's own scheduling.)
 */
int ks_debug_tc_split(int64_t len_f, int64_t len_g, int coeff_bits, int is_signed,
                      int variant, int grid, int64_t *at, int32_t *first_q,
                      int32_t *first_tile, int64_t *total);

/*
 * The plan ks_mul_ex would run, as int64 fields (n of them are written):
 * 0 variant, 1 engine, 2 N, 3 digit bits d, 4 sub-products, 5 digits of each
 * f-side operand, 6 digits of each g-side operand, 7 column sums per
 * sub-product, 8 words per normalized value, 9 normalized values,
 * 10 reconstruction digit bits M (0 for KS_1 / KS_2), 11 chain length,
 * 12 exact seed values (two per seed pair of each run), 13 output limbs, 14 input limbs, 15 workspace bytes,
 * 16 log2 of the transform length (NTT engine, else 0), 17-20 workspace byte
 * offsets of the digits, column sums, normalized words and seeds, 21 words
 * per seed, 22-23 reconstruction chains of the two runs.
 */
int ks_plan_info(int64_t len_f, int64_t len_g, int coeff_bits, int is_signed,
                 int variant, int engine, int64_t *info, int n);
/* The plan ks_mul_bits (or a batch problem with coeff_bits_g) would run, as
 * ks_plan_info's fields; field 14 is the larger operand's limb count. */
int ks_plan_info_bits(int64_t len_f, int64_t len_g, int bits_f, int bits_g, int is_signed,
                      int variant, int engine, int64_t *info, int n);
void ks_profile_enable(int on);
int ks_profile_collect(double *ms, long long *count, int n);
const char *ks_phase_name(int phase);

/* Library version (major * 10000 + minor * 100 + patch). */
int ks_version(void);

/* Releases the cached workspaces of the calling device. */
void ks_release_cache(void);

#ifdef __cplusplus
}
#endif

#endif /* KS_H */
