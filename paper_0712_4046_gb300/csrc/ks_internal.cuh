// Internal declarations shared by the CUDA translation units of the library.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stddef.h>
#include <cuda_fp16.h>

#include "../../include/ks.h"

namespace ks {

// ---------------------------------------------------------------- limits
constexpr int kMaxOperands = 8;      // 4 sub-products x 2 sides
constexpr int kMaxSeedWords = 136;   // exact seeds: (2b + e) bits, b <= 2048
constexpr int kAccSeedWords = 8;     // words of a narrow seed value (six column sums, mod 2^192)
constexpr int kMaxDigitWordsM = 72;  // reconstruction digit: M <= 2304 bits

// ---------------------------------------------------------------- planning
// Geometry of the tensor-core engine for one sub-product of nA x nB 7-bit digits.
struct TcGeom {
  int64_t nA = 0, nB = 0;
  int64_t dmax = 0;   // largest block offset delta (blocks of 128 digits)
  int64_t R = 0;      // rows (blocks of 128 digits) of the B operand
  int64_t Pcols = 0;  // output block columns
  int64_t T = 0;      // output tiles of 128 block columns
  int64_t nE = 0;     // rows of the A window array (8 fp16 digits each, zero padded)
  int64_t rows = 0;   // rows per B plane, zero padding included
  int64_t ncols = 0;  // output column sums of four 8-bit digits (32-bit digits)
};

struct Plan {
  int variant = 0, engine = 0;
  int64_t lf = 0, lg = 0, lh = 0;
  int b = 0, e = 0, N = 0, is_signed = 0, in_limbs = 0, out_limbs = 0;
  // coefficient bits and limbs of f and of g (b, in_limbs: the larger ones);
  // bf + bg takes the place of 2b in every size bound
  int bf = 0, bg = 0, ilf = 0, ilg = 0;
  int d = 16;           // digit bits of the sub-product operands
  int dn = 16;          // digit bits of the column sums fed to the normalization
  TcGeom tg;
  int nprod = 0;        // independent sub-products (1, 2, 2, 4)
  int64_t nA = 0, nB = 0;  // digits of each f-side / g-side operand
  int64_t ncols = 0;    // column sums per sub-product
  int64_t nwords = 0;   // 32-bit words per normalized combination
  int nnorm = 0;        // normalized combinations (1, 2, 2, 4)
  int kb = -1;           // signed: coefficients are read shifted by K = 2^kb
  // reconstruction (Sec. 3.2; run twice for Sec. 3.4)
  int M = 0;            // digit bits: N (KS3) or 2N (KS4)
  int nruns = 0;
  int64_t run_n[2] = {0, 0};
  int64_t chain = 0;
  int64_t nchains[2] = {0, 0};
  int seed_words = 0;
  int C = 0;            // seed values per cluster: 2 (KS3) or 4 (KS4)
  int64_t ncl = 0;      // seed clusters (the pairs of the longest run)
  int64_t k00 = 0, kstep = 0;  // first h index of cluster j: k00 + kstep j
  int64_t nseeds = 0;   // seed values: ncl C
  // number-theoretic-transform engine
  int ntt_log = 0;      // transform length 2^ntt_log
  // workspace layout (byte offsets from the base)
  size_t off_digits = 0, off_cols = 0, off_flags = 0, off_words = 0;
  int64_t flag_bytes = 0;  // the normalization's per-tile transfer functions
  int64_t zero_words = 0;  // 64-bit words cleared before a product: column sums, flags
  size_t off_seeds = 0, off_seedacc = 0, off_planes = 0, off_hp = 0, off_ntt = 0;
  size_t total = 0;
  int64_t ntiles = 0;   // scan tiles per normalized combination
};

int ceil_log2(int64_t n);
// Retires the graphs a host-buffer call captured (a setting they bake in changed).
void bump_epoch();
// N of a variant for coefficient sizes adding up to s = bf + bg (2b for equal ones)
int variant_N_sum(int variant, int s, int e);
int variant_N(int variant, int b, int e);
// Fills `p` (layout included) for an explicit variant and engine; KS_OK or
// error.  f has b-bit coefficients, g bg-bit ones (bg = 0: b bits as well).
int make_plan(Plan &p, int64_t lf, int64_t lg, int b, int is_signed, int variant,
              int engine, int bg = 0);
int choose(int64_t lf, int64_t lg, int b, int is_signed, int *variant, int *engine);
// g's coefficient bits of a batch problem, and the equal size the dispatch
// sees for it (ceil((bf + bg) / 2): the exponents N depend on bf + bg only)
inline int problem_bits_g(const ks_problem &q) {
  return q.coeff_bits_g != 0 ? q.coeff_bits_g : q.coeff_bits;
}
inline int problem_bits(const ks_problem &q) { return (q.coeff_bits + problem_bits_g(q) + 1) / 2; }
int signed_N_sum(int variant, int s, int e);

// ---------------------------------------------------------------- kernels
struct PackOp {
  const uint64_t *poly;
  int64_t L;
  int reversed;  // coefficient t of the evaluated polynomial is poly[L-1-t]
  int sigma;     // +1: f(X); -1: f(-X) (odd coefficients negated)
  int32_t *out;
  int64_t ndig;
  int b = 0;       // coefficient bits of this operand
  int il = 0;      // 64-bit limbs per coefficient
  int narrow = 0;  // every bit position of this evaluation is below 2^31
};

struct PackArgs {
  PackOp op[kMaxOperands];
  int nops;
  int N, b, d, in_limbs, flip;  // b, in_limbs: the largest over the operands
  uint64_t ninv = 0;  // floor(2^64 / N) + 1: floor(x / N) = umulhi(x, ninv), x < 2^31
  int fields = 0;     // > 0: coefficient fields per CTA of the field-centric path (N >= b)
};
// Fills ninv and the per-operand narrow flags (after the operands are set).
void pack_finish(PackArgs &a);

struct Product;
// Squaring: keeps only the f-side operand of each sub-product (2 q) and makes
// every sub-product read it on both sides.
void squaring_pack(PackArgs &a, Product *prods, int nprod);

// Signed digits of each evaluation (Sec. 3.1-3.4 evaluations at +-2^N and
// the reversed polynomial), `d` bits per digit position.
cudaError_t launch_pack(const PackArgs &a, cudaStream_t s);
int64_t pack_blocks(const PackArgs &a);
cudaError_t launch_pack_batch(const PackArgs *d, const int64_t *prefix, int n, int64_t blocks,
                              cudaStream_t s);

struct Product {
  const int32_t *A;
  int64_t nA;
  const int32_t *B;
  int64_t nB;
  int64_t *C;  // nA + nB - 1 column sums, accumulated atomically (zero first)
};

cudaError_t launch_schoolbook(const Product *prods, int nprod, cudaStream_t s);

struct SchoolArgs {
  Product p[4];
  int nprod;
  int64_t block_prefix[5];
  int64_t ichunks[4];
};
int make_school_args(const Product *prods, int nprod, SchoolArgs &a);  // 0 on success
cudaError_t launch_schoolbook_batch(const SchoolArgs *d, const int64_t *prefix, int n,
                                    int64_t blocks, cudaStream_t s);

// Tensor-core engine (tcgen05, kind::f16): fp16 operand layouts, then the MMA kernel.
void tc_geometry(int64_t nA, int64_t nB, TcGeom &g);
size_t tc_operand_bytes(const TcGeom &g);
// also clears `nzero` column-sum words at `zero`
cudaError_t launch_tc_pack(const PackArgs &pa, const TcGeom &g, int nprod, char *base,
                           int64_t *zero, int64_t nzero, cudaStream_t s);
cudaError_t launch_tc_products(const TcGeom &g, int nprod, char *base,
                               int64_t *const *C, int *status, cudaStream_t s);
struct TcProduct {
  const __half *E;     // A windows: row h holds digits h - 127 .. h - 120
  int64_t nE;
  const __half *BRT;
  int64_t rows;
  int64_t dmax, R, T;  // largest delta, rows of B, tiles
  int64_t work;    // block offsets over all output tiles (the kernel's split unit)
  int64_t *C;
  int64_t ncols;
};

struct TcArgs {
  TcProduct p[4];
  int nprod;
  int64_t work_prefix[5];  // block offsets of the sub-products before each one
  int *status;
};

struct TcPackArgs {
  PackOp op[kMaxOperands];
  int nprod;
  int N, b, in_limbs, flip;
  uint64_t ninv;
  __half *E[4];
  __half *BRT[4];
  int64_t nE, rows, R, nA, nB;
  int64_t segA, segB;  // pack CTAs per A operand and per B operand
  int64_t *zero;       // column sums cleared by the same launch (nzero words), or null
  int64_t nzero;
};

void make_tc_pack_args(const PackArgs &pa, const TcGeom &g, int nprod, char *base,
                       TcPackArgs &a, int64_t &blocks, int64_t *zero = nullptr,
                       int64_t nzero = 0);
cudaError_t launch_tc_pack_batch(const TcPackArgs *d, const int64_t *prefix, int n,
                                 int64_t blocks, cudaStream_t s);
int64_t tc_work(const TcGeom &g);  // block offsets over the output tiles of one sub-product
void make_tc_args(const TcGeom &g, int nprod, char *base, int64_t *const *C, int *status,
                  TcArgs &a);
// The split of the tensor-core work (block offsets of all output tiles, in
// order) over the persistent CTAs, made on the host: CTA b takes positions
// [at[b], at[b + 1]), and its first work item lies in tile `tile[b]` of
// sub-product q[b] of descriptor desc[b].  A share that crosses into another
// tile pays for a second item (its own drain and reduction), so crossings
// are charged kTcSwitchCost offsets (measured: a second item costs about as
// much as two offsets once its descriptor is decoded ahead) and the split
// equalises that cost; a split point that falls inside a charge snaps to the
// tile's start.  n = 0: the kernel splits the offsets evenly itself.
constexpr int kTcMaxCtas = 160;
constexpr int64_t kTcSwitchCost = 2;
struct TcSplit {
  int n = 0;
  int64_t at[kTcMaxCtas + 1];
  int32_t desc[kTcMaxCtas];
  int32_t q[kTcMaxCtas];
  int32_t tile[kTcMaxCtas];  // tiles per sub-product are at most 2^20
};
// args: n descriptors (host copies) whose work starts at prefix[i]; grid CTAs
void tc_make_split(const TcArgs *args, const int64_t *prefix, int n, int grid, TcSplit &sp);
int tc_grid(int64_t work);  // CTAs of a launch over `work` offsets (one per SM at most)
// the prefix (in offsets) over the descriptors is split as `split` says
cudaError_t launch_tc_batch(const TcArgs *d, const int64_t *prefix, int n, int64_t work,
                            const TcSplit &split, cudaStream_t s);

// NTT engine: column sums of each product by a two-prime transform + CRT.
// Loads the transform's twiddle tables on the current device (once; 0 on
// success).  Every entry point calls it on its first call per device.
int ntt_init_tables();
size_t ntt_workspace_bytes(int log_n, int nprod);
cudaError_t launch_ntt_products(const Product *prods, int nprod, int log_n, int d,
                                void *scratch, cudaStream_t s);
// Sub-products of one transform length 2^log_n from a DEVICE array of
// descriptors (all squarings or none; at most kMaxNttBatch), their transform
// arrays at scratch (ntt_workspace_bytes(log_n, nprod)): one launch sequence.
constexpr int kMaxNttBatch = 4096;
cudaError_t launch_ntt_batch(const Product *dprods, int nprod, int64_t max_ncols, int square,
                             int log_n, void *scratch, cudaStream_t s);

struct NormJob {
  const int64_t *c1;
  int64_t n1;
  const int64_t *c2;  // may be null
  int64_t n2;
  int sigma;          // value = sum (c1_k + sigma c2_k) 2^(d k) + sum_i 2^(pstart + i pstride)
  uint32_t *out;
  uint32_t *flags;    // one flag word per scan tile; the jobs' arrays lie back to back
                      // from job 0's, and a tile counter follows the last (clear
                      // before the launch)
  // the shift of signed coefficients: one bit per coefficient read from this
  // value (K U(Y) with K = 2^kb); pcount = 0 for none
  int64_t pstart = 0, pstride = 1, pcount = 0;
};

// Normalizes up to 4 column-sum combinations into two's complement words:
// one launch while the tiles fit in about one wave (a tile takes its carry
// from its predecessors' flags), else a tile pass and a carry pass.
cudaError_t launch_normalize(const NormJob *jobs, int njobs, int d, int64_t nwords,
                             int64_t ntiles, int *status, cudaStream_t s);

struct NormArgs {
  NormJob job[4];
  int njobs;
  int paired;         // jobs (0,1) and (2,3) are +- pairs of the same columns
  int d;
  int64_t nwords;
  int64_t ntiles;
  int *status;        // a wait that gave up records 1 here
};
int make_norm_args(const NormJob *jobs, int njobs, int d, int64_t nwords, int64_t ntiles,
                   int *status, NormArgs &a);
int64_t norm_blocks(const NormArgs &a);        // CTAs of the tile pass
int64_t norm_carry_blocks(const NormArgs &a);  // CTAs of the carry pass (two-pass form)
// bytes of a product's flag region (the tiles' flags and the tile counter)
int64_t norm_flag_bytes(int njobs, int64_t ntiles);
// the launches for a whole batch, per digit width d (16 or 32): one (single
// pass) or two (tile pass, carry pass), by the number of tile CTAs
cudaError_t launch_normalize_batch(int d, const NormArgs *da, const int64_t *prefix_tiles,
                                   const int64_t *prefix_carry, int n, int64_t tile_blocks,
                                   int64_t carry_blocks, cudaStream_t s);
// scan tiles of a combination of nwords words at digit width d
int64_t norm_tiles_for(int64_t nwords, int d);

struct RecoverRun;
// The reconstruction runs of a plan over its normalized values (returns nruns),
// and its normalization jobs (which column sums combine, the shift pattern).
int plan_runs(const Plan &p, const uint32_t *words, RecoverRun *runs);
void plan_norm_jobs(const Plan &p, int64_t *cols, uint32_t *words, uint32_t *flags,
                    NormJob *jobs);

// KS1 / KS2 unpack: h'_k = bits [off + kN, off + kN + width) of V (k even) or
// V_odd (k odd).
// Signed coefficients arrive shifted by K = 2^kb (kb < 0: unsigned, no shift);
// the unpack subtracts it.
struct UnpackArgs {
  uint64_t *h;
  int ol;
  int64_t lh;
  const uint32_t *V;
  const uint32_t *V_odd;
  int64_t nwords, off, N;
  int width;
  int kb;
};
cudaError_t launch_unpack(const UnpackArgs &a, cudaStream_t s);
int64_t unpack_blocks(const UnpackArgs &a);
cudaError_t launch_unpack_batch(const UnpackArgs *d, const int64_t *prefix, int n,
                                int64_t blocks, cudaStream_t s);

// One run of the reconstruction of Sec. 3.2 (KS3: one run over h; KS4: one
// run over the even-index and one over the odd-index coefficients): the digit
// strings fwd = sum c_i X^i (Vf, from bit off_f) and rev = sum c_(n-1-i) X^i
// (Vr, from bit off_r) of its n coefficients, c_i = h'_(kbase + kstride i).
// The run is cut into chains of `chain` coefficients, chain c covering
// [c chain, (c + 1) chain): an odd chain runs upward from s = c chain, an even
// one downward from s = (c + 1) chain -- the same recurrence on the reversed
// problem x^(n-1) h(1/x), whose fwd is rev and whose rev is fwd -- so one exact
// pair (c_(s-1), c_s) at every s = chain (2j + 1) starts two chains.  An even
// chain whose s would reach n runs downward from n without seeds.  The pair
// j of this run is cluster j of the seed kernel, values slot_prev (c_(s-1))
// and slot_cur (c_s).
struct RecoverRun {
  const uint32_t *Vf;
  int64_t off_f;
  const uint32_t *Vr;
  int64_t off_r;
  int64_t n;               // coefficients in this run
  int64_t kbase, kstride;  // h index of run coefficient i: kbase + kstride * i
  int64_t nchains;         // ceil(n / chain)
  int slot_prev, slot_cur;
};
// Chain c of a run: its direction, start s, length, and whether it is seeded.
__host__ __device__ __forceinline__ void chain_geom(int64_t n, int64_t chain, int64_t c,
                                                    bool &up, int64_t &s, int64_t &len,
                                                    bool &seeded) {
  const int64_t lo = c * chain;
  const int64_t hi = lo + chain < n ? lo + chain : n;
  up = (c & 1) != 0;
  s = up ? lo : hi;
  len = hi - lo;
  seeded = up || hi <= n - 1;
}
// seed pairs of a run: every s = chain (2j + 1) <= n - 1
__host__ __device__ __forceinline__ int64_t run_pairs(int64_t n, int64_t chain) {
  return n - 1 >= chain ? (n - 1 - chain) / (2 * chain) + 1 : 0;
}

// Exact values h'_k (h_k + K for signed inputs, K = 2^kb) for the chain
// starts: ncl clusters of C consecutive k, cluster j starting at
// k0 = k00 + kstep j.  Value r of cluster j is value index j C + r.
struct SeedArgs {
  const uint64_t *f, *g;
  int64_t lf, lg;
  int bf, bg, ilf, ilg;  // coefficient bits and limbs of each operand
  int sgn;               // two's complement inputs
  int kb;                // K = 2^kb is added (sgn), else kb < 0
  int64_t k00, kstep, ncl;
  int C;
  int64_t slices;           // narrow path: windows of the t' axis (partials per value)
  int G;                    // narrow path: clusters per CTA (1, 2 or 4)
  int smem;                 // narrow path: dynamic shared memory of a CTA
  int P;                    // narrow path: balanced 8-bit digits per coefficient (2 .. 9)
  int64_t Z;                // narrow path: origin of the reversed g planes (Z = k00 mod 8)
  __half *planes;           // narrow path: the digit planes (fp16)
  // narrow path: per value six 64-bit column sums of its 32-bit words (value
  // v at acc + 6 v), zeroed by the digit-plane kernel
  unsigned long long *acc;
  uint32_t *seeds;          // wide path: seed_words words per value
  int seed_words;
  int *status;              // the product's status word (a bounded wait that gave up: 1)
};
struct SeedPlan {
  // 0 none; 10 P + C narrow (both operands <= 64 bits; P digits per
  // coefficient, clusters of C values); 100 + words: wide
  int kind = 0;
  SeedArgs a;
  int64_t blocks = 0, nvalues = 0;
  bool narrow() const { return kind >= 1 && kind < 100; }
};
// windows of the t' axis of the narrow seed kernel
int64_t seed_slices(int64_t lf, int64_t lg, int C);
int make_seed_plan(const uint64_t *f, int64_t lf, int bf, const uint64_t *g, int64_t lg, int bg,
                   int sgn, int kb, int64_t k00, int64_t kstep, int64_t ncl, int C,
                   unsigned long long *acc, uint32_t *seeds, int seed_words, __half *planes,
                   int *status, SeedPlan &sp);
// narrow seeds: digits per coefficient (-1: too wide), bytes of the digit
// planes, blocks of their kernel
int seed_digits(int bf, int bg, int sgn);
int64_t seed_planes_bytes(int64_t lf, int64_t lg, int P);
int64_t planes_blocks(const SeedArgs &a);
cudaError_t launch_seed_planes(const SeedArgs *d, const int64_t *prefix, int n, int64_t blocks,
                               cudaStream_t s);
// the digit planes of a narrow seed plan (before launch_seed_plan, same or
// earlier stream order), then the seed values themselves
cudaError_t launch_seed_planes_one(const SeedPlan &sp, cudaStream_t s);
cudaError_t launch_seed_plan(const SeedPlan &sp, cudaStream_t s);
// smem: the largest dynamic shared memory of the batch's CTAs (narrow kinds)
cudaError_t launch_seeds_batch(int kind, const SeedArgs *d, const int64_t *prefix, int n,
                               int64_t blocks, int smem, cudaStream_t s);
int seed_kind_index(int kind);  // 0 .. kSeedKinds - 1, or -1
constexpr int kSeedKinds = 16;  // ten narrow kinds, then wide classes of 2 .. 64 words
extern const int kSeedKindList[kSeedKinds];

struct RecoverArgs {
  RecoverRun run[2];
  int nruns;
  int64_t nwords;
  int M;
  int64_t chain;
  uint64_t *h;
  int ol;
  int kb;              // signed: subtract K = 2^kb from every coefficient
  int *status;
  // the exact seed values: value index (pair C + slot)
  int C;
  const unsigned long long *seed_acc;  // narrow seeds: six column sums per value
  const uint32_t *seeds;               // wide seeds: seed_words words per value
  int seed_words;
  int64_t rblocks[2];  // M <= 63: CTAs of cpc chains per run
  int smem;            // M <= 63: staged digit words of one CTA (bytes)
  int cpc;             // M <= 63: chains per CTA (a power of two, 8 .. 32)
};
int make_recover_args(uint64_t *h, int ol, int kb, const RecoverRun *runs, int nruns,
                      int64_t nwords, int M, int64_t chain, int C,
                      const unsigned long long *seed_acc, const uint32_t *seeds,
                      int seed_words, int *status, RecoverArgs &a, int64_t &blocks);
// 1 .. kRecoverClasses: the kernel that reconstructs digits of M bits on
// chains of the given length
int recover_class(int M, int64_t chain);
constexpr int kRecoverClasses = 6;
cudaError_t launch_recover(const RecoverArgs &a, int64_t blocks, cudaStream_t s);
// smem: the largest RecoverArgs::smem of the batch (class 1)
cudaError_t launch_recover_batch(int cls, const RecoverArgs *d, const int64_t *prefix, int n,
                                 int64_t blocks, int smem, cudaStream_t s);

// (Z/pZ)[x, y] by the substitutions of Sec. 2 (ks_biv.cu).
constexpr int kMaxBivEvals = 10;
struct BivEval {  // one evaluation of f or g at +-x^N or +-x^-N, or a part at i x^N
  const uint64_t *f;
  uint64_t *out;
  int64_t lx, ly, N, len;
  int reversed, alternate;
  uint64_t p;
  // 0: every row (sign -1 for odd rows if alternate); complex point y = i x^N:
  // 1 the real part (even rows i, sign (-1)^(i/2)), 2 the imaginary part (odd
  // rows, sign (-1)^((i-1)/2)), 3 their sum (every row, sign (-1)^floor(i/2))
  int part;
};
struct BivEvalArgs {
  BivEval e[kMaxBivEvals];
  int n;
};
struct BivReadArgs {  // KS_1 / KS_2 read-off of the rows of h
  uint64_t *h;
  const uint64_t *P1, *P2;
  int64_t lx, ly, N;
  uint64_t p;
};
struct BivSeq {  // P1, or (P1 + sign P2) / 2, read from index shift on
  const uint64_t *P1, *P2;
  int sign;
  int64_t shift, len;
};
struct BivRecoverArgs {  // KS_3 / KS_4 reciprocal recovery of n blocks
  uint64_t *h;
  BivSeq A, B;
  int64_t n, M, ell, lx, row0, rstep;
  uint64_t p;
};
cudaError_t launch_biv_eval(const BivEvalArgs &a, int64_t maxlen, cudaStream_t s);
cudaError_t launch_biv_readoff(const BivReadArgs &a, cudaStream_t s);
struct BivComplexArgs {  // KS_C read-off (Sec. 2.5) from the five products
  uint64_t *h;
  const uint64_t *P[5];
  int64_t lx, ly, M;
  uint64_t p;
};
cudaError_t launch_biv_readoff_complex(const BivComplexArgs &a, cudaStream_t s);
cudaError_t launch_biv_recover(const BivRecoverArgs &a, cudaStream_t s);

// (Z/pZ)[x]: out_k = h'_k mod p.
cudaError_t launch_reduce_mod(uint64_t *out, const uint64_t *h, int ol, int64_t lh,
                              uint64_t p, cudaStream_t s);

// ---------------------------------------------------------------- bulk copies
// Bulk copies into shared memory: one thread issues them on an mbarrier, all
// threads wait (bounded: about one second of %globaltimer).
__device__ __forceinline__ uint32_t smem_addr(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void stage_init(uint64_t *bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(bar)) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void stage_expect(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void stage_copy(void *dst, const void *src, uint32_t bytes,
                                           uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}
// wait for phase 0 of the barrier, about one second at most; false on timeout
__device__ __forceinline__ bool stage_wait(uint64_t *bar) {
  uint64_t t0;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
  for (;;) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar))
        : "memory");
    if (ok) return true;
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    if (t - t0 > 1000000000ull) return false;
  }
}

// ---------------------------------------------------------------- launches
// Programmatic dependent launch (ks_set_pdl; off by default).  With it on, the
// library's kernels are launched with the programmatic stream-serialization
// attribute: a kernel may be scheduled while the kernel before it in the
// stream is still running, so its launch latency hides behind that kernel's
// tail.  Every such kernel calls pdl_enter() before
// its first global memory access: it waits until the previous kernel has
// finished and its writes are visible (both read-after-write and
// write-after-read hazards stay covered), then lets the next kernel start
// launching.  For a kernel launched without the attribute both are no-ops.
__device__ __forceinline__ void pdl_enter() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
bool pdl_enabled();  // ks_set_pdl
template <typename... KArgs, typename... Args>
cudaError_t launch_k(void (*k)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                     Args... args) {
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = pdl_enabled() ? 1 : 0;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k, args...);
}

// ---------------------------------------------------------------- accounting
// Kernel launches issued by the library (host counter), and optional per-phase
// CUDA-event timing on the caller's stream.
void note_launches(int n);
enum Phase { PH_PACK = 0, PH_PRODUCT, PH_NORMALIZE, PH_UNPACK, PH_SEEDS, PH_RECOVER, PH_MOD,
             PH_COUNT };
struct PhaseTimer {
  cudaStream_t s;
  int phase;
  void *ev0;
  PhaseTimer(cudaStream_t s_, int phase_);
  ~PhaseTimer();
};

// ---------------------------------------------------------------- device helpers
// Status words hold the first failure a kernel recorded (0 = none): 1 a
// bounded wait gave up, 2 a reconstruction carry out of range, 3 an internal
// range check.  Writers use atomicCAS(status, 0, code), so a later failure
// that follows from the first (garbage in, range checks out) does not hide it.
// bits [pos, pos + 64) of a little-endian word array; words >= n read as 0.
__device__ __forceinline__ uint64_t get_bits64(const uint32_t *w, int64_t n, int64_t pos) {
  int64_t i = pos >> 5;
  int sh = (int)(pos & 31);
  uint64_t w0 = (i >= 0 && i < n) ? w[i] : 0u;
  uint64_t w1 = (i + 1 >= 0 && i + 1 < n) ? w[i + 1] : 0u;
  uint64_t w2 = (i + 2 >= 0 && i + 2 < n) ? w[i + 2] : 0u;
  uint64_t lo = w0 | (w1 << 32);
  if (sh == 0) return lo;
  return (lo >> sh) | (w2 << (64 - sh));
}

// Bits [x, x + len) (len <= 32, x >= 0) of a coefficient reduced to its low
// b bits, with bit b-1 flipped when `flip` (the signed bias of 2^(b-1)).
__device__ __forceinline__ uint32_t coeff_slice(const uint64_t *c, int in_limbs, int b,
                                                int flip, int x, int len) {
  if (x >= b) return 0u;
  int li = x >> 6, sh = x & 63;
  uint64_t lo = c[li];
  uint64_t hi = (li + 1 < in_limbs) ? c[li + 1] : 0ull;
  uint64_t v = sh ? ((lo >> sh) | (hi << (64 - sh))) : lo;
  int keep = b - x;
  if (keep < 64) v &= (1ull << keep) - 1ull;
  if (flip) {
    int fb = b - 1 - x;
    if (fb < 64) v ^= 1ull << fb;
  }
  return (uint32_t)(v & ((1ull << len) - 1ull));
}

// floor(x / N) for 0 <= x < 2^31 from m = floor(2^64 / N) + 1: with
// m = (2^64 + delta) / N, 1 <= delta <= N, x m / 2^64 exceeds x / N by less
// than 2^-33 < 1 / N, so the high word is the exact quotient (N = 1: x).
__device__ __forceinline__ int64_t div_by_n(int64_t x, int64_t N, uint64_t m) {
  return N == 1 ? x : (int64_t)__umul64hi((uint64_t)x, m);
}

// The fields t of the digits jlo .. jhi (inclusive): [t_lo, t_hi] (empty if
// t_hi < t_lo).
template <int D>
__device__ __forceinline__ void field_range(const PackOp &op, int64_t jlo, int64_t jhi,
                                            int64_t N, uint64_t ninv, int b, int64_t &t_lo,
                                            int64_t &t_hi) {
  const int64_t lo = jlo * D, hi = (jhi + 1) * D;
  if (op.narrow) {
    t_lo = lo - b < 0 ? 0 : div_by_n(lo - b, N, ninv) + 1;
    t_hi = hi - 1 < 0 ? -1 : div_by_n(hi - 1, N, ninv);
  } else {
    t_lo = lo - b < 0 ? 0 : (lo - b) / N + 1;
    t_hi = hi - 1 < 0 ? -1 : (hi - 1) / N;
  }
  if (t_hi > op.L - 1) t_hi = op.L - 1;
}

// Coefficients src0 .. src0 + n - 1 of an operand (n * in_limbs words) are
// copied to shared memory by the CTA when they fit in `cap` words; returns
// true (block-uniform) when they were.
__device__ __forceinline__ bool stage_coeffs(const PackOp &op, int64_t t_lo, int64_t t_hi,
                                             int in_limbs, uint64_t *sm, int cap,
                                             int64_t &src0) {
  const int64_t n = t_hi - t_lo + 1;
  src0 = op.reversed ? op.L - 1 - t_hi : t_lo;
  if (n <= 0 || n * in_limbs > cap) return false;
  const uint64_t *g = op.poly + src0 * in_limbs;
  const int words = (int)(n * in_limbs);
  // four loads in flight per thread (read-only path), then the stores
  for (int i0 = threadIdx.x; i0 < words; i0 += 4 * blockDim.x) {
    uint64_t r[4];
#pragma unroll
    for (int u = 0; u < 4; u++) {
      const int i = i0 + u * blockDim.x;
      r[u] = i < words ? __ldg(g + i) : 0ull;
    }
#pragma unroll
    for (int u = 0; u < 4; u++) {
      const int i = i0 + u * blockDim.x;
      if (i < words) sm[i] = r[u];
    }
  }
  return true;
}

// Limb i of a b-bit (biased) coefficient: the top limb is cut to the
// coefficient's bits (inputs are sign-extended) and, for signed inputs, has
// bit b-1 flipped (the bias 2^(b-1)); limbs past the top are zero.
__device__ __forceinline__ uint64_t coeff_limb(const uint64_t *c, int i, int in_limbs, int b,
                                               int flip) {
  if (i >= in_limbs) return 0ull;
  uint64_t v = c[i];
  if (i == in_limbs - 1) {
    const int top = b - 64 * i;  // 1 .. 64 bits in the top limb
    if (top < 64) v &= (1ull << top) - 1ull;
    if (flip) v ^= 1ull << (top - 1);
  }
  return v;
}

// Bits [x, x + 128) of a b-bit (biased) coefficient, as (lo, hi) 64-bit halves.
__device__ __forceinline__ void coeff_bits128(const uint64_t *c, int x, int in_limbs, int b,
                                              int flip, uint64_t &lo, uint64_t &hi) {
  const int li = x >> 6, sh = x & 63;
  const uint64_t w0 = coeff_limb(c, li, in_limbs, b, flip);
  const uint64_t w1 = coeff_limb(c, li + 1, in_limbs, b, flip);
  const uint64_t w2 = coeff_limb(c, li + 2, in_limbs, b, flip);
  lo = sh ? (w0 >> sh) | (w1 << (64 - sh)) : w0;
  hi = sh ? (w1 >> sh) | (w2 << (64 - sh)) : w1;
}

// Digits j0 .. j0 + K - 1 of one evaluation.  Digit j (bits [jd, jd + d)) is
// the sum over the coefficients t whose field [tN, tN + b) meets the window of
// +- their bits inside it, with the sign -1 for odd t at the point -2^N
// (Sec. 3.3, 3.4).  Signed coefficients (flip) are two's complement: bit
// b - 1 weighs -2^(b-1), so the evaluation is exact on the signed values
// themselves (the digits of a piece stay within +-(2^D - 1)).  One pair of divisions finds the coefficient fields that meet the K-digit
// window [lo, lo + K D); each field contributes the window's bits of its
// coefficient placed at its offset (one 128-bit extraction), which split
// into the K digits by compile-time shifts.
template <int D, int K>
__device__ __forceinline__ void digit_run(const PackOp &op, int64_t j0, int64_t N, uint64_t ninv,
                                          int b, int in_limbs, int flip, int32_t (&v)[K],
                                          const uint64_t *base = nullptr, int64_t src0 = 0) {
  static_assert(D * K <= 128, "window of at most 128 bits");
  constexpr int KD = D * K;
#pragma unroll
  for (int m = 0; m < K; m++) v[m] = 0;
  const int64_t lo = j0 * D;
  int64_t t_lo, t_hi;
  field_range<D>(op, j0, j0 + K - 1, N, ninv, b, t_lo, t_hi);
  for (int64_t t = t_lo; t <= t_hi; t++) {
    const int64_t src = op.reversed ? (op.L - 1 - t) : t;
    // the coefficient in global memory, or in the CTA's staged copy
    const uint64_t *c = base ? base + (src - src0) * in_limbs : op.poly + src * in_limbs;
    const bool neg = op.sigma < 0 && (t & 1);
    // the field overlaps the window: -b < off < K D
    const int off = (int)(t * N - lo);
    uint64_t wlo, whi;
    if (off >= 0) {
      coeff_bits128(c, 0, in_limbs, b, flip, wlo, whi);
      if (off >= 64) {
        whi = wlo << (off - 64);
        wlo = 0;
      } else if (off > 0) {
        whi = (whi << off) | (wlo >> (64 - off));
        wlo <<= off;
      }
    } else {
      coeff_bits128(c, -off, in_limbs, b, flip, wlo, whi);
    }
    if (KD < 64) {
      wlo &= (1ull << (KD % 64)) - 1ull;
      whi = 0;
    } else if (KD < 128) {
      whi &= (1ull << (KD % 64)) - 1ull;
    }
#pragma unroll
    for (int m = 0; m < K; m++) {
      const int sh = m * D;
      uint64_t bits;
      if (sh + D <= 64)
        bits = wlo >> sh;
      else if (sh >= 64)
        bits = whi >> (sh - 64);
      else
        bits = (wlo >> sh) | (whi << (64 - sh));
      const int32_t piece = (int32_t)(bits & ((1ull << D) - 1ull));
      v[m] += neg ? -piece : piece;
    }
    if (flip) {
      // signed input: the pieces above are those of c + 2^(b-1) (bit b-1
      // flipped); the field's top bit takes the bias back, with the field's sign
      const int top = off + b - 1;
#pragma unroll
      for (int m = 0; m < K; m++)
        if (top >= m * D && top < m * D + D) {
          const int32_t bias = (int32_t)1 << (top - m * D);
          v[m] += neg ? bias : -bias;
        }
    }
  }
}

}  // namespace ks
