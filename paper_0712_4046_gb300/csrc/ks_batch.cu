// Batched executor: many independent products (uneven lengths, bit sizes,
// variants and engines) in one launch sequence.
//
// ks_plan_create plans every product (variant and engine per the dispatch
// mode), carves one workspace for all of them, and scatters each product's
// kernel descriptors into per-kernel arrays in device memory together with
// the prefix sums of their block counts.  ks_plan_execute then issues one
// launch per phase for the whole batch -- pack, tensor-core operand layout,
// the INT32 and tensor-core products (the tensor-core kernel is persistent
// over the work items of every sub-product of every product, so the four
// sub-products of a four-point product are independent items), carry
// normalization, unpack, seeds and reconstruction per word-size class -- about
// a dozen launches whatever the batch size.
// Products routed to the transform engine (large ones) run their transform
// launches individually inside the same sequence.  The first execute on a
// stream captures the sequence into a CUDA graph; later executes replay it.
#include <mutex>
#include <stdlib.h>
#include <string.h>
#include <vector>

#include "ks_internal.cuh"
#include "ks_src.cuh"

namespace ks {

int *status_ptr();
cudaError_t alloc_device(void **p, size_t bytes);
int choose_mode(int64_t lf, int64_t lg, int b, int is_signed, int mode, int *variant,
                int *engine);
bool mlp_choose_batch(const ks_problem *probs, int64_t n, int *variants, int *engines);

struct ZeroArgs {
  uint64_t *p;
  int64_t n;  // 64-bit words
};

template <class Src>
__global__ void __launch_bounds__(256) zero_kernel(Src src) {
  pdl_enter();
  int64_t local;
  const ZeroArgs &a = src.locate(blockIdx.x, local);
  const int64_t i = local * 256 + threadIdx.x;
  if (i < a.n) a.p[i] = 0ull;
}

namespace {
size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// one per-kernel descriptor list: host vector + block counts, then uploaded
template <class T>
struct List {
  std::vector<T> v;
  std::vector<int64_t> prefix{0};
  T *d = nullptr;
  int64_t *dprefix = nullptr;
  void add(const T &x, int64_t blocks) {
    v.push_back(x);
    prefix.push_back(prefix.back() + blocks);
  }
  int n() const { return (int)v.size(); }
  int64_t blocks() const { return prefix.back(); }
  size_t bytes() const { return align256(v.size() * sizeof(T)) + align256(prefix.size() * 8); }
  void place(char *&hbase, char *&dbase) {
    d = reinterpret_cast<T *>(dbase);
    memcpy(hbase, v.data(), v.size() * sizeof(T));
    hbase += align256(v.size() * sizeof(T));
    dbase += align256(v.size() * sizeof(T));
    dprefix = reinterpret_cast<int64_t *>(dbase);
    memcpy(hbase, prefix.data(), prefix.size() * 8);
    hbase += align256(prefix.size() * 8);
    dbase += align256(prefix.size() * 8);
  }
};

// Transform sub-products of one length (and all squarings or none): one
// launch sequence for all of them, their arrays side by side in one scratch.
struct NttGroup {
  int log_n = 0, square = 0;
  std::vector<Product> prods;
  int64_t max_ncols = 0;
  int64_t first = 0;       // index of the first descriptor in the plan's list
  char *scratch = nullptr;
};
}  // namespace

}  // namespace ks

struct ks_plan {
  int64_t n = 0;
  std::vector<ks::Plan> plans;
  std::vector<ks_problem> probs;
  char *ws = nullptr;       // device workspace of all products
  size_t ws_bytes = 0;
  char *desc = nullptr;     // device descriptor arrays
  char *hdesc = nullptr;    // pinned host copy
  size_t desc_bytes = 0;
  ks::List<ks::ZeroArgs> zero;
  ks::List<ks::PackArgs> pack;
  ks::List<ks::TcPackArgs> tcpack;
  ks::List<ks::SchoolArgs> school;
  ks::List<ks::TcArgs> tc;
  ks::List<ks::NormArgs> norm[2];   // digit width 16 and 32 (tensor cores): tile pass
  ks::List<ks::NormArgs> normc[2];  // the same descriptors, carry-pass block counts
  ks::List<ks::UnpackArgs> unpack;
  ks::List<ks::SeedArgs> seeds[ks::kSeedKinds];  // per kernel kind (kSeedKindList)
  ks::List<ks::SeedArgs> planes;                  // the narrow seeds' digit planes
  int seed_smem[ks::kSeedKinds] = {0};            // per kind: the largest CTA's shared memory
  ks::List<ks::RecoverArgs> recover[ks::kRecoverClasses];
  int recover_smem[ks::kRecoverClasses] = {0};  // per class: the largest staged-digit buffer
  std::vector<ks::NttGroup> ntt;
  ks::List<ks::Product> nttd;  // the groups' descriptors, side by side
  char *ntt_scratch = nullptr;
  size_t ntt_bytes = 0;
  int64_t tc_work = 0;
  ks::TcSplit tc_split;  // the tensor-core work over the CTAs (made at creation)
  long long launches = 0;
  cudaGraphExec_t graph = nullptr;
  cudaStream_t graph_stream = nullptr;
  cudaStream_t last_stream = nullptr;  // where the last execute ran (ks_plan_status)
  int device = 0;
  int *status = nullptr;  // the plan's device status word (the first bytes of ws)
  // the seeds read only the inputs: they run on a helper stream, forked after
  // the products and joined before the reconstruction (in a captured graph: a
  // parallel branch)
  cudaStream_t side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
};

namespace ks {
namespace {
#define KS_TRY(call)                                  \
  do {                                                \
    cudaError_t e_ = (call);                          \
    if (e_ != cudaSuccess) return e_;                 \
  } while (0)

cudaError_t issue(ks_plan *P, cudaStream_t s) {
  // the seeds read only the inputs, on the helper stream: the digit planes
  // from the start (beside the packing), the seed contraction after the
  // products (which want every SM); joined before the reconstruction
  bool any_seeds = false;
  for (int i = 0; i < kSeedKinds; i++) any_seeds = any_seeds || P->seeds[i].n() > 0;
  const bool fork = P->side != nullptr && any_seeds;
  cudaStream_t side = fork ? P->side : s;
  if (fork) {
    KS_TRY(cudaEventRecord(P->ev_fork, s));
    KS_TRY(cudaStreamWaitEvent(side, P->ev_fork, 0));
  }
  if (P->planes.n())
    KS_TRY(launch_seed_planes(P->planes.d, P->planes.dprefix, P->planes.n(), P->planes.blocks(),
                              side));
  if (P->zero.n()) {
    (void)launch_k(zero_kernel<Many<ZeroArgs>>, dim3((unsigned)P->zero.blocks()), dim3(256), 0, s, 
        Many<ZeroArgs>{P->zero.d, P->zero.dprefix, P->zero.n()});
    note_launches(1);
    KS_TRY(cudaGetLastError());
  }
  if (P->pack.n())
    KS_TRY(launch_pack_batch(P->pack.d, P->pack.dprefix, P->pack.n(), P->pack.blocks(), s));
  if (P->tcpack.n())
    KS_TRY(launch_tc_pack_batch(P->tcpack.d, P->tcpack.dprefix, P->tcpack.n(),
                                P->tcpack.blocks(), s));
  if (P->school.n())
    KS_TRY(launch_schoolbook_batch(P->school.d, P->school.dprefix, P->school.n(),
                                   P->school.blocks(), s));
  if (P->tc.n())
    KS_TRY(launch_tc_batch(P->tc.d, P->tc.dprefix, P->tc.n(), P->tc_work, P->tc_split, s));
  for (auto &g : P->ntt)
    KS_TRY(launch_ntt_batch(P->nttd.d + g.first, (int)g.prods.size(), g.max_ncols, g.square,
                            g.log_n, g.scratch, s));
  if (fork) {
    KS_TRY(cudaEventRecord(P->ev_fork, s));
    KS_TRY(cudaStreamWaitEvent(side, P->ev_fork, 0));
  }
  for (int i = 0; i < kSeedKinds; i++)
    if (P->seeds[i].n())
      KS_TRY(launch_seeds_batch(kSeedKindList[i], P->seeds[i].d, P->seeds[i].dprefix,
                                P->seeds[i].n(), P->seeds[i].blocks(), P->seed_smem[i], side));
  if (fork) KS_TRY(cudaEventRecord(P->ev_join, side));
  for (int c = 0; c < 2; c++)
    if (P->norm[c].n())
      KS_TRY(launch_normalize_batch(c == 0 ? 16 : 32, P->norm[c].d, P->norm[c].dprefix,
                                    P->normc[c].dprefix, P->norm[c].n(), P->norm[c].blocks(),
                                    P->normc[c].blocks(), s));
  if (P->unpack.n())
    KS_TRY(launch_unpack_batch(P->unpack.d, P->unpack.dprefix, P->unpack.n(),
                               P->unpack.blocks(), s));
  if (fork) KS_TRY(cudaStreamWaitEvent(s, P->ev_join, 0));
  for (int c = 0; c < kRecoverClasses; c++)
    if (P->recover[c].n())
      KS_TRY(launch_recover_batch(c + 1, P->recover[c].d, P->recover[c].dprefix,
                                  P->recover[c].n(), P->recover[c].blocks(), P->recover_smem[c], s));
  return cudaSuccess;
}
}  // namespace

// Fills the descriptor lists of one product (same launches as the single path).
static int add_product(ks_plan *P, const Plan &p, const ks_problem &q, char *ws, int *status) {
  int32_t *dig = reinterpret_cast<int32_t *>(ws + p.off_digits);
  int64_t *cols = reinterpret_cast<int64_t *>(ws + p.off_cols);
  uint32_t *words = reinterpret_cast<uint32_t *>(ws + p.off_words);
  uint32_t *flags = reinterpret_cast<uint32_t *>(ws + p.off_flags);
  // the column sums accumulate from zero; the tile flags start clear
  const int64_t nzero = p.zero_words;
  uint32_t *seeds = reinterpret_cast<uint32_t *>(ws + p.off_seeds);
  static const int kRev[5][4] = {{0}, {0}, {0, 0}, {0, 1}, {0, 0, 1, 1}};
  static const int kSig[5][4] = {{1}, {1}, {1, -1}, {1, 1}, {1, -1, 1, -1}};
  PackArgs pa{};
  pa.nops = 2 * p.nprod;
  pa.N = p.N;
  pa.b = p.b;
  pa.d = p.d;
  pa.in_limbs = p.in_limbs;
  pa.flip = p.is_signed;
  Product prods[4];
  for (int k = 0; k < p.nprod; k++) {
    // operands padded to multiples of four digits: every one 16-byte aligned
    int32_t *A = dig + (int64_t)k * (((p.nA + 3) & ~(int64_t)3) + ((p.nB + 3) & ~(int64_t)3));
    int32_t *B = A + ((p.nA + 3) & ~(int64_t)3);
    pa.op[2 * k] =
        PackOp{q.f, p.lf, kRev[p.variant][k], kSig[p.variant][k], A, p.nA, p.bf, p.ilf};
    pa.op[2 * k + 1] =
        PackOp{q.g, p.lg, kRev[p.variant][k], kSig[p.variant][k], B, p.nB, p.bg, p.ilg};
    prods[k] = Product{A, p.nA, B, p.nB, cols + (int64_t)k * p.ncols};
  }
  // squaring (f = g, equal lengths and sizes): the int32-digit engines pack every
  // evaluation once and multiply its digits by themselves
  if (q.f == q.g && p.lf == p.lg && p.bf == p.bg && p.engine != KS_ENGINE_TC)
    squaring_pack(pa, prods, p.nprod);
  pack_finish(pa);
  if (p.engine == KS_ENGINE_TC) {
    TcPackArgs ta;
    int64_t blocks;
    // the packing kernel also zeroes the column sums the products accumulate into
    make_tc_pack_args(pa, p.tg, p.nprod, ws + p.off_digits, ta, blocks, cols, nzero);
    P->tcpack.add(ta, blocks);
  } else {
    P->pack.add(pa, pack_blocks(pa));
    if (p.engine == KS_ENGINE_SCHOOLBOOK) {
      SchoolArgs sa;
      if (make_school_args(prods, p.nprod, sa) != 0) return KS_EINVAL;
      P->school.add(sa, sa.block_prefix[p.nprod]);
      P->zero.add(ZeroArgs{reinterpret_cast<uint64_t *>(cols), nzero}, (nzero + 255) / 256);
    } else {
      // the transform writes every column sum; only the tile flags need clearing
      P->zero.add(ZeroArgs{reinterpret_cast<uint64_t *>(flags), (p.flag_bytes + 7) / 8},
                  (p.flag_bytes / 8 + 255) / 256);
      // into the last group of this length and kind that has room
      const int square = (prods[0].A == prods[0].B) ? 1 : 0;
      NttGroup *g = nullptr;
      for (auto it = P->ntt.rbegin(); it != P->ntt.rend(); ++it)
        if (it->log_n == p.ntt_log && it->square == square &&
            (int64_t)it->prods.size() + p.nprod <= kMaxNttBatch) {
          g = &*it;
          break;
        }
      if (g == nullptr) {
        P->ntt.emplace_back();
        g = &P->ntt.back();
        g->log_n = p.ntt_log;
        g->square = square;
      }
      for (int k = 0; k < p.nprod; k++) g->prods.push_back(prods[k]);
      if (p.ncols > g->max_ncols) g->max_ncols = p.ncols;
    }
  }
  NormJob jobs[4];
  plan_norm_jobs(p, cols, words, flags, jobs);
  NormArgs na;
  if (make_norm_args(jobs, p.nnorm, p.dn, p.nwords, p.ntiles, status, na) != 0)
    return KS_EINVAL;
  P->norm[p.dn == 32 ? 1 : 0].add(na, norm_blocks(na));
  P->normc[p.dn == 32 ? 1 : 0].add(na, norm_carry_blocks(na));
  const uint32_t *V0 = words, *V1 = words + p.nwords;
  const int ol = p.out_limbs;
  if (p.variant == KS_1 || p.variant == KS_2) {
    UnpackArgs ua = p.variant == KS_1
                        ? UnpackArgs{q.h, ol, p.lh, V0, nullptr, p.nwords, 0, p.N, p.N, p.kb}
                        : UnpackArgs{q.h, ol, p.lh, V0, V1, p.nwords, 1, p.N, 2 * p.N, p.kb};
    P->unpack.add(ua, unpack_blocks(ua));
  } else {
    RecoverRun runs[2];
    plan_runs(p, words, runs);
    unsigned long long *acc = reinterpret_cast<unsigned long long *>(ws + p.off_seedacc);
    SeedPlan sp;
    if (make_seed_plan(q.f, p.lf, p.bf, q.g, p.lg, p.bg, p.is_signed, p.kb, p.k00, p.kstep, p.ncl,
                       p.C, acc, seeds, p.seed_words,
                       reinterpret_cast<__half *>(ws + p.off_planes), status, sp) != 0)
      return KS_ERANGE;
    if (sp.kind != 0) {
      const int i = seed_kind_index(sp.kind);
      if (i < 0) return KS_ERANGE;
      P->seeds[i].add(sp.a, sp.blocks);
      if (sp.narrow()) {
        P->planes.add(sp.a, planes_blocks(sp.a));
        if (sp.a.smem > P->seed_smem[i]) P->seed_smem[i] = sp.a.smem;
      }
    }
    RecoverArgs ra;
    int64_t blocks;
    if (make_recover_args(q.h, ol, p.kb, runs, p.nruns, p.nwords, p.M, p.chain, p.C,
                          sp.narrow() ? acc : nullptr, seeds, p.seed_words, status,
                          ra, blocks) != 0)
      return KS_ERANGE;
    const int rc = recover_class(p.M, p.chain) - 1;
    P->recover[rc].add(ra, blocks);
    if (ra.smem > P->recover_smem[rc]) P->recover_smem[rc] = ra.smem;
  }
  return KS_OK;
}

}  // namespace ks

using namespace ks;

extern "C" {

int ks_plan_create(ks_plan **out, const ks_problem *probs, int64_t n, int dispatch_mode) {
  if (out == nullptr || n < 0 || (n > 0 && probs == nullptr)) return KS_EINVAL;
  *out = nullptr;
  ks_plan *P = new (std::nothrow) ks_plan();
  if (P == nullptr) return KS_ENOMEM;
  // the transform's tables are loaded here, before any capture of the plan
  if (cudaGetDevice(&P->device) != cudaSuccess || ntt_init_tables() != 0) {
    delete P;
    return KS_ECUDA;
  }
  P->n = n;
  P->plans.resize(n);
  P->probs.assign(probs, probs + n);
  std::vector<size_t> offs(n);
  size_t total = 0;
  // the learned model, where installed and allowed, chooses for the whole batch at once
  std::vector<int> mv(n, 0), me(n, 0);
  const bool learned = (dispatch_mode == KS_DISPATCH_MLP || dispatch_mode == KS_DISPATCH_AUTO) &&
                       n > 0 && mlp_choose_batch(probs, n, mv.data(), me.data());
  for (int64_t i = 0; i < n; i++) {
    const ks_problem &q = probs[i];
    if (!q.h || !q.f || !q.g) {
      delete P;
      return KS_EINVAL;
    }
    int v = learned ? mv[i] : q.variant, e = learned ? me[i] : q.engine;
    const int bg = problem_bits_g(q);
    int rc = q.coeff_bits_g < 0 ? KS_EINVAL : KS_OK;
    if (rc == KS_OK)
      rc = choose_mode(q.len_f, q.len_g, problem_bits(q), q.is_signed, dispatch_mode, &v, &e);
    if (rc == KS_OK)
      rc = make_plan(P->plans[i], q.len_f, q.len_g, q.coeff_bits, q.is_signed, v, e, bg);
    // unequal sizes: an engine chosen for the equal size may exceed its limits
    if (rc != KS_OK && bg != q.coeff_bits && q.engine == KS_ENGINE_AUTO && e != KS_ENGINE_NTT)
      rc = make_plan(P->plans[i], q.len_f, q.len_g, q.coeff_bits, q.is_signed, v, KS_ENGINE_NTT,
                     bg);
    if (rc != KS_OK) {
      delete P;
      return rc;
    }
    offs[i] = total;
    // a transform product's scratch lives with its group's (below)
    const Plan &pi = P->plans[i];
    total += align256(pi.engine == KS_ENGINE_NTT ? pi.off_ntt : pi.total);
  }
  if (cudaStreamCreateWithFlags(&P->side, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&P->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&P->ev_join, cudaEventDisableTiming) != cudaSuccess) {
    ks_plan_destroy(P);
    return KS_ECUDA;
  }
  // the plan's status word, then every product's workspace
  P->ws_bytes = 256 + total;
  if (alloc_device(reinterpret_cast<void **>(&P->ws), P->ws_bytes) != cudaSuccess) {
    P->ws = nullptr;
    ks_plan_destroy(P);
    return KS_ENOMEM;
  }
  P->status = reinterpret_cast<int *>(P->ws);
  if (cudaMemset(P->status, 0, 256) != cudaSuccess) {
    ks_plan_destroy(P);
    return KS_ECUDA;
  }
  int *status = P->status;
  for (int64_t i = 0; i < n; i++) {
    const Plan &p = P->plans[i];
    char *ws = P->ws + 256 + offs[i];
    int rc = add_product(P, p, probs[i], ws, status);
    if (rc == KS_OK && p.engine == KS_ENGINE_TC) {
      TcArgs ta;
      int64_t *C[4];
      for (int k = 0; k < p.nprod; k++)
        C[k] = reinterpret_cast<int64_t *>(ws + p.off_cols) + (int64_t)k * p.ncols;
      make_tc_args(p.tg, p.nprod, ws + p.off_digits, C, status, ta);
      P->tc.add(ta, ta.work_prefix[p.nprod]);
    }
    if (rc != KS_OK) {
      ks_plan_destroy(P);
      return rc;
    }
  }
  P->tc_work = P->tc.blocks();
  if (P->tc.n() > 0)
    tc_make_split(P->tc.v.data(), P->tc.prefix.data(), P->tc.n(), tc_grid(P->tc_work),
                  P->tc_split);
  // the transform groups: one scratch allocation, descriptors in the list
  size_t &ntt_bytes = P->ntt_bytes;
  for (auto &g : P->ntt) {
    g.first = P->nttd.n();
    for (const Product &x : g.prods) P->nttd.add(x, 0);
    ntt_bytes += align256(ntt_workspace_bytes(g.log_n, (int)g.prods.size()));
  }
  if (ntt_bytes > 0) {
    if (alloc_device(reinterpret_cast<void **>(&P->ntt_scratch), ntt_bytes) != cudaSuccess) {
      P->ntt_scratch = nullptr;
      ks_plan_destroy(P);
      return KS_ENOMEM;
    }
    char *at = P->ntt_scratch;
    for (auto &g : P->ntt) {
      g.scratch = at;
      at += align256(ntt_workspace_bytes(g.log_n, (int)g.prods.size()));
    }
  }
  // descriptor arrays: one device allocation, filled from a pinned host copy
  size_t db = P->zero.bytes() + P->pack.bytes() + P->tcpack.bytes() + P->school.bytes() +
              P->tc.bytes() + P->norm[0].bytes() + P->norm[1].bytes() + P->normc[0].bytes() +
              P->normc[1].bytes() + P->unpack.bytes() +
              0;
  for (int i = 0; i < kSeedKinds; i++) db += P->seeds[i].bytes();
  db += P->planes.bytes();
  db += P->nttd.bytes();
  for (int c = 0; c < kRecoverClasses; c++) db += P->recover[c].bytes();
  P->desc_bytes = db;
  if (alloc_device(reinterpret_cast<void **>(&P->desc), db) != cudaSuccess ||
      cudaMallocHost(&P->hdesc, db) != cudaSuccess) {
    ks_plan_destroy(P);
    return KS_ENOMEM;
  }
  char *h = P->hdesc, *d = P->desc;
  P->zero.place(h, d);
  P->pack.place(h, d);
  P->tcpack.place(h, d);
  P->school.place(h, d);
  P->tc.place(h, d);
  for (int c = 0; c < 2; c++) {
    P->norm[c].place(h, d);
    P->normc[c].place(h, d);
    P->normc[c].d = P->norm[c].d;  // both lists describe the same jobs
  }
  P->unpack.place(h, d);
  for (int i = 0; i < kSeedKinds; i++) P->seeds[i].place(h, d);
  P->planes.place(h, d);
  P->nttd.place(h, d);
  for (int c = 0; c < kRecoverClasses; c++) P->recover[c].place(h, d);
  if (cudaMemcpy(P->desc, P->hdesc, db, cudaMemcpyHostToDevice) != cudaSuccess) {
    ks_plan_destroy(P);
    return KS_ECUDA;
  }
  *out = P;
  return KS_OK;
}

int ks_plan_execute(ks_plan *P, ks_stream_t stream) {
  if (P == nullptr) return KS_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev != P->device) return KS_EINVAL;
  const long long before = ks_launch_count();
  P->last_stream = s;
  if (P->graph != nullptr && P->graph_stream == s) {
    if (cudaGraphLaunch(P->graph, s) != cudaSuccess) return KS_ECUDA;
    return KS_OK;
  }
  cudaError_t e = issue(P, s);
  if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? KS_ENOMEM : KS_ECUDA;
  P->launches = ks_launch_count() - before;
  return KS_OK;
}

int ks_plan_capture(ks_plan *P, ks_stream_t stream) {
  if (P == nullptr) return KS_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (s == nullptr) return KS_EINVAL;  // the legacy stream cannot be captured
  if (P->graph != nullptr) {
    cudaGraphExecDestroy(P->graph);
    P->graph = nullptr;
  }
  // kernels with large shared memory and the transform tables are set up
  // by one plain execution first
  int rc = ks_plan_execute(P, stream);
  if (rc != KS_OK) return rc;
  if (cudaStreamSynchronize(s) != cudaSuccess) return KS_ECUDA;
  cudaGraph_t g = nullptr;
  if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return KS_ECUDA;
  cudaError_t e = issue(P, s);
  cudaError_t e2 = cudaStreamEndCapture(s, &g);
  if (e != cudaSuccess || e2 != cudaSuccess || g == nullptr) {
    if (g) cudaGraphDestroy(g);
    return KS_ECUDA;
  }
  e = cudaGraphInstantiate(&P->graph, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    P->graph = nullptr;
    return KS_ECUDA;
  }
  P->graph_stream = s;
  return KS_OK;
}

int ks_plan_status(ks_plan *P) {
  if (P == nullptr || P->status == nullptr) return KS_EINVAL;
  int cur = 0;
  if (cudaGetDevice(&cur) != cudaSuccess) return KS_ECUDA;
  if (cur != P->device && cudaSetDevice(P->device) != cudaSuccess) return KS_ECUDA;
  int rc = KS_OK, v = 0;
  cudaStream_t s = P->last_stream;
  if (cudaStreamSynchronize(s) != cudaSuccess ||
      cudaMemcpyAsync(&v, P->status, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess) {
    rc = KS_ECUDA;
  } else if (v != 0) {
    rc = v == 1 ? KS_ETIMEOUT : KS_ERANGE;
    if (cudaMemsetAsync(P->status, 0, sizeof(int), s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      rc = KS_ECUDA;
  }
  if (cur != P->device) cudaSetDevice(cur);
  return rc;
}

long long ks_plan_launches(const ks_plan *P) { return P ? P->launches : -1; }

int64_t ks_plan_workspace_bytes(const ks_plan *P) {
  return P ? (int64_t)(P->ws_bytes + P->ntt_bytes + P->desc_bytes) : -1;
}

int ks_plan_choice(const ks_plan *P, int64_t i, int *variant, int *engine) {
  if (P == nullptr || i < 0 || i >= P->n || !variant || !engine) return KS_EINVAL;
  *variant = P->plans[i].variant;
  *engine = P->plans[i].engine;
  return KS_OK;
}

void ks_plan_destroy(ks_plan *P) {
  if (P == nullptr) return;
  int cur = 0;
  cudaGetDevice(&cur);
  cudaSetDevice(P->device);
  cudaDeviceSynchronize();
  if (P->graph) cudaGraphExecDestroy(P->graph);
  if (P->ws) cudaFree(P->ws);
  if (P->ntt_scratch) cudaFree(P->ntt_scratch);
  if (P->desc) cudaFree(P->desc);
  if (P->hdesc) cudaFreeHost(P->hdesc);
  if (P->ev_fork) cudaEventDestroy(P->ev_fork);
  if (P->ev_join) cudaEventDestroy(P->ev_join);
  if (P->side) cudaStreamDestroy(P->side);
  cudaSetDevice(cur);
  delete P;
}

}  // extern "C"
