// C ABI of libhmgb300 (see include/hmgb300.h): context, H-matrix build, H-LU, solve,
// matvec, standalone rounded truncation, and the host-only structure export.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <memory>
#include <stdexcept>
#include <string>
#include <thread>
#include <vector>

#include "../../include/hmgb300.h"
#include "kernels.h"
#include "plan.h"
#include "structure.h"

using namespace hm;

namespace {

thread_local std::string g_err;
// rounded additions not touched by the next wave overlap it on a side stream (hm_set_overlap)
std::atomic<int> g_overlap{1};
// host threads of task-graph construction and planning (0: all hardware threads)
std::atomic<int> g_host_threads{0};

int fail(int code, const std::string& msg) {
  g_err = msg;
  return code;
}

struct Buf {
  void* p = nullptr;
  size_t bytes = 0;
};

}  // namespace

struct hm_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  hm_alloc_fn af = nullptr;
  hm_free_fn ff = nullptr;
  void* user = nullptr;
  bool profiling = false;
  // side stream of the deferred rounded additions and its events (created on first use)
  bool side_ready = false;
  cudaStream_t side = nullptr;
  cudaEvent_t main_done[2] = {nullptr, nullptr}, side_done[2] = {nullptr, nullptr};
  ~hm_ctx() {
    if (!side_ready) return;
    cudaStreamDestroy(side);
    for (int q = 0; q < 2; ++q) {
      cudaEventDestroy(main_done[q]);
      cudaEventDestroy(side_done[q]);
    }
  }
};

namespace {

bool dalloc(hm_ctx* c, Buf& b, size_t bytes) {
  b.bytes = bytes < 256 ? 256 : bytes;
  if (c->af) {
    b.p = c->af(b.bytes, c->user);
  } else {
    if (cudaMalloc(&b.p, b.bytes) != cudaSuccess) b.p = nullptr;
  }
  if (!b.p) b.bytes = 0;
  return b.p != nullptr;
}

void dfree(hm_ctx* c, Buf& b) {
  if (!b.p) return;
  if (c->ff) c->ff(b.p, b.bytes, c->user);
  else cudaFree(b.p);
  b.p = nullptr;
  b.bytes = 0;
}

#define CU(call)                                                                            \
  do {                                                                                      \
    cudaError_t e_ = (call);                                                                \
    if (e_ != cudaSuccess) return fail(HM_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

struct DevPlan {
  Plan host;
  Buf ops[NKIND];
  Buf entries;
  bool uploaded = false;
  double eps = -1.0;
  int precision = -1;
  double gemm_work = -1.0;   // GEMM split target the plan was built with
  int overlap = -1;          // deferred rounded additions on a side stream (plan built with)
  int accumulate = -1;       // accumulator H-LU (plan built with)
  double plan_seconds = 0.0;
  // replay state of solve / matvec plans: persistent scratch and the captured CUDA graph
  Buf sd, si, cnt;
  cudaGraphExec_t exec = nullptr;
};

size_t op_size(int kind) {
  switch (kind) {
    case K_GETRF: return sizeof(GetrfOp);
    case K_TRSM: return sizeof(TrsmOp);
    case K_GEMM:
    case K_GEMM32:
    case K_GEMM_TC: return sizeof(GemmOp);
    case K_COPY: return sizeof(CopyOp);
    case K_STACK:
    case K_CORE: return sizeof(TruncOp);
    case K_EVAL: return sizeof(EvalOp);
    default: return sizeof(AcaOp);
  }
}

template <class V>
int upload_vec(hm_ctx* c, Buf& b, const V& v) {
  if (v.empty()) return HM_OK;
  const size_t bytes = v.size() * sizeof(*v.data());
  if (!dalloc(c, b, bytes)) return fail(HM_ENOMEM, "allocator returned NULL (plan upload)");
  CU(cudaMemcpyAsync(b.p, v.data(), bytes, cudaMemcpyHostToDevice, c->stream));
  return HM_OK;
}

void free_ops(hm_ctx* c, DevPlan& dp) {
  for (int k = 0; k < NKIND; ++k) dfree(c, dp.ops[k]);
  dfree(c, dp.entries);
}

// micro-op arrays to the device; on a failure nothing stays allocated (a later call retries)
int upload(hm_ctx* c, DevPlan& dp) {
  if (dp.uploaded) return HM_OK;
  int rc = HM_OK;
  if (!rc) rc = upload_vec(c, dp.ops[K_GETRF], dp.host.getrf);
  if (!rc) rc = upload_vec(c, dp.ops[K_TRSM], dp.host.trsm);
  if (!rc) rc = upload_vec(c, dp.ops[K_GEMM], dp.host.gemm);
  if (!rc) rc = upload_vec(c, dp.ops[K_COPY], dp.host.copy);
  if (!rc) rc = upload_vec(c, dp.ops[K_STACK], dp.host.trunc);
  if (!rc) rc = upload_vec(c, dp.ops[K_EVAL], dp.host.eval);
  if (!rc) rc = upload_vec(c, dp.ops[K_ACA], dp.host.aca);
  if (!rc) rc = upload_vec(c, dp.entries, dp.host.entries);
  if (!rc) {
    const cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e) rc = fail(HM_ECUDA, std::string("plan upload: ") + cudaGetErrorString(e));
  }
  if (rc) {
    free_ops(c, dp);
    return rc;
  }
  dp.uploaded = true;
  return HM_OK;
}

void free_plan(hm_ctx* c, DevPlan& dp) {
  free_ops(c, dp);
  dfree(c, dp.sd);
  dfree(c, dp.si);
  dfree(c, dp.cnt);
  if (dp.exec) cudaGraphExecDestroy(dp.exec);
  dp.exec = nullptr;
  dp.uploaded = false;
}

struct Profile {
  double ms[NKIND] = {0};
  int64_t launches[NKIND] = {0};
};

bool ensure_side(hm_ctx* c) {
  if (c->side_ready) return true;
  bool ok = cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking) == cudaSuccess;
  for (int q = 0; q < 2 && ok; ++q)
    ok = cudaEventCreateWithFlags(&c->main_done[q], cudaEventDisableTiming) == cudaSuccess &&
         cudaEventCreateWithFlags(&c->side_done[q], cudaEventDisableTiming) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    return false;
  }
  c->side_ready = true;
  return true;
}

// A plan with side launches (deferred rounded additions): wave w's side launches run on the side
// stream after an event that marks the end of w's other launches, and overlap wave w + 1 (which
// does not touch their targets, and works in the other scratch space); wave w + 2 waits for them
// before it reuses their scratch. Without profiling only; a profiled run is sequential.
int run_plan_overlapped(hm_ctx* c, DevPlan& dp, const Bases& B, double h, cudaStream_t stream) {
  const std::vector<Launch>& Ls = dp.host.launches;
  bool pending[2] = {false, false};
  int cur = -1;
  for (size_t i = 0; i < Ls.size(); ++i) {
    const Launch& L = Ls[i];
    const int par = L.wave & 1;
    if (!L.side && L.wave != cur) {
      cur = L.wave;
      if (pending[par]) {   // wave - 2's side launches used this scratch space
        CU(cudaStreamWaitEvent(stream, c->side_done[par], 0));
        pending[par] = false;
      }
    }
    cudaStream_t st = stream;
    if (L.side) {
      if (i == 0 || !Ls[i - 1].side || Ls[i - 1].wave != L.wave) {
        CU(cudaEventRecord(c->main_done[par], stream));
        CU(cudaStreamWaitEvent(c->side, c->main_done[par], 0));
      }
      st = c->side;
    }
    const int buf = L.kind == K_CORE ? K_STACK : ((L.kind == K_GEMM_TC || L.kind == K_GEMM32) ? K_GEMM : L.kind);
    const void* ops = (const char*)dp.ops[buf].p + (size_t)L.begin * op_size(L.kind);
    cudaError_t e = launch_kind(L.kind, ops, L.count, (const StackEntry*)dp.entries.p, B, h, st, L.gy, L.gz);
    if (e != cudaSuccess) return fail(HM_ECUDA, std::string("kernel launch: ") + cudaGetErrorString(e));
    if (L.side && (i + 1 == Ls.size() || !Ls[i + 1].side || Ls[i + 1].wave != L.wave)) {
      CU(cudaEventRecord(c->side_done[par], c->side));
      pending[par] = true;
    }
  }
  for (int q = 0; q < 2; ++q)
    if (pending[q]) CU(cudaStreamWaitEvent(stream, c->side_done[q], 0));
  return HM_OK;
}

int run_plan(hm_ctx* c, DevPlan& dp, const Bases& B, double h, Profile* prof, cudaStream_t stream_override = nullptr,
             bool use_override = false) {
  const cudaStream_t stream = use_override ? stream_override : c->stream;
  if (!prof && dp.host.deferred_truncations > 0 && ensure_side(c)) return run_plan_overlapped(c, dp, B, h, stream);
  std::vector<cudaEvent_t> ev;
  std::vector<int> evkind;
  // with the launch log on, the kind's FLOP counter is copied after every launch (pinned host
  // buffer, asynchronous), so that the log carries each launch's FLOPs
  const char* log_path = prof ? std::getenv("HMGB300_LAUNCH_LOG") : nullptr;
  unsigned long long* fl_host = nullptr;
  if (log_path && cudaMallocHost(&fl_host, (dp.host.launches.size() + 1) * sizeof(unsigned long long)) != cudaSuccess)
    fl_host = nullptr;
  size_t li = 0;
  for (const Launch& L : dp.host.launches) {
    const int buf = L.kind == K_CORE ? K_STACK : ((L.kind == K_GEMM_TC || L.kind == K_GEMM32) ? K_GEMM : L.kind);
    const char* base = (const char*)dp.ops[buf].p;
    const void* ops = base + (size_t)L.begin * op_size(L.kind);
    if (prof) {
      cudaEvent_t a, b;
      cudaEventCreate(&a);
      cudaEventCreate(&b);
      cudaEventRecord(a, stream);
      ev.push_back(a);
      ev.push_back(b);
      evkind.push_back(L.kind);
    }
    cudaError_t e = launch_kind(L.kind, ops, L.count, (const StackEntry*)dp.entries.p, B, h, stream, L.gy, L.gz);
    if (e != cudaSuccess) {
      if (fl_host) cudaFreeHost(fl_host);
      return fail(HM_ECUDA, std::string("kernel launch: ") + cudaGetErrorString(e));
    }
    if (prof) cudaEventRecord(ev.back(), stream);
    if (fl_host)
      cudaMemcpyAsync(fl_host + li, B.flops + NFC + L.kind, sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                      stream);
    ++li;
  }
  if (prof) {
    CU(cudaStreamSynchronize(stream));
    // HMGB300_LAUNCH_LOG=<file>: one CSV line per launch of a profiled run (kind, micro-ops,
    // grid y/z, ms and, for GEMM launches, the largest static m n k with 'd' marking a
    // dimension that has a dynamic part)
    FILE* log = log_path ? std::fopen(log_path, "a") : nullptr;
    if (log) std::fprintf(log, "kind,count,gy,gz,ms,flops,m,n,k\n");
    unsigned long long prev[NKIND] = {0};
    for (size_t q = 0; q < evkind.size(); ++q) {
      float ms = 0.f;
      cudaEventElapsedTime(&ms, ev[2 * q], ev[2 * q + 1]);
      prof->ms[evkind[q]] += ms;
      prof->launches[evkind[q]] += 1;
      cudaEventDestroy(ev[2 * q]);
      cudaEventDestroy(ev[2 * q + 1]);
      if (log) {
        const Launch& L = dp.host.launches[q];
        std::string dims = ",,,";
        if (L.kind == K_GEMM) {
          double wmax = -1.0;
          for (int i = L.begin; i < L.begin + L.count; ++i) {
            const GemmOp& o = dp.host.gemm[i];
            const double w = (o.m + (o.md ? 16.0 : 0.0)) * (o.n + (o.nd ? 16.0 : 0.0)) * (o.k + (o.kd ? 16.0 : 0.0));
            if (w > wmax) {
              wmax = w;
              dims = "," + std::to_string(o.m) + (o.md ? "d" : "") + "," + std::to_string(o.n) + (o.nd ? "d" : "") +
                     "," + std::to_string(o.k) + (o.kd ? "d" : "");
            }
          }
        }
        unsigned long long f = 0;
        if (fl_host) {
          f = fl_host[q] - prev[L.kind];
          prev[L.kind] = fl_host[q];
        }
        std::fprintf(log, "%d,%d,%d,%d,%.4f,%llu%s\n", L.kind, L.count, L.gy, L.gz, ms, f, dims.c_str());
      }
    }
    if (log) std::fclose(log);
  }
  if (fl_host) cudaFreeHost(fl_host);
  return HM_OK;
}

}  // namespace

struct hm_matrix {
  hm_ctx* ctx = nullptr;
  int64_t n = 0;
  hm_build_opts opts{};
  double h = 0.0;
  ClusterTree ct;
  BlockTree bt;
  Layout lay;
  Buf perm, pts, pts_orig, vals, ranks;
  TaskGraph dag;
  bool dag_built = false;
  DevPlan lu_plan;
  DevPlan mv_plan;
  Buf mv_work;
  double build_seconds = 0.0;
  int64_t aca_unconverged = 0;
  // host preparation of the H-LU started by hm_build (task graph and plan at the matrix's eps,
  // FP64, the current overlap and GEMM settings) while the device assembles the matrix; every
  // reader of dag / lu_plan joins it first
  std::thread prep;
};

// One allocation of factor values, ranks and pivots shared by the factors of a batch
// (hm_lu_batch); freed with the last of them.
struct SharedArena {
  Buf vals, ranks, piv;
  int refs = 0;
};

struct hm_factor {
  hm_ctx* ctx = nullptr;
  hm_matrix* A = nullptr;
  double eps = 0.0;
  Buf vals, ranks, piv;     // own buffers, or views into `arena`
  SharedArena* arena = nullptr;
  DevPlan solve_plan;
  DevPlan mv_plan;
  Buf work;   // SP_X buffer of the solve / matvec plans
  hm_stats st{};
};

namespace {

constexpr int SOLVE_CHUNK = 32;

// task graph and H-LU plan of A for the defaults of hm_lu (the matrix's eps, FP64, no
// accumulators), on the host; on any failure nothing is kept and hm_lu plans (and reports) itself
void prep_lu(hm_matrix* A, int ov) {
  try {
    build_task_graph(A->ct, A->bt, A->dag, false, g_host_threads.load());
    if (!compute_levels(A->dag)) return;
    A->dag_built = true;
    auto t0 = std::chrono::steady_clock::now();
    plan_lu(A->ct, A->bt, A->lay, A->dag, A->opts.eps, A->lu_plan.host, g_host_threads.load(), HM_PREC_FP64,
            ov != 0, false);
    A->lu_plan.plan_seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    A->lu_plan.eps = A->opts.eps;
    A->lu_plan.precision = HM_PREC_FP64;
    A->lu_plan.gemm_work = gemm_min_work();
    A->lu_plan.overlap = ov;
    A->lu_plan.accumulate = 0;
  } catch (...) {
    A->lu_plan.host = Plan();
    A->lu_plan.eps = -1.0;
  }
}

void prep_join(const hm_matrix* A) {
  hm_matrix* M = const_cast<hm_matrix*>(A);
  if (M->prep.joinable()) M->prep.join();
}

void fill_matrix_stats(const hm_matrix* A, hm_stats* s) {
  prep_join(A);
  std::memset(s, 0, sizeof(*s));
  s->n = A->n;
  s->nclusters = (int64_t)A->ct.cl.size();
  for (const Cluster& c : A->ct.cl) s->nleaf_clusters += c.leaf() ? 1 : 0;
  s->depth = A->ct.depth;
  for (const LeafStore& L : A->lay.leaf) {
    if (L.lr) s->nleaves_lowrank++;
    else s->nleaves_dense++;
  }
  s->value_bytes = A->lay.nvalues * 8;
  s->h = A->h;
  s->eps = A->opts.eps;
  s->rank_cap = A->opts.rank_cap;
  s->dag_nodes = (int64_t)A->dag.nodes.size();
  s->dag_edges = (int64_t)A->dag.edges.size();
  s->dag_levels = A->dag.nlevels;
  s->dag_seconds = A->dag.build_seconds;
  s->plan_launches = (int64_t)A->lu_plan.host.launches.size();
  s->plan_phases = A->lu_plan.host.nphases;
  s->plan_truncations = A->lu_plan.host.ntrunc;
  s->scratch_bytes = (A->lu_plan.host.scratch_doubles * 8 + A->lu_plan.host.scratch_ints * 4) *
                     (A->lu_plan.host.two_scratch ? 2 : 1);
  s->plan_deferred = A->lu_plan.host.deferred_truncations;
  s->accumulate = A->lu_plan.accumulate > 0 ? 1 : 0;
  s->arena_bytes = A->lu_plan.host.arena_doubles * 8;
  s->accumulated_pieces = A->lu_plan.host.accumulated_pieces;
  s->plan_seconds = A->lu_plan.plan_seconds;
  s->seconds = A->build_seconds;
  s->aca_unconverged = A->aca_unconverged;
}

int read_ranks(hm_ctx* c, const Buf& ranks, int nr, int64_t* maxr, int64_t* sumr) {
  std::vector<int> r(nr);
  if (nr) CU(cudaMemcpyAsync(r.data(), ranks.p, nr * sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  CU(cudaStreamSynchronize(c->stream));
  *maxr = 0;
  *sumr = 0;
  for (int v : r) {
    *maxr = std::max<int64_t>(*maxr, v);
    *sumr += v;
  }
  return HM_OK;
}

constexpr int NCOUNT = NFC + NKIND;

constexpr int NSTATUS = 8;

struct Counters {
  Buf b;   // NCOUNT unsigned long long + NSTATUS ints
  unsigned long long* flops() { return (unsigned long long*)b.p; }
  int* status() { return (int*)((char*)b.p + NCOUNT * sizeof(unsigned long long)); }
};

int counters_init(hm_ctx* c, Counters& k) {
  if (!dalloc(c, k.b, NCOUNT * sizeof(unsigned long long) + NSTATUS * sizeof(int)))
    return fail(HM_ENOMEM, "allocator returned NULL (counters)");
  CU(cudaMemsetAsync(k.b.p, 0, NCOUNT * sizeof(unsigned long long) + NSTATUS * sizeof(int), c->stream));
  return HM_OK;
}

int counters_read(hm_ctx* c, Counters& k, unsigned long long* fl, int* st) {
  CU(cudaMemcpyAsync(fl, k.b.p, NCOUNT * sizeof(unsigned long long), cudaMemcpyDeviceToHost, c->stream));
  CU(cudaMemcpyAsync(st, k.status(), NSTATUS * sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  CU(cudaStreamSynchronize(c->stream));
  return HM_OK;
}

// per-kernel-kind device time, launches and flops: kinds 0..7 in the kind arrays, the tensor-core
// GEMM kind in its own fields
void fill_kind_stats(hm_stats* st, const Profile& prof, const unsigned long long* fl) {
  for (int q = 0; q < 8; ++q) {
    st->kind_ms[q] = prof.ms[q];
    st->kind_launches[q] = prof.launches[q];
    st->kind_flops[q] = (double)fl[NFC + q];
  }
  st->tc_ms = prof.ms[K_GEMM_TC];
  st->tc_launches = prof.launches[K_GEMM_TC];
  st->tc_flops = (double)fl[NFC + K_GEMM_TC];
  st->f32_ms = prof.ms[K_GEMM32];
  st->f32_launches = prof.launches[K_GEMM32];
  st->f32_flops = (double)fl[NFC + K_GEMM32];
}

Bases make_bases() {
  Bases B;
  std::memset(&B, 0, sizeof(B));
  B.gemm_work = (float)gemm_min_work();
  return B;
}

}  // namespace

// ====================================================================================== ABI
extern "C" {

const char* hm_last_error(void) { return g_err.c_str(); }

int hm_ctx_create(int device, void* stream, hm_alloc_fn af, hm_free_fn ff, void* user, hm_ctx** out) {
  if (!out) return fail(HM_EINVAL, "hm_ctx_create: out is NULL");
  if ((af == nullptr) != (ff == nullptr)) return fail(HM_EINVAL, "hm_ctx_create: give both allocator callbacks or none");
  int ndev = 0;
  cudaError_t e = cudaGetDeviceCount(&ndev);
  if (e != cudaSuccess || ndev <= 0) return fail(HM_ECUDA, "hm_ctx_create: no CUDA device available");
  if (device < 0 || device >= ndev) return fail(HM_EINVAL, "hm_ctx_create: bad device ordinal");
  CU(cudaSetDevice(device));
  hm_ctx* c = new hm_ctx();
  c->device = device;
  c->stream = (cudaStream_t)stream;
  c->af = af;
  c->ff = ff;
  c->user = user;
  *out = c;
  return HM_OK;
}

void hm_ctx_destroy(hm_ctx* c) { delete c; }

int hm_ctx_set_profiling(hm_ctx* c, int enable) {
  if (!c) return fail(HM_EINVAL, "hm_ctx_set_profiling: NULL context");
  c->profiling = enable != 0;
  return HM_OK;
}

// ------------------------------------------------------------------------------ build
int hm_build(hm_ctx* c, const double* pts, int64_t n, const hm_build_opts* o, hm_matrix** out) {
  if (!c || !pts || !out) return fail(HM_EINVAL, "hm_build: NULL argument");
  if (n < 1 || n > (int64_t)1 << 30) return fail(HM_EINVAL, "hm_build: n out of range");
  hm_build_opts opts{64, 2.0, 1e-6, 64, -1.0, 0};
  if (o) opts = *o;
  if (opts.leaf_size < 1 || opts.leaf_size > 64) return fail(HM_EINVAL, "hm_build: leaf_size must be in 1..64");
  if (!(opts.eta >= 0.0)) return fail(HM_EINVAL, "hm_build: eta must be >= 0");
  if (!(opts.eps >= HM_EPS_MIN) || opts.eps >= 1.0)
    return fail(HM_EINVAL, "hm_build: eps must be in [HM_EPS_MIN, 1) (HM_EPS_MIN = 1e-8, the truncation's floor)");
  if (opts.rank_cap < 1 || opts.rank_cap > 64) return fail(HM_EINVAL, "hm_build: rank_cap must be in 1..64");
  CU(cudaSetDevice(c->device));
  auto A = std::make_unique<hm_matrix>();
  A->ctx = c;
  A->n = n;
  A->opts = opts;
  try {
    build_cluster_tree(pts, n, opts.leaf_size, A->ct);
    build_block_tree(A->ct, opts.eta, A->bt);
    build_layout(A->ct, A->bt, opts.rank_cap, A->lay);
  } catch (const std::exception& ex) {
    return fail(HM_EINTERNAL, std::string("hm_build: ") + ex.what());
  }
  auto cleanup = [&](int rc) {
    prep_join(A.get());
    dfree(c, A->perm);
    dfree(c, A->pts);
    dfree(c, A->pts_orig);
    dfree(c, A->vals);
    dfree(c, A->ranks);
    return rc;
  };
  if (!dalloc(c, A->perm, n * sizeof(int64_t)) || !dalloc(c, A->pts, n * 3 * sizeof(double)) ||
      !dalloc(c, A->pts_orig, n * 3 * sizeof(double)) || !dalloc(c, A->vals, A->lay.nvalues * sizeof(double)) ||
      !dalloc(c, A->ranks, std::max(1, A->lay.nranks) * sizeof(int)))
    return cleanup(fail(HM_ENOMEM, "hm_build: allocator returned NULL"));
  // the H-LU's host preparation needs only the trees and the layout: it runs beside the assembly
  if (opts.prepare_lu) {
    try {
      A->prep = std::thread(prep_lu, A.get(), g_overlap.load());
    } catch (...) {
      // no thread: hm_lu plans itself
    }
  }
  cudaStream_t s = c->stream;
  int rc = HM_OK;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  do {
    if (cudaMemcpyAsync(A->perm.p, A->ct.perm.data(), n * sizeof(int64_t), cudaMemcpyHostToDevice, s) ||
        cudaMemcpyAsync(A->pts_orig.p, pts, n * 3 * sizeof(double), cudaMemcpyHostToDevice, s) ||
        cudaMemsetAsync(A->ranks.p, 0, std::max(1, A->lay.nranks) * sizeof(int), s)) {
      rc = fail(HM_ECUDA, "hm_build: copy of the inputs failed");
      break;
    }
    cudaEventRecord(e0, s);
    if (launch_permute_points((double*)A->pts_orig.p, (int64_t*)A->perm.p, (int)n, (double*)A->pts.p, s)) {
      rc = fail(HM_ECUDA, "hm_build: permute kernel failed");
      break;
    }
    // h = mean nearest-neighbour distance (deterministic host sum of device minima)
    if (opts.kernel_h > 0.0) {
      A->h = opts.kernel_h;
    } else if (n == 1) {
      A->h = 1.0;
    } else {
      Buf nn;
      if (!dalloc(c, nn, n * sizeof(double))) {
        rc = fail(HM_ENOMEM, "hm_build: allocator returned NULL");
        break;
      }
      std::vector<double> d2(n);
      cudaError_t e = launch_nn2((double*)A->pts_orig.p, (int)n, (double*)nn.p, s);
      if (!e) e = cudaMemcpyAsync(d2.data(), nn.p, n * sizeof(double), cudaMemcpyDeviceToHost, s);
      if (!e) e = cudaStreamSynchronize(s);
      dfree(c, nn);
      if (e) {
        rc = fail(HM_ECUDA, std::string("hm_build: nearest-neighbour kernel: ") + cudaGetErrorString(e));
        break;
      }
      double sum = 0.0;
      for (int64_t i = 0; i < n; ++i) sum += std::sqrt(d2[i]);
      A->h = sum / (double)n;
      if (!(A->h > 0.0)) A->h = 1.0;
    }
    // dense leaves by evaluation; admissible leaves by ACA + rounded truncation
    DevPlan dp;
    try {
      plan_build(A->ct, A->bt, A->lay, opts.eps, 160, (int64_t)1 << 28, dp.host);
    } catch (const std::exception& ex) {
      rc = fail(HM_EINTERNAL, std::string("hm_build: ") + ex.what());
      break;
    }
    if ((rc = upload(c, dp)) != HM_OK) {
      free_plan(c, dp);
      break;
    }
    Buf sd, si;
    Counters k;
    if (!dalloc(c, sd, std::max<int64_t>(1, dp.host.scratch_doubles) * 8) ||
        !dalloc(c, si, std::max<int64_t>(1, dp.host.scratch_ints) * 4)) {
      dfree(c, sd);
      free_plan(c, dp);
      rc = fail(HM_ENOMEM, "hm_build: allocator returned NULL (scratch)");
      break;
    }
    if ((rc = counters_init(c, k)) != HM_OK) {
      dfree(c, sd);
      dfree(c, si);
      free_plan(c, dp);
      break;
    }
    Bases B = make_bases();
    B.d[SP_A] = (double*)A->vals.p;
    B.d[SP_S] = (double*)sd.p;
    B.d[SP_P] = (double*)A->pts.p;
    B.i[IS_ARANK] = (int*)A->ranks.p;
    B.i[IS_S] = (int*)si.p;
    B.flops = k.flops();
    B.status = k.status();
    rc = run_plan(c, dp, B, A->h, nullptr);
    unsigned long long fl[NCOUNT];
    int st[NSTATUS];
    if (rc == HM_OK) rc = counters_read(c, k, fl, st);
    cudaEventRecord(e1, s);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    A->build_seconds = ms * 1e-3;
    if (rc == HM_OK) A->aca_unconverged = st[2];
    dfree(c, sd);
    dfree(c, si);
    dfree(c, k.b);
    free_plan(c, dp);
  } while (false);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != HM_OK) return cleanup(rc);
  *out = A.release();
  return HM_OK;
}

void hm_matrix_free(hm_matrix* A) {
  if (!A) return;
  prep_join(A);
  hm_ctx* c = A->ctx;
  free_plan(c, A->lu_plan);
  free_plan(c, A->mv_plan);
  dfree(c, A->mv_work);
  dfree(c, A->perm);
  dfree(c, A->pts);
  dfree(c, A->pts_orig);
  dfree(c, A->vals);
  dfree(c, A->ranks);
  delete A;
}

// ------------------------------------------------------------------------------ H-LU
int hm_lu(hm_ctx* c, hm_matrix* A, const hm_lu_opts* o, hm_factor** out) {
  if (!c || !A || !out) return fail(HM_EINVAL, "hm_lu: NULL argument");
  double eps = (o && o->eps > 0.0) ? o->eps : A->opts.eps;
  if (!(eps >= HM_EPS_MIN) || eps >= 1.0) return fail(HM_EINVAL, "hm_lu: eps must be in [HM_EPS_MIN, 1)");
  const int precision = o ? o->precision : HM_PREC_FP64;
  if (precision != HM_PREC_FP64 && precision != HM_PREC_MIXED && precision != HM_PREC_MIXED_TC)
    return fail(HM_EINVAL, "hm_lu: precision must be HM_PREC_FP64, HM_PREC_MIXED or HM_PREC_MIXED_TC");
  const int accumulate = o ? o->accumulate : 0;
  if (accumulate != 0 && accumulate != 1) return fail(HM_EINVAL, "hm_lu: accumulate must be 0 or 1");
  prep_join(A);
  CU(cudaSetDevice(c->device));
  try {
    if (!A->dag_built) {
      build_task_graph(A->ct, A->bt, A->dag, false, g_host_threads.load());
      if (!compute_levels(A->dag)) return fail(HM_EINTERNAL, "hm_lu: task graph has a cycle");
      A->dag_built = true;
    }
    const int ov = g_overlap.load();
    if (A->lu_plan.eps != eps || A->lu_plan.precision != precision || A->lu_plan.gemm_work != gemm_min_work() ||
        A->lu_plan.overlap != ov || A->lu_plan.accumulate != accumulate) {
      free_plan(c, A->lu_plan);
      auto t0 = std::chrono::steady_clock::now();
      plan_lu(A->ct, A->bt, A->lay, A->dag, eps, A->lu_plan.host, g_host_threads.load(), precision, ov != 0,
              accumulate != 0);
      A->lu_plan.plan_seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
      A->lu_plan.eps = eps;
      A->lu_plan.precision = precision;
      A->lu_plan.gemm_work = gemm_min_work();
      A->lu_plan.overlap = ov;
      A->lu_plan.accumulate = accumulate;
    }
  } catch (const std::exception& ex) {
    return fail(HM_EINTERNAL, std::string("hm_lu: ") + ex.what());
  }
  int rc = upload(c, A->lu_plan);
  if (rc) return rc;
  auto F = std::make_unique<hm_factor>();
  F->ctx = c;
  F->A = A;
  F->eps = eps;
  Buf sd, si, sd2, si2, acc;
  Counters k;
  auto cleanup = [&](int r) {
    dfree(c, sd);
    dfree(c, si);
    dfree(c, sd2);
    dfree(c, si2);
    dfree(c, acc);
    dfree(c, k.b);
    dfree(c, F->vals);
    dfree(c, F->ranks);
    dfree(c, F->piv);
    return r;
  };
  const Plan& P = A->lu_plan.host;
  if (!dalloc(c, F->vals, A->lay.nvalues * 8) || !dalloc(c, F->ranks, std::max(1, A->lay.nranks) * 4) ||
      !dalloc(c, F->piv, std::max<int64_t>(1, A->lay.npiv) * 4) ||
      !dalloc(c, sd, std::max<int64_t>(1, P.scratch_doubles) * 8) ||
      !dalloc(c, si, std::max<int64_t>(1, P.scratch_ints) * 4) ||
      (P.two_scratch && (!dalloc(c, sd2, std::max<int64_t>(1, P.scratch_doubles) * 8) ||
                         !dalloc(c, si2, std::max<int64_t>(1, P.scratch_ints) * 4))) ||
      (P.arena_doubles > 0 && !dalloc(c, acc, P.arena_doubles * 8)))
    return cleanup(fail(HM_ENOMEM, "hm_lu: allocator returned NULL"));
  if ((rc = counters_init(c, k))) return cleanup(rc);
  cudaStream_t s = c->stream;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaEventRecord(e0, s);
  cudaError_t ce = cudaMemcpyAsync(F->vals.p, A->vals.p, A->lay.nvalues * 8, cudaMemcpyDeviceToDevice, s);
  if (!ce) ce = cudaMemcpyAsync(F->ranks.p, A->ranks.p, std::max(1, A->lay.nranks) * 4, cudaMemcpyDeviceToDevice, s);
  if (ce) {
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return cleanup(fail(HM_ECUDA, std::string("hm_lu: copy of A: ") + cudaGetErrorString(ce)));
  }
  Bases B = make_bases();
  B.d[SP_F] = (double*)F->vals.p;
  B.d[SP_S] = (double*)sd.p;
  B.d[SP_S2] = (double*)sd2.p;
  B.d[SP_ACC] = (double*)acc.p;
  B.d[SP_A] = (double*)A->vals.p;
  B.d[SP_P] = (double*)A->pts.p;
  B.i[IS_RANK] = (int*)F->ranks.p;
  B.i[IS_PIV] = (int*)F->piv.p;
  B.i[IS_S] = (int*)si.p;
  B.i[IS_S2] = (int*)si2.p;
  B.i[IS_ARANK] = (int*)A->ranks.p;
  B.flops = k.flops();
  B.status = k.status();
  Profile prof;
  rc = run_plan(c, A->lu_plan, B, A->h, c->profiling ? &prof : nullptr);
  cudaEventRecord(e1, s);
  cudaError_t se = cudaEventSynchronize(e1);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc) return cleanup(rc);
  if (se) return cleanup(fail(HM_ECUDA, std::string("hm_lu: ") + cudaGetErrorString(se)));
  unsigned long long fl[NCOUNT];
  int st[NSTATUS];
  if ((rc = counters_read(c, k, fl, st))) return cleanup(rc);
  fill_matrix_stats(A, &F->st);
  F->st.eps = eps;
  F->st.seconds = ms * 1e-3;
  for (int q = 0; q < 5; ++q) F->st.flops[q] = (double)fl[q];
  F->st.singular_pivots = st[0];
  F->st.rank_cap_hits = st[1];
  F->st.row_interchanges = st[3];
  F->st.precision = precision;
  fill_kind_stats(&F->st, prof, fl);
  F->st.launches = (int64_t)P.launches.size();
  if (st[4] > 0) {
    hm_factor_free(F.release());
    dfree(c, sd);
    dfree(c, si);
    dfree(c, k.b);
    return fail(HM_ETIMEOUT, "hm_lu: a bounded device wait gave up (tensor-core MMA completion)");
  }
  if ((rc = read_ranks(c, F->ranks, A->lay.nranks, &F->st.max_rank, &F->st.sum_rank))) return cleanup(rc);
  dfree(c, sd);
  dfree(c, si);
  dfree(c, sd2);
  dfree(c, si2);
  dfree(c, acc);
  dfree(c, k.b);
  hm_factor* f = F.release();
  *out = f;
  if (st[0] > 0) return fail(HM_ESINGULAR, "hm_lu: zero pivot in a diagonal leaf");
  return HM_OK;
}

void hm_factor_free(hm_factor* F) {
  if (!F) return;
  hm_ctx* c = F->ctx;
  free_plan(c, F->solve_plan);
  free_plan(c, F->mv_plan);
  dfree(c, F->work);
  if (F->arena) {
    if (--F->arena->refs == 0) {
      dfree(c, F->arena->vals);
      dfree(c, F->arena->ranks);
      dfree(c, F->arena->piv);
      delete F->arena;
    }
  } else {
    dfree(c, F->vals);
    dfree(c, F->ranks);
    dfree(c, F->piv);
  }
  delete F;
}

int hm_lu_batch(hm_ctx* c, hm_matrix* const* A, int count, const hm_lu_opts* o, hm_factor** out) {
  if (!c || !A || !out || count < 1) return fail(HM_EINVAL, "hm_lu_batch: bad argument");
  for (int i = 0; i < count; ++i) {
    if (!A[i]) return fail(HM_EINVAL, "hm_lu_batch: NULL matrix");
    out[i] = nullptr;
  }
  for (int i = 0; i < count; ++i) prep_join(A[i]);
  const int precision = o ? o->precision : HM_PREC_FP64;
  if (precision != HM_PREC_FP64 && precision != HM_PREC_MIXED && precision != HM_PREC_MIXED_TC)
    return fail(HM_EINVAL, "hm_lu_batch: precision must be HM_PREC_FP64, HM_PREC_MIXED or HM_PREC_MIXED_TC");
  if (o && o->accumulate) return fail(HM_EINVAL, "hm_lu_batch: the accumulator H-LU is not batched");
  const bool given = o && o->eps > 0.0;
  const double eps = given ? o->eps : A[0]->opts.eps;
  if (!(eps >= HM_EPS_MIN) || eps >= 1.0) return fail(HM_EINVAL, "hm_lu_batch: eps must be in [HM_EPS_MIN, 1)");
  for (int i = 0; i < count; ++i)
    if (!given && A[i]->opts.eps != eps)
      return fail(HM_EINVAL, "hm_lu_batch: matrices of different eps need opts->eps");
  CU(cudaSetDevice(c->device));
  try {
    for (int i = 0; i < count; ++i)
      if (!A[i]->dag_built) {
        build_task_graph(A[i]->ct, A[i]->bt, A[i]->dag, false, g_host_threads.load());
        if (!compute_levels(A[i]->dag)) return fail(HM_EINTERNAL, "hm_lu_batch: task graph has a cycle");
        A[i]->dag_built = true;
      }
  } catch (const std::exception& ex) {
    return fail(HM_EINTERNAL, std::string("hm_lu_batch: ") + ex.what());
  }
  size_t free_b = 0, total_b = 0;
  CU(cudaMemGetInfo(&free_b, &total_b));
  const double budget = 0.85 * (double)free_b;
  std::vector<hm_factor*> made;
  auto abort_all = [&](int rc) {
    for (hm_factor* f : made) hm_factor_free(f);
    for (int i = 0; i < count; ++i) out[i] = nullptr;
    return rc;
  };
  int singular = 0;
  for (int i0 = 0; i0 < count;) {
    // the next group: as many of the remaining instances as fit the device-memory budget
    int i1 = count;
    DevPlan dp;
    std::vector<int64_t> bd, br, bp;
    for (;;) {
      std::vector<LuInstance> inst;
      bd.assign(1, 0);
      br.assign(1, 0);
      bp.assign(1, 0);
      for (int i = i0; i < i1; ++i) {
        inst.push_back({&A[i]->ct, &A[i]->bt, &A[i]->lay, &A[i]->dag, bd.back(), br.back(), bp.back()});
        bd.push_back(bd.back() + (A[i]->lay.nvalues + 31) / 32 * 32);
        br.push_back(br.back() + A[i]->lay.nranks);
        bp.push_back(bp.back() + A[i]->lay.npiv);
      }
      try {
        const auto tp = std::chrono::steady_clock::now();
        plan_lu_batch(inst, eps, dp.host, g_host_threads.load(), precision);
        dp.plan_seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - tp).count();
      } catch (const std::exception& ex) {
        return abort_all(fail(HM_EINTERNAL, std::string("hm_lu_batch: ") + ex.what()));
      }
      const Plan& P = dp.host;
      const double ops = (double)P.gemm.size() * sizeof(GemmOp) + (double)P.trunc.size() * sizeof(TruncOp) +
                         (double)P.entries.size() * sizeof(StackEntry) + (double)P.copy.size() * sizeof(CopyOp) +
                         (double)P.trsm.size() * sizeof(TrsmOp) + (double)P.getrf.size() * sizeof(GetrfOp);
      const double need = 8.0 * bd.back() + 4.0 * (br.back() + bp.back()) + 8.0 * P.scratch_doubles +
                          4.0 * P.scratch_ints + ops;
      if (need <= budget || i1 - i0 == 1) break;
      i1 = i0 + (i1 - i0 + 1) / 2;
    }
    int rc = upload(c, dp);
    if (rc) {
      free_plan(c, dp);
      return abort_all(rc);
    }
    SharedArena* ar = new SharedArena;
    Buf sd, si;
    Counters k;
    auto cleanup = [&](int r) {
      free_plan(c, dp);
      dfree(c, sd);
      dfree(c, si);
      dfree(c, k.b);
      if (ar->refs == 0) {
        dfree(c, ar->vals);
        dfree(c, ar->ranks);
        dfree(c, ar->piv);
        delete ar;
      }
      return abort_all(r);
    };
    const Plan& P = dp.host;
    if (!dalloc(c, ar->vals, (size_t)bd.back() * 8) || !dalloc(c, ar->ranks, std::max<int64_t>(1, br.back()) * 4) ||
        !dalloc(c, ar->piv, std::max<int64_t>(1, bp.back()) * 4) ||
        !dalloc(c, sd, std::max<int64_t>(1, P.scratch_doubles) * 8) ||
        !dalloc(c, si, std::max<int64_t>(1, P.scratch_ints) * 4))
      return cleanup(fail(HM_ENOMEM, "hm_lu_batch: allocator returned NULL"));
    if ((rc = counters_init(c, k))) return cleanup(rc);
    cudaStream_t s = c->stream;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, s);
    cudaError_t ce = cudaSuccess;
    for (int i = i0; i < i1 && !ce; ++i) {
      const int q = i - i0;
      ce = cudaMemcpyAsync((char*)ar->vals.p + 8 * bd[q], A[i]->vals.p, A[i]->lay.nvalues * 8,
                           cudaMemcpyDeviceToDevice, s);
      if (!ce && A[i]->lay.nranks)
        ce = cudaMemcpyAsync((char*)ar->ranks.p + 4 * br[q], A[i]->ranks.p, A[i]->lay.nranks * 4,
                             cudaMemcpyDeviceToDevice, s);
    }
    if (ce) {
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      return cleanup(fail(HM_ECUDA, std::string("hm_lu_batch: copy of A: ") + cudaGetErrorString(ce)));
    }
    Bases B = make_bases();
    B.d[SP_F] = (double*)ar->vals.p;
    B.d[SP_S] = (double*)sd.p;
    B.i[IS_RANK] = (int*)ar->ranks.p;
    B.i[IS_PIV] = (int*)ar->piv.p;
    B.i[IS_S] = (int*)si.p;
    B.flops = k.flops();
    B.status = k.status();
    rc = run_plan(c, dp, B, 0.0, nullptr);
    cudaEventRecord(e1, s);
    cudaError_t se = cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return cleanup(rc);
    if (se) return cleanup(fail(HM_ECUDA, std::string("hm_lu_batch: ") + cudaGetErrorString(se)));
    unsigned long long fl[NCOUNT];
    int st[NSTATUS];
    if ((rc = counters_read(c, k, fl, st))) return cleanup(rc);
    if (st[4] > 0) return cleanup(fail(HM_ETIMEOUT, "hm_lu_batch: a bounded device wait gave up"));
    singular += st[0];
    for (int i = i0; i < i1; ++i) {
      const int q = i - i0;
      hm_factor* F = new hm_factor;
      F->ctx = c;
      F->A = A[i];
      F->eps = eps;
      F->arena = ar;
      ar->refs++;
      F->vals = Buf{(char*)ar->vals.p + 8 * bd[q], (size_t)A[i]->lay.nvalues * 8};
      F->ranks = Buf{(char*)ar->ranks.p + 4 * br[q], (size_t)A[i]->lay.nranks * 4};
      F->piv = Buf{(char*)ar->piv.p + 4 * bp[q], (size_t)A[i]->lay.npiv * 4};
      made.push_back(F);
      out[i] = F;
      // time, counters and launches are those of the whole group
      fill_matrix_stats(A[i], &F->st);
      F->st.eps = eps;
      F->st.seconds = ms * 1e-3;
      F->st.plan_seconds = dp.plan_seconds;         // the group's merged plan
      F->st.plan_launches = (int64_t)P.launches.size();
      F->st.plan_phases = P.nphases;
      F->st.plan_truncations = P.ntrunc;
      F->st.scratch_bytes = P.scratch_doubles * 8 + P.scratch_ints * 4;
      F->st.plan_deferred = 0;
      F->st.accumulate = 0;
      F->st.arena_bytes = 0;
      F->st.accumulated_pieces = 0;
      for (int f = 0; f < 5; ++f) F->st.flops[f] = (double)fl[f];
      F->st.singular_pivots = st[0];
      F->st.rank_cap_hits = st[1];
      F->st.row_interchanges = st[3];
      F->st.precision = precision;
      fill_kind_stats(&F->st, Profile(), fl);
      F->st.launches = (int64_t)P.launches.size();
      if ((rc = read_ranks(c, F->ranks, A[i]->lay.nranks, &F->st.max_rank, &F->st.sum_rank))) return cleanup(rc);
    }
    free_plan(c, dp);
    dfree(c, sd);
    dfree(c, si);
    dfree(c, k.b);
    i0 = i1;
  }
  if (singular > 0) return fail(HM_ESINGULAR, "hm_lu_batch: zero pivot in a diagonal leaf");
  return HM_OK;
}

}  // extern "C"

namespace {

// run a solve / matvec plan on the SP_X work buffer; `nv` goes to scratch int 0. The plan's
// scratch is allocated once and the whole launch sequence is captured once into a CUDA graph
// (on a private stream) and then replayed on the context stream: a solve is thousands of
// small dependent launches, and graph replay removes their host launch cost.
int run_aux(hm_ctx* c, hm_matrix* A, hm_factor* F, DevPlan& dp, Buf& work, int nv) {
  if (!dp.sd.p) {
    // all three or none: the replay below needs every one of them
    if (!dalloc(c, dp.sd, std::max<int64_t>(1, dp.host.scratch_doubles) * 8) ||
        !dalloc(c, dp.si, std::max<int64_t>(8, dp.host.scratch_ints) * 4) ||
        !dalloc(c, dp.cnt, NCOUNT * sizeof(unsigned long long) + NSTATUS * sizeof(int))) {
      dfree(c, dp.sd);
      dfree(c, dp.si);
      dfree(c, dp.cnt);
      return fail(HM_ENOMEM, "allocator returned NULL (scratch)");
    }
    CU(cudaMemsetAsync(dp.cnt.p, 0, NCOUNT * sizeof(unsigned long long) + NSTATUS * sizeof(int), c->stream));
  }
  if (launch_set_int((int*)dp.si.p, nv, c->stream)) return fail(HM_ECUDA, "set-int kernel failed");
  if (!dp.exec) {
    Bases B = make_bases();
    B.d[SP_S] = (double*)dp.sd.p;
    B.d[SP_X] = (double*)work.p;
    B.d[SP_A] = (double*)A->vals.p;
    B.d[SP_P] = (double*)A->pts.p;
    B.i[IS_S] = (int*)dp.si.p;
    B.i[IS_ARANK] = (int*)A->ranks.p;
    if (F) {
      B.d[SP_F] = (double*)F->vals.p;
      B.i[IS_RANK] = (int*)F->ranks.p;
      B.i[IS_PIV] = (int*)F->piv.p;
    }
    B.flops = (unsigned long long*)dp.cnt.p;
    B.status = (int*)((char*)dp.cnt.p + NCOUNT * sizeof(unsigned long long));
    prepare_kernels();
    cudaStream_t cs;
    CU(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    int rc = HM_OK;
    if (!e) rc = run_plan(c, dp, B, A->h, nullptr, cs, true);
    cudaError_t e2 = cudaStreamEndCapture(cs, &graph);
    if (!e) e = e2;
    if (!e && rc == HM_OK) e = cudaGraphInstantiate(&dp.exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    cudaStreamDestroy(cs);
    if (rc) return rc;
    if (e) {
      dp.exec = nullptr;
      return fail(HM_ECUDA, std::string("plan capture: ") + cudaGetErrorString(e));
    }
  }
  CU(cudaGraphLaunch(dp.exec, c->stream));
  return HM_OK;
}

int plain_solve(hm_ctx* c, hm_factor* F, const double* b, double* x, int64_t nrhs, int64_t ld) {
  hm_matrix* A = F->A;
  const int n = (int)A->n;
  if (!F->solve_plan.uploaded) {
    try {
      plan_solve(A->ct, A->bt, A->lay, SOLVE_CHUNK, F->solve_plan.host);
    } catch (const std::exception& ex) {
      return fail(HM_EINTERNAL, std::string("hm_solve: ") + ex.what());
    }
    int rc = upload(c, F->solve_plan);
    if (rc) return rc;
  }
  if (!F->work.p && !dalloc(c, F->work, (size_t)n * 4 * SOLVE_CHUNK * 8))
    return fail(HM_ENOMEM, "hm_solve: allocator returned NULL");
  for (int64_t c0 = 0; c0 < nrhs; c0 += SOLVE_CHUNK) {
    const int nc = (int)std::min<int64_t>(SOLVE_CHUNK, nrhs - c0);
    if (launch_permute(b + c0 * ld, ld, (double*)F->work.p, n, (int64_t*)A->perm.p, n, nc, 0, 1.0, 0.0, 0,
                       c->stream))
      return fail(HM_ECUDA, "hm_solve: permute kernel failed");
    int rc = run_aux(c, A, F, F->solve_plan, F->work, nc);
    if (rc) return rc;
    if (launch_permute((double*)F->work.p, n, x + c0 * ld, ld, (int64_t*)A->perm.p, n, nc, 1, 1.0, 0.0, 0,
                       c->stream))
      return fail(HM_ECUDA, "hm_solve: permute kernel failed");
  }
  CU(cudaStreamSynchronize(c->stream));
  return HM_OK;
}

}  // namespace

extern "C" {

int hm_matvec(hm_ctx* c, hm_matrix* A, hm_factor* F, int op, double alpha, const double* x, double beta, double* y,
              int64_t nrhs, int64_t ld) {
  if (!c || !A || !x || !y) return fail(HM_EINVAL, "hm_matvec: NULL argument");
  if (nrhs < 0 || ld < A->n) return fail(HM_EINVAL, "hm_matvec: bad nrhs or ld");
  if (op < HM_OP_A || op > HM_OP_EXACT) return fail(HM_EINVAL, "hm_matvec: unknown op");
  if (op >= HM_OP_L && op <= HM_OP_LU && !F) return fail(HM_EINVAL, "hm_matvec: op needs a factor");
  if (F && F->A != A) return fail(HM_EINVAL, "hm_matvec: factor belongs to another matrix");
  if (nrhs == 0) return HM_OK;
  CU(cudaSetDevice(c->device));
  const int n = (int)A->n;
  if (op == HM_OP_EXACT) {
    Buf t;
    if (!dalloc(c, t, (size_t)n * nrhs * 8)) return fail(HM_ENOMEM, "hm_matvec: allocator returned NULL");
    cudaError_t e = launch_exact_mv((double*)A->pts_orig.p, n, A->h, x, ld, (double*)t.p, n, (int)nrhs, c->stream);
    if (!e) e = launch_axpby((double*)t.p, n, y, ld, n, (int)nrhs, alpha, beta, c->stream);
    if (!e) e = cudaStreamSynchronize(c->stream);
    dfree(c, t);
    if (e) return fail(HM_ECUDA, std::string("hm_matvec: ") + cudaGetErrorString(e));
    return HM_OK;
  }
  DevPlan& dp = F ? F->mv_plan : A->mv_plan;
  Buf& work = F ? F->work : A->mv_work;
  const int want = op;
  if (dp.uploaded && (int)dp.eps != want) free_plan(c, dp);
  if (!dp.uploaded) {
    try {
      plan_matvec(A->ct, A->bt, A->lay, want, SOLVE_CHUNK, dp.host);
    } catch (const std::exception& ex) {
      return fail(HM_EINTERNAL, std::string("hm_matvec: ") + ex.what());
    }
    dp.eps = want;
    int rc = upload(c, dp);
    if (rc) return rc;
  }
  if (!work.p && !dalloc(c, work, (size_t)n * 4 * SOLVE_CHUNK * 8))
    return fail(HM_ENOMEM, "hm_matvec: allocator returned NULL");
  double* W = (double*)work.p;
  for (int64_t c0 = 0; c0 < nrhs; c0 += SOLVE_CHUNK) {
    const int nc = (int)std::min<int64_t>(SOLVE_CHUNK, nrhs - c0);
    if (launch_permute(x + c0 * ld, ld, W, n, (int64_t*)A->perm.p, n, nc, 0, 1.0, 0.0, 0, c->stream))
      return fail(HM_ECUDA, "hm_matvec: permute kernel failed");
    int rc = run_aux(c, A, F, dp, work, nc);
    if (rc) return rc;
    if (launch_permute(W + (size_t)SOLVE_CHUNK * n, n, y + c0 * ld, ld, (int64_t*)A->perm.p, n, nc, 1, alpha, beta,
                       1, c->stream))
      return fail(HM_ECUDA, "hm_matvec: permute kernel failed");
  }
  CU(cudaStreamSynchronize(c->stream));
  return HM_OK;
}

int hm_solve(hm_ctx* c, hm_factor* F, hm_matrix* A, const double* b, double* x, int64_t nrhs, int64_t ld,
             const hm_solve_opts* o, hm_solve_info* info) {
  if (!c || !F || !b || !x) return fail(HM_EINVAL, "hm_solve: NULL argument");
  if (nrhs < 0 || ld < F->A->n) return fail(HM_EINVAL, "hm_solve: bad nrhs or ld");
  if (A && A != F->A) return fail(HM_EINVAL, "hm_solve: A is not the factored matrix");
  if (info) {
    info->iterations = 0;
    info->rel_residual = -1.0;
  }
  if (nrhs == 0) return HM_OK;
  CU(cudaSetDevice(c->device));
  const int n = (int)F->A->n;
  const bool refine = o && o->max_iter > 0 && A;
  if (refine && o->residual_op != HM_OP_A && o->residual_op != HM_OP_EXACT)
    return fail(HM_EINVAL, "hm_solve: residual_op must be HM_OP_A or HM_OP_EXACT");
  Buf bb, r, d, nrm;
  auto done = [&](int rc) {
    dfree(c, bb);
    dfree(c, r);
    dfree(c, d);
    dfree(c, nrm);
    return rc;
  };
  if (refine) {
    // keep b: x and b may alias
    if (!dalloc(c, bb, (size_t)n * nrhs * 8) || !dalloc(c, r, (size_t)n * nrhs * 8) ||
        !dalloc(c, d, (size_t)n * nrhs * 8) || !dalloc(c, nrm, (size_t)2 * nrhs * 8))
      return done(fail(HM_ENOMEM, "hm_solve: allocator returned NULL"));
    if (launch_axpby(b, ld, (double*)bb.p, n, n, (int)nrhs, 1.0, 0.0, c->stream))
      return done(fail(HM_ECUDA, "hm_solve: copy kernel failed"));
  }
  int rc = plain_solve(c, F, b, x, nrhs, ld);
  if (rc || !refine) return done(rc);
  std::vector<double> hn(2 * nrhs);
  if (launch_colnorm2((double*)bb.p, n, n, (int)nrhs, (double*)nrm.p, c->stream))
    return done(fail(HM_ECUDA, "hm_solve: norm kernel failed"));
  CU(cudaMemcpyAsync(hn.data(), nrm.p, nrhs * 8, cudaMemcpyDeviceToHost, c->stream));
  CU(cudaStreamSynchronize(c->stream));
  std::vector<double> bnorm(hn.begin(), hn.begin() + nrhs);
  double rel = 0.0;
  int it = 0;
  for (;;) {
    // r = b - A x
    if (launch_axpby((double*)bb.p, n, (double*)r.p, n, n, (int)nrhs, 1.0, 0.0, c->stream))
      return done(fail(HM_ECUDA, "hm_solve: copy kernel failed"));
    if ((rc = hm_matvec(c, F->A, nullptr, o->residual_op, -1.0, x, 1.0, (double*)r.p, nrhs, ld))) return done(rc);
    if (launch_colnorm2((double*)r.p, n, n, (int)nrhs, (double*)nrm.p, c->stream))
      return done(fail(HM_ECUDA, "hm_solve: norm kernel failed"));
    CU(cudaMemcpyAsync(hn.data(), nrm.p, nrhs * 8, cudaMemcpyDeviceToHost, c->stream));
    CU(cudaStreamSynchronize(c->stream));
    rel = 0.0;
    for (int64_t q = 0; q < nrhs; ++q)
      rel = std::max(rel, bnorm[q] > 0 ? std::sqrt(hn[q] / bnorm[q]) : std::sqrt(hn[q]));
    if (info) {
      info->iterations = it;
      info->rel_residual = rel;
    }
    if (rel <= o->refine_tol || it >= o->max_iter) break;
    if ((rc = plain_solve(c, F, (double*)r.p, (double*)d.p, nrhs, n))) return done(rc);
    if (launch_axpby((double*)d.p, n, x, ld, n, (int)nrhs, 1.0, 1.0, c->stream))
      return done(fail(HM_ECUDA, "hm_solve: update kernel failed"));
    ++it;
  }
  CU(cudaStreamSynchronize(c->stream));
  if (rel > o->refine_tol) return done(fail(HM_ENOTCONV, "hm_solve: refinement did not reach refine_tol"));
  return done(HM_OK);
}

int hm_matrix_layout(const hm_matrix* A, int64_t* leaves, int64_t* perm, int64_t* cluster_lo, int64_t* nleaves,
                     int64_t* nvalues, int64_t* nclusters) {
  if (!A) return fail(HM_EINVAL, "hm_matrix_layout: NULL matrix");
  if (nleaves) *nleaves = (int64_t)A->lay.leaf.size();
  if (nvalues) *nvalues = A->lay.nvalues;
  if (nclusters) *nclusters = (int64_t)A->ct.cl.size();
  if (leaves)
    for (size_t q = 0; q < A->lay.leaf.size(); ++q) {
      const LeafStore& L = A->lay.leaf[q];
      const int64_t r[10] = {L.row, L.col, L.m, L.n, L.lr ? 1 : 0, L.cap, L.off, L.voff, L.rank_idx, L.piv_off};
      std::memcpy(leaves + 10 * q, r, sizeof(r));
    }
  if (perm) std::memcpy(perm, A->ct.perm.data(), A->n * sizeof(int64_t));
  if (cluster_lo)
    for (size_t q = 0; q < A->ct.cl.size(); ++q) cluster_lo[q] = A->ct.cl[q].lo;
  return HM_OK;
}

int hm_matrix_copy_values(hm_ctx* c, hm_matrix* A, double* buf, int to_matrix) {
  if (!c || !A || !buf) return fail(HM_EINVAL, "hm_matrix_copy_values: NULL argument");
  CU(cudaSetDevice(c->device));
  const size_t bytes = (size_t)A->lay.nvalues * 8;
  if (to_matrix) CU(cudaMemcpyAsync(A->vals.p, buf, bytes, cudaMemcpyDeviceToDevice, c->stream));
  else CU(cudaMemcpyAsync(buf, A->vals.p, bytes, cudaMemcpyDeviceToDevice, c->stream));
  CU(cudaStreamSynchronize(c->stream));
  return HM_OK;
}

int hm_matrix_stats(const hm_matrix* A, hm_stats* out) {
  if (!A || !out) return fail(HM_EINVAL, "hm_matrix_stats: NULL argument");
  fill_matrix_stats(A, out);
  int rc = read_ranks(A->ctx, A->ranks, A->lay.nranks, &out->max_rank, &out->sum_rank);
  return rc;
}

int hm_factor_stats(const hm_factor* F, hm_stats* out) {
  if (!F || !out) return fail(HM_EINVAL, "hm_factor_stats: NULL argument");
  *out = F->st;
  return HM_OK;
}

// ------------------------------------------------------------------------------ truncate
int hm_truncate(hm_ctx* c, int64_t m, int64_t n, int K, const double* W, int64_t ldw, const double* Z, int64_t ldz,
                double eps, int cap, double* U, int64_t ldu, double* V, int64_t ldv, int* k_out) {
  if (!c || !W || !Z || !U || !V || !k_out) return fail(HM_EINVAL, "hm_truncate: NULL argument");
  if (m < 1 || n < 1 || K < 0 || K > 256 || cap < 1 || cap > 64 || ldw < m || ldz < n || ldu < m || ldv < n)
    return fail(HM_EINVAL, "hm_truncate: bad sizes (1 <= m, n; 0 <= K <= 256; 1 <= cap <= 64; ld >= rows)");
  if (!(eps >= HM_EPS_MIN)) return fail(HM_EINVAL, "hm_truncate: eps must be >= HM_EPS_MIN (1e-8)");
  if (m > (int64_t)1 << 30 || n > (int64_t)1 << 30) return fail(HM_EINVAL, "hm_truncate: m or n too large");
  CU(cudaSetDevice(c->device));
  const int capk = (int)std::min<int64_t>(cap, std::min(m, n));
  const int Kc = std::max(2, (K + 1) / 2 * 2);
  // scratch layout (doubles): Uo m*capk | Vo n*capk | Wst m*Kc | Zst n*Kc | Gw | Gz | Tw | Tz | work
  const int64_t a = 32;
  auto al = [&](int64_t v) { return (v + a - 1) / a * a; };
  int64_t off = 0;
  const int64_t oU = off; off += al(m * capk);
  const int64_t oV = off; off += al(n * capk);
  const int64_t oW = off; off += al(m * Kc);
  const int64_t oZ = off; off += al(n * Kc);
  const int64_t oGw = off; off += al((int64_t)Kc * Kc);
  const int64_t oGz = off; off += al((int64_t)Kc * Kc);
  const int64_t oTw = off; off += al((int64_t)Kc * capk);
  const int64_t oTz = off; off += al((int64_t)Kc * capk);
  const int64_t oWk = off; off += al(2 * (int64_t)Kc * Kc);
  Buf sd, si, ops, ent;
  Counters k;
  auto done = [&](int r) {
    dfree(c, sd);
    dfree(c, si);
    dfree(c, ops);
    dfree(c, ent);
    dfree(c, k.b);
    return r;
  };
  if (!dalloc(c, sd, off * 8) || !dalloc(c, si, 64)) return done(fail(HM_ENOMEM, "hm_truncate: allocator returned NULL"));
  int rc = counters_init(c, k);
  if (rc) return done(rc);
  // one piece: W Z^T over the whole target; target starts empty (rank 0)
  StackEntry e;
  std::memset(&e, 0, sizeof(e));
  e.W = mkref(SP_X, 0);
  e.w_rs = 1;
  e.w_cs = ldw;
  e.Z = mkref(SP_A, 0);
  e.z_rs = 1;
  e.z_cs = ldz;
  e.k = K;
  e.nrows = (int)m;
  e.ncols = (int)n;
  e.alpha = 1.0;
  TruncOp t;
  std::memset(&t, 0, sizeof(t));
  t.U = mkref(SP_S, oU);
  t.V = mkref(SP_S, oV);
  t.rank = mkref(IS_S, 0);
  t.m = (int)m;
  t.n = (int)n;
  t.cap = capk;
  t.Kcap = Kc;
  t.first_entry = 0;
  t.n_entries = 1;
  t.Wst = mkref(SP_S, oW);
  t.Zst = mkref(SP_S, oZ);
  t.Gw = mkref(SP_S, oGw);
  t.Gz = mkref(SP_S, oGz);
  t.Tw = mkref(SP_S, oTw);
  t.Tz = mkref(SP_S, oTz);
  t.work = mkref(SP_S, oWk);
  t.Kd = mkref(IS_S, 8);
  t.eps = eps;
  GemmOp g[4];
  std::memset(g, 0, sizeof(g));
  const int64_t rows[2] = {m, n};
  const uint64_t st[2] = {t.Wst, t.Zst}, gr[2] = {t.Gw, t.Gz}, tr[2] = {t.Tw, t.Tz}, out[2] = {t.U, t.V};
  for (int q = 0; q < 2; ++q) {   // Gram matrices
    g[q].A = st[q];
    g[q].a_rs = rows[q];
    g[q].a_cs = 1;
    g[q].B = st[q];
    g[q].b_rs = 1;
    g[q].b_cs = rows[q];
    g[q].C = gr[q];
    g[q].c_rs = 1;
    g[q].c_cs = Kc;
    g[q].md = t.Kd;
    g[q].nd = t.Kd;
    g[q].k = (int)rows[q];
    g[q].flags = GF_ATOMIC | GF_SYM_UPPER;
    g[q].alpha = 1.0;
    g[q].fclass = FC_NONE;
  }
  for (int q = 0; q < 2; ++q) {   // rebuild
    g[2 + q].A = st[q];
    g[2 + q].a_rs = 1;
    g[2 + q].a_cs = rows[q];
    g[2 + q].B = tr[q];
    g[2 + q].b_rs = 1;
    g[2 + q].b_cs = Kc;
    g[2 + q].C = out[q];
    g[2 + q].c_rs = 1;
    g[2 + q].c_cs = rows[q];
    g[2 + q].m = (int)rows[q];
    g[2 + q].nd = t.rank;
    g[2 + q].kd = t.Kd;
    g[2 + q].flags = GF_OVERWRITE;
    g[2 + q].alpha = 1.0;
    g[2 + q].fclass = FC_NONE;
  }
  if (!dalloc(c, ops, sizeof(t) + sizeof(g)) || !dalloc(c, ent, sizeof(e)))
    return done(fail(HM_ENOMEM, "hm_truncate: allocator returned NULL"));
  for (int q = 0; q < 4; ++q) g[q].split = (int)Kc;   // expected stacked rank, for the grid split
  int gy0, gz0, gy1, gz1;
  gemm_grid(g, 2, gy0, gz0);
  gemm_grid(g + 2, 2, gy1, gz1);
  cudaStream_t s = c->stream;
  CU(cudaMemcpyAsync(ops.p, &t, sizeof(t), cudaMemcpyHostToDevice, s));
  CU(cudaMemcpyAsync((char*)ops.p + sizeof(t), g, sizeof(g), cudaMemcpyHostToDevice, s));
  CU(cudaMemcpyAsync(ent.p, &e, sizeof(e), cudaMemcpyHostToDevice, s));
  CU(cudaMemsetAsync(si.p, 0, 64, s));
  Bases B = make_bases();
  B.d[SP_S] = (double*)sd.p;
  B.d[SP_X] = const_cast<double*>(W);
  B.d[SP_A] = const_cast<double*>(Z);
  B.i[IS_S] = (int*)si.p;
  B.flops = k.flops();
  B.status = k.status();
  const TruncOp* dt = (const TruncOp*)ops.p;
  const GemmOp* dg = (const GemmOp*)((char*)ops.p + sizeof(t));
  cudaError_t ce = launch_kind(K_STACK, dt, 1, (const StackEntry*)ent.p, B, 0.0, s);
  if (!ce) ce = launch_kind(K_GEMM, dg, 2, nullptr, B, 0.0, s, gy0, gz0);
  if (!ce) ce = launch_kind(K_CORE, dt, 1, (const StackEntry*)ent.p, B, 0.0, s);
  if (!ce) ce = launch_kind(K_GEMM, dg + 2, 2, nullptr, B, 0.0, s, gy1, gz1);
  if (ce) return done(fail(HM_ECUDA, std::string("hm_truncate: ") + cudaGetErrorString(ce)));
  int kk = 0;
  CU(cudaMemcpyAsync(&kk, si.p, sizeof(int), cudaMemcpyDeviceToHost, s));
  CU(cudaStreamSynchronize(s));
  if (kk > 0) {
    CU(cudaMemcpy2DAsync(U, ldu * 8, (double*)sd.p + oU, m * 8, m * 8, kk, cudaMemcpyDeviceToDevice, s));
    CU(cudaMemcpy2DAsync(V, ldv * 8, (double*)sd.p + oV, n * 8, n * 8, kk, cudaMemcpyDeviceToDevice, s));
  }
  CU(cudaStreamSynchronize(s));
  *k_out = kk;
  return done(HM_OK);
}

int hm_set_gemm_work(double fmas_per_cta) {
  if (!(fmas_per_cta >= 256.0) || fmas_per_cta > 16777216.0)
    return fail(HM_EINVAL, "hm_set_gemm_work: fmas_per_cta must be in [256, 2^24]");
  set_gemm_min_work(fmas_per_cta);
  return HM_OK;
}

double hm_get_gemm_work(void) { return gemm_min_work(); }

int hm_set_overlap(int on) {
  if (on != 0 && on != 1) return fail(HM_EINVAL, "hm_set_overlap: on must be 0 or 1");
  g_overlap.store(on);
  return HM_OK;
}

int hm_get_overlap(void) { return g_overlap.load(); }

int hm_autotune_gemm(hm_ctx* c, hm_matrix* A, const hm_lu_opts* o, const double* candidates, int ncand,
                     double* best, double* seconds) {
  if (!c || !A || !candidates || ncand < 1 || !best) return fail(HM_EINVAL, "hm_autotune_gemm: bad argument");
  for (int q = 0; q < ncand; ++q)
    if (!(candidates[q] >= 256.0) || candidates[q] > 16777216.0)
      return fail(HM_EINVAL, "hm_autotune_gemm: candidates must be in [256, 2^24]");
  const double before = gemm_min_work();
  double best_s = -1.0, best_w = before;
  for (int q = 0; q < ncand; ++q) {
    set_gemm_min_work(candidates[q]);
    double t = 0.0;
    for (int rep = 0; rep < 2; ++rep) {   // the first factorization plans at this setting
      hm_factor* F = nullptr;
      const int rc = hm_lu(c, A, o, &F);
      if (F) {
        t = F->st.seconds;
        hm_factor_free(F);
      }
      if (rc != HM_OK && rc != HM_ESINGULAR) {
        set_gemm_min_work(before);
        return rc;
      }
    }
    if (seconds) seconds[q] = t;
    if (best_s < 0.0 || t < best_s) {
      best_s = t;
      best_w = candidates[q];
    }
  }
  set_gemm_min_work(best_w);
  *best = best_w;
  return HM_OK;
}

int hm_selftest_reciprocals(void* cuda_stream, int which, const double* x, double* y, int64_t n) {
  if (which < 0 || which > 3 || n < 0) return fail(HM_EINVAL, "hm_selftest_reciprocals: bad which or n");
  if (n == 0) return HM_OK;
  if (!x || !y) return fail(HM_EINVAL, "hm_selftest_reciprocals: NULL argument");
  cudaStream_t s = (cudaStream_t)cuda_stream;
  cudaError_t e = launch_selftest_rcp(x, y, n, which, s);
  if (!e) e = cudaStreamSynchronize(s);
  if (e) return fail(HM_ECUDA, std::string("hm_selftest_reciprocals: ") + cudaGetErrorString(e));
  return HM_OK;
}

// ------------------------------------------------------------------------------ structure (host only)
}  // extern "C"

struct hm_structure {
  int64_t n = 0;
  ClusterTree ct;
  BlockTree bt;
  TaskGraph g;
  Plan plan;
  bool planned = false;
  Layout lay;
  std::vector<int64_t> leaf_table, sizes;   // plan tables built by hm_structure_plan
  std::vector<int64_t> instances;           // batched plan: first leaf, leaves, value / rank / pivot bases
};

extern "C" {

int hm_structure_build(const double* pts, int64_t n, int leaf_size, double eta, int with_plan, hm_structure** out) {
  if (!pts || !out || n < 1) return fail(HM_EINVAL, "hm_structure_build: bad argument");
  if (leaf_size < 1 || leaf_size > 64) return fail(HM_EINVAL, "hm_structure_build: leaf_size must be in 1..64");
  auto S = std::make_unique<hm_structure>();
  S->n = n;
  try {
    build_cluster_tree(pts, n, leaf_size, S->ct);
    build_block_tree(S->ct, eta, S->bt);
    build_task_graph(S->ct, S->bt, S->g, false, g_host_threads.load());
    if (!compute_levels(S->g)) return fail(HM_EINTERNAL, "hm_structure_build: task graph has a cycle");
    if (with_plan) {
      Layout lay;
      build_layout(S->ct, S->bt, 64, lay);
      plan_lu(S->ct, S->bt, lay, S->g, 1e-6, S->plan, g_host_threads.load());
      S->planned = true;
    }
  } catch (const std::exception& ex) {
    return fail(HM_EINTERNAL, std::string("hm_structure_build: ") + ex.what());
  }
  *out = S.release();
  return HM_OK;
}

int hm_structure_build_accumulator(const double* pts, int64_t n, int leaf_size, double eta, int merged,
                                   hm_structure** out) {
  if (!pts || !out || n < 1) return fail(HM_EINVAL, "hm_structure_build_accumulator: bad argument");
  if (leaf_size < 1 || leaf_size > 64)
    return fail(HM_EINVAL, "hm_structure_build_accumulator: leaf_size must be in 1..64");
  auto S = std::make_unique<hm_structure>();
  S->n = n;
  try {
    build_cluster_tree(pts, n, leaf_size, S->ct);
    build_block_tree(S->ct, eta, S->bt);
    if (merged)
      build_merged_accumulator_graph(S->ct, S->bt, S->g, g_host_threads.load());
    else
      build_task_graph(S->ct, S->bt, S->g, true, g_host_threads.load());
    if (!compute_levels(S->g)) return fail(HM_EINTERNAL, "hm_structure_build_accumulator: task graph has a cycle");
  } catch (const std::exception& ex) {
    return fail(HM_EINTERNAL, std::string("hm_structure_build_accumulator: ") + ex.what());
  }
  *out = S.release();
  return HM_OK;
}

}  // extern "C"

namespace {
// per leaf: row, col, m, n, low-rank, cap, value offset, V offset, rank index, pivot offset,
// with the instance's bases added
void append_leaf_table(const Layout& lay, int64_t bd, int64_t br, int64_t bp, std::vector<int64_t>& out) {
  for (const LeafStore& L : lay.leaf) {
    const int64_t r[10] = {L.row,      L.col,           L.m, L.n, L.lr ? 1 : 0, L.cap, L.off + bd,
                           L.voff + bd, L.rank_idx < 0 ? -1 : L.rank_idx + br, L.piv_off < 0 ? -1 : L.piv_off + bp};
    out.insert(out.end(), r, r + 10);
  }
}
}  // namespace

extern "C" {

int hm_structure_build_sparsified(const double* pts, int64_t n, int leaf_size, double eta, int accumulators,
                                  hm_structure** out) {
  if (!pts || !out || n < 1) return fail(HM_EINVAL, "hm_structure_build_sparsified: bad argument");
  if (leaf_size < 1 || leaf_size > 64)
    return fail(HM_EINVAL, "hm_structure_build_sparsified: leaf_size must be in 1..64");
  auto S = std::make_unique<hm_structure>();
  S->n = n;
  try {
    build_cluster_tree(pts, n, leaf_size, S->ct);
    build_block_tree(S->ct, eta, S->bt);
    build_task_graph(S->ct, S->bt, S->g, accumulators != 0, g_host_threads.load(), true);
    if (!compute_levels(S->g)) return fail(HM_EINTERNAL, "hm_structure_build_sparsified: task graph has a cycle");
  } catch (const std::exception& ex) {
    return fail(HM_EINTERNAL, std::string("hm_structure_build_sparsified: ") + ex.what());
  }
  *out = S.release();
  return HM_OK;
}

int hm_set_host_threads(int threads) {
  if (threads < 0) return fail(HM_EINVAL, "hm_set_host_threads: threads must be >= 0");
  g_host_threads.store(threads);
  return HM_OK;
}

int hm_structure_plan(hm_structure* S, int which, double eps, int rank_cap, int nrhs_max, int threads) {
  if (!S) return fail(HM_EINVAL, "hm_structure_plan: NULL structure");
  if (which < 0 || which > 9) return fail(HM_EINVAL, "hm_structure_plan: which must be in 0..9");
  if (rank_cap < 1 || rank_cap > 64) return fail(HM_EINVAL, "hm_structure_plan: rank_cap must be in 1..64");
  if ((which == 0 || which >= 6) && !(eps > 0.0)) return fail(HM_EINVAL, "hm_structure_plan: eps must be > 0");
  if (which >= 1 && which <= 5 && nrhs_max < 1) return fail(HM_EINVAL, "hm_structure_plan: nrhs_max must be >= 1");
  if (threads < 0) return fail(HM_EINVAL, "hm_structure_plan: threads must be >= 0");
  for (const Task& t : S->g.nodes)
    if (t.type > T_TRSU) return fail(HM_EINVAL, "hm_structure_plan: the structure holds an accumulator task graph");
  try {
    build_layout(S->ct, S->bt, rank_cap, S->lay);
    if (which == 0 || which >= 7)
      plan_lu(S->ct, S->bt, S->lay, S->g, eps, S->plan, threads ? threads : g_host_threads.load(), 0,
              which == 7 || which == 9, which >= 8);
    else if (which == 1)
      plan_solve(S->ct, S->bt, S->lay, nrhs_max, S->plan);
    else if (which <= 5)
      plan_matvec(S->ct, S->bt, S->lay, which - 2, nrhs_max, S->plan);
    else
      plan_build(S->ct, S->bt, S->lay, eps, 160, (int64_t)1 << 28, S->plan);
  } catch (const std::exception& ex) {
    S->planned = false;
    return fail(HM_EINTERNAL, std::string("hm_structure_plan: ") + ex.what());
  }
  S->planned = true;
  S->leaf_table.clear();
  append_leaf_table(S->lay, 0, 0, 0, S->leaf_table);
  const Plan& P = S->plan;
  S->sizes = {P.scratch_doubles, P.scratch_ints, S->lay.nvalues, S->lay.nranks, S->lay.npiv,
              P.ntrunc,          P.nwaves,       P.nphases,         P.arena_doubles};
  S->instances = {0, (int64_t)S->lay.leaf.size(), 0, 0, 0};
  return HM_OK;
}

int hm_structure_plan_lu_batch(hm_structure* const* S, int count, double eps, int rank_cap) {
  if (!S || count < 1) return fail(HM_EINVAL, "hm_structure_plan_lu_batch: bad argument");
  if (rank_cap < 1 || rank_cap > 64) return fail(HM_EINVAL, "hm_structure_plan_lu_batch: rank_cap must be in 1..64");
  if (!(eps > 0.0)) return fail(HM_EINVAL, "hm_structure_plan_lu_batch: eps must be > 0");
  for (int i = 0; i < count; ++i) {
    if (!S[i]) return fail(HM_EINVAL, "hm_structure_plan_lu_batch: NULL structure");
    for (int j = 0; j < i; ++j)
      if (S[j] == S[i]) return fail(HM_EINVAL, "hm_structure_plan_lu_batch: a structure is listed twice");
    for (const Task& t : S[i]->g.nodes)
      if (t.type > T_TRSU) return fail(HM_EINVAL, "hm_structure_plan_lu_batch: an accumulator task graph");
  }
  hm_structure* H = S[0];
  std::vector<LuInstance> inst;
  std::vector<int64_t> table, insts;
  int64_t bd = 0, br = 0, bp = 0, nleaves = 0;
  try {
    for (int i = 0; i < count; ++i) {
      build_layout(S[i]->ct, S[i]->bt, rank_cap, S[i]->lay);
      inst.push_back({&S[i]->ct, &S[i]->bt, &S[i]->lay, &S[i]->g, bd, br, bp});
      append_leaf_table(S[i]->lay, bd, br, bp, table);
      insts.insert(insts.end(), {nleaves, (int64_t)S[i]->lay.leaf.size(), bd, br, bp});
      nleaves += (int64_t)S[i]->lay.leaf.size();
      bd += (S[i]->lay.nvalues + 31) / 32 * 32;
      br += S[i]->lay.nranks;
      bp += S[i]->lay.npiv;
    }
    plan_lu_batch(inst, eps, H->plan, g_host_threads.load());
  } catch (const std::exception& ex) {
    H->planned = false;
    H->sizes.clear();
    return fail(HM_EINTERNAL, std::string("hm_structure_plan_lu_batch: ") + ex.what());
  }
  H->planned = true;
  H->leaf_table.swap(table);
  H->instances.swap(insts);
  const Plan& P = H->plan;
  H->sizes = {P.scratch_doubles, P.scratch_ints, bd, br, bp, P.ntrunc, P.nwaves, P.nphases, 0};
  return HM_OK;
}

int hm_structure_plan_table(const hm_structure* S, int table, const void** data, int64_t* count,
                            int64_t* elem_bytes) {
  if (!S || !data || !count || !elem_bytes) return fail(HM_EINVAL, "hm_structure_plan_table: NULL argument");
  if (!S->planned || S->sizes.empty()) return fail(HM_EINVAL, "hm_structure_plan_table: no plan (hm_structure_plan)");
  const Plan& P = S->plan;
  auto put = [&](const void* d, size_t n, size_t b) {
    *data = d;
    *count = (int64_t)n;
    *elem_bytes = (int64_t)b;
    return HM_OK;
  };
  switch (table) {
    case HM_PLAN_LAUNCHES: return put(P.launches.data(), P.launches.size(), sizeof(Launch));
    case HM_PLAN_GETRF: return put(P.getrf.data(), P.getrf.size(), sizeof(GetrfOp));
    case HM_PLAN_TRSM: return put(P.trsm.data(), P.trsm.size(), sizeof(TrsmOp));
    case HM_PLAN_GEMM: return put(P.gemm.data(), P.gemm.size(), sizeof(GemmOp));
    case HM_PLAN_COPY: return put(P.copy.data(), P.copy.size(), sizeof(CopyOp));
    case HM_PLAN_TRUNC: return put(P.trunc.data(), P.trunc.size(), sizeof(TruncOp));
    case HM_PLAN_ENTRIES: return put(P.entries.data(), P.entries.size(), sizeof(StackEntry));
    case HM_PLAN_LEAVES: return put(S->leaf_table.data(), S->leaf_table.size() / 10, 10 * sizeof(int64_t));
    case HM_PLAN_SIZES: return put(S->sizes.data(), 1, S->sizes.size() * sizeof(int64_t));
    case HM_PLAN_INSTANCES: return put(S->instances.data(), S->instances.size() / 5, 5 * sizeof(int64_t));
    case HM_PLAN_EVAL: return put(P.eval.data(), P.eval.size(), sizeof(EvalOp));
    case HM_PLAN_ACA: return put(P.aca.data(), P.aca.size(), sizeof(AcaOp));
    default: return fail(HM_EINVAL, "hm_structure_plan_table: unknown table");
  }
}

int hm_structure_info_get(const hm_structure* S, hm_structure_info* o) {
  if (!S || !o) return fail(HM_EINVAL, "hm_structure_info_get: NULL argument");
  std::memset(o, 0, sizeof(*o));
  o->n = S->n;
  o->nclusters = (int64_t)S->ct.cl.size();
  o->nleaves = (int64_t)S->bt.leaves.size();
  o->ntasks = (int64_t)S->g.nodes.size();
  o->nedges = (int64_t)S->g.edges.size();
  o->nlevels = S->g.nlevels;
  o->dag_seconds = S->g.build_seconds;
  if (S->planned) {
    o->plan_launches = (int64_t)S->plan.launches.size();
    o->plan_phases = S->plan.nphases;
    o->plan_gemm_ops = (int64_t)S->plan.gemm.size();
    o->plan_truncations = S->plan.ntrunc;
    o->plan_scratch_bytes = S->plan.scratch_doubles * 8 + S->plan.scratch_ints * 4;
  }
  return HM_OK;
}

int hm_structure_export(const hm_structure* S, int64_t* perm, int32_t* clusters, int32_t* leaves, int32_t* tasks,
                        int32_t* edges, int32_t* levels) {
  if (!S) return fail(HM_EINVAL, "hm_structure_export: NULL structure");
  if (perm)
    for (int64_t i = 0; i < S->n; ++i) perm[i] = S->ct.perm[i];
  if (clusters)
    for (size_t i = 0; i < S->ct.cl.size(); ++i) {
      const Cluster& c = S->ct.cl[i];
      int32_t* r = clusters + 6 * i;
      r[0] = c.lo;
      r[1] = c.hi;
      r[2] = c.son0;
      r[3] = c.son1;
      r[4] = c.level;
      r[5] = c.parent;
    }
  if (leaves)
    for (size_t i = 0; i < S->bt.leaves.size(); ++i) {
      const BlockNode& b = S->bt.nodes[S->bt.leaves[i]];
      leaves[3 * i] = b.row;
      leaves[3 * i + 1] = b.col;
      leaves[3 * i + 2] = b.adm ? 1 : 0;
    }
  if (tasks)
    for (size_t i = 0; i < S->g.nodes.size(); ++i) {
      const Task& t = S->g.nodes[i];
      tasks[4 * i] = t.type;
      tasks[4 * i + 1] = t.a;
      tasks[4 * i + 2] = t.b;
      tasks[4 * i + 3] = t.c;
    }
  if (edges)
    for (size_t i = 0; i < S->g.edges.size(); ++i) {
      edges[2 * i] = S->g.edges[i].first;
      edges[2 * i + 1] = S->g.edges[i].second;
    }
  if (levels)
    for (size_t i = 0; i < S->g.nodes.size(); ++i) levels[i] = S->g.level[i];
  return HM_OK;
}

void hm_structure_free(hm_structure* S) { delete S; }

}  // extern "C"

namespace hm {
// Last-error setter for entry points defined in other translation units (noalloc.cu).
int set_last_error(int code, const char* msg) {
  g_err = msg;
  return code;
}
}  // namespace hm
