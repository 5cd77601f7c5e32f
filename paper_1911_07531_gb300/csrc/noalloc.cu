// hm_truncate_noalloc: the rounded truncation of hm_truncate with all of its device scratch
// in one file-scope array, for callers that must not allocate device memory.
//
// Some callers cannot allocate: a serving loop that sizes every device buffer at start-up and
// forbids allocation afterwards (fixed memory budget, no allocator latency on the request
// path), or a plugin that runs inside another framework's memory pool and has no allocator
// of its own to pass to hm_ctx_create. This entry point takes a stream instead of a context
// and never calls cudaMalloc, cudaFree or any allocating routine: its work space is the
// static device array below, which every GPU that loads the library holds until the process
// exits.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <mutex>
#include <string>

#include "../../include/hmgb300.h"
#include "kernels.h"
#include "plan.h"

namespace hm {
// defined in api.cu: sets the thread's last-error message and returns `code`
int set_last_error(int code, const char* msg);
}  // namespace hm

using namespace hm;

namespace {

// 2^21 doubles = 16 MiB of scratch per device
constexpr int64_t NOALLOC_DOUBLES = (int64_t)1 << 21;
static __device__ __align__(256) double g_noalloc_scratch[NOALLOC_DOUBLES];

constexpr int MAX_DEVICES = 64;
std::mutex g_mu;
double* g_base[MAX_DEVICES] = {nullptr};

// Device address of g_noalloc_scratch on the current device; looked up once per device and
// cached by device ordinal. The address belongs to the device's primary context (the one the
// CUDA runtime uses): callers in other contexts, or after cudaDeviceReset, are not supported.
int scratch_base(double** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return set_last_error(HM_ECUDA, "hm_truncate_noalloc: no current CUDA device");
  if (dev < 0 || dev >= MAX_DEVICES) return set_last_error(HM_EINVAL, "hm_truncate_noalloc: device ordinal >= 64");
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_base[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p)
      return set_last_error(HM_ECUDA, (std::string("hm_truncate_noalloc: cudaGetSymbolAddress: ") +
                                       cudaGetErrorString(e)).c_str());
    g_base[dev] = (double*)p;
  }
  *out = g_base[dev];
  return HM_OK;
}

inline int64_t al(int64_t v) { return (v + 31) / 32 * 32; }

}  // namespace

extern "C" int hm_truncate_noalloc(void* cuda_stream, int64_t m, int64_t n, int K, const double* W, int64_t ldw,
                                   const double* Z, int64_t ldz, double eps, int cap, double* U, int64_t ldu,
                                   double* V, int64_t ldv, int* k_out) {
  if (!W || !Z || !U || !V || !k_out) return set_last_error(HM_EINVAL, "hm_truncate_noalloc: NULL argument");
  if (m < 1 || n < 1 || K < 0 || K > 256 || cap < 1 || cap > 64 || ldw < m || ldz < n || ldu < m || ldv < n)
    return set_last_error(HM_EINVAL, "hm_truncate_noalloc: bad sizes (1 <= m, n; 0 <= K <= 256; 1 <= cap <= 64; "
                                     "ld >= rows)");
  if (!(eps >= HM_EPS_MIN)) return set_last_error(HM_EINVAL, "hm_truncate_noalloc: eps must be >= HM_EPS_MIN (1e-8)");
  if (m > (int64_t)1 << 30 || n > (int64_t)1 << 30)
    return set_last_error(HM_EINVAL, "hm_truncate_noalloc: m or n too large");
  const int capk = (int)std::min<int64_t>(cap, std::min(m, n));
  const int Kc = K < 2 ? 2 : (K + 1) / 2 * 2;
  // layout of the static array (doubles): descriptors | ints + counters | Wst | Zst | Gw | Gz | Tw | Tz | work
  const int64_t oDesc = 0;
  const int64_t oInts = oDesc + al((sizeof(TruncOp) + 4 * sizeof(GemmOp) + sizeof(StackEntry) + 7) / 8);
  const int64_t oCnt = oInts + 8;                       // ints: [0] rank, [8] stacked K (16 ints)
  const int64_t oW = oCnt + al(NFC + NKIND + 4);
  const int64_t oZ = oW + al(m * Kc);
  const int64_t oGw = oZ + al(n * Kc);
  const int64_t oGz = oGw + al((int64_t)Kc * Kc);
  const int64_t oTw = oGz + al((int64_t)Kc * Kc);
  const int64_t oTz = oTw + al((int64_t)Kc * capk);
  const int64_t oWk = oTz + al((int64_t)Kc * capk);
  const int64_t need = oWk + al(2 * (int64_t)Kc * Kc);
  if (need > NOALLOC_DOUBLES)
    return set_last_error(HM_EINVAL, "hm_truncate_noalloc: m, n, K exceed the 16 MiB static scratch "
                                     "(m + n <= 8192 with K <= 128 always fits)");
  double* base = nullptr;
  int rc = scratch_base(&base);
  if (rc != HM_OK) return rc;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  int* ints = (int*)(base + oInts);

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
  t.U = mkref(SP_F, 0);           // the caller's U and V receive the result directly
  t.V = mkref(SP_P, 0);
  t.rank = mkref(IS_S, 0);        // starts at 0: the target is empty
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
  const int64_t rows[2] = {m, n}, ld_out[2] = {ldu, ldv};
  const uint64_t st[2] = {t.Wst, t.Zst}, gr[2] = {t.Gw, t.Gz}, tr[2] = {t.Tw, t.Tz}, out[2] = {t.U, t.V};
  for (int q = 0; q < 2; ++q) {   // Gram matrices of the stacked factors
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
  for (int q = 0; q < 2; ++q) {   // U = W_st T_W, V = Z_st T_Z into the caller's buffers
    g[2 + q].A = st[q];
    g[2 + q].a_rs = 1;
    g[2 + q].a_cs = rows[q];
    g[2 + q].B = tr[q];
    g[2 + q].b_rs = 1;
    g[2 + q].b_cs = Kc;
    g[2 + q].C = out[q];
    g[2 + q].c_rs = 1;
    g[2 + q].c_cs = ld_out[q];
    g[2 + q].m = (int)rows[q];
    g[2 + q].nd = t.rank;
    g[2 + q].kd = t.Kd;
    g[2 + q].flags = GF_OVERWRITE;
    g[2 + q].alpha = 1.0;
    g[2 + q].fclass = FC_NONE;
  }
  char* desc = (char*)(base + oDesc);
  TruncOp* dt = (TruncOp*)desc;
  GemmOp* dg = (GemmOp*)(desc + sizeof(TruncOp));
  StackEntry* de = (StackEntry*)(desc + sizeof(TruncOp) + sizeof(g));
  for (int q = 0; q < 4; ++q) g[q].split = (int)Kc;   // expected stacked rank, for the grid split
  int gy0, gz0, gy1, gz1;
  gemm_grid(g, 2, gy0, gz0);
  gemm_grid(g + 2, 2, gy1, gz1);
  cudaError_t ce = cudaMemcpyAsync(dt, &t, sizeof(t), cudaMemcpyHostToDevice, s);
  if (!ce) ce = cudaMemcpyAsync(dg, g, sizeof(g), cudaMemcpyHostToDevice, s);
  if (!ce) ce = cudaMemcpyAsync(de, &e, sizeof(e), cudaMemcpyHostToDevice, s);
  // the previous call's rank, stacked rank and counters must not leak into this one
  if (!ce) ce = cudaMemsetAsync(base + oInts, 0, (oW - oInts) * sizeof(double), s);
  if (ce) return set_last_error(HM_ECUDA, (std::string("hm_truncate_noalloc: ") + cudaGetErrorString(ce)).c_str());
  Bases B;
  std::memset(&B, 0, sizeof(B));
  B.d[SP_S] = base;
  B.d[SP_X] = const_cast<double*>(W);
  B.d[SP_A] = const_cast<double*>(Z);
  B.d[SP_F] = U;
  B.d[SP_P] = V;
  B.i[IS_S] = ints;
  B.flops = (unsigned long long*)(base + oCnt);
  B.status = (int*)(base + oCnt + NFC + NKIND);
  ce = launch_kind(K_STACK, dt, 1, de, B, 0.0, s);
  if (!ce) ce = launch_kind(K_GEMM, dg, 2, nullptr, B, 0.0, s, gy0, gz0);
  if (!ce) ce = launch_kind(K_CORE, dt, 1, de, B, 0.0, s);
  if (!ce) ce = launch_kind(K_GEMM, dg + 2, 2, nullptr, B, 0.0, s, gy1, gz1);
  int kk = 0;
  if (!ce) ce = cudaMemcpyAsync(&kk, ints, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (!ce) ce = cudaStreamSynchronize(s);
  if (ce) {
    // kernels already queued may still use the shared array: let them finish before the next
    // call can start on another stream
    cudaStreamSynchronize(s);
    return set_last_error(HM_ECUDA, (std::string("hm_truncate_noalloc: ") + cudaGetErrorString(ce)).c_str());
  }
  *k_out = kk;
  return HM_OK;
}
