// Planner: expansion of H-LU tasks (and of solves / matvecs) into batched micro-ops.
//
// The task graph of Alg 11 is executed in waves (its longest-path levels). A task of a
// wave is a leaf task of the refinement: hlu on a diagonal leaf, htrsl / htrsu on a leaf
// block (possibly with a structured triangle), or hmul with at least one leaf operand
// (Alg 1, non-recursive branch). Each is expanded here into micro-ops in phases:
//
//   phase 0..2   leaf LU, triangular solves, and the products A B of hmul formed as
//                low-rank pieces W Z^T (thin H-matrix products through the leaves of the
//                structured operand);
//   phase 3..    application of the pieces: atomic GEMMs into dense leaves; for low-rank
//                leaves, one rounded addition per leaf and wave that stacks the leaf and
//                all pieces reaching it (STACK -> Gram GEMMs -> CORE -> rebuild GEMMs),
//                repeated in rounds when the stacked rank would exceed KMAX.
//
// Two updates of one block inside a wave have no edge between them (Def 3.2 only orders
// writes before reads); they commute up to rounding, so merging them into one rounded
// addition is a valid schedule of the same task graph.
#include "plan.h"

#include <algorithm>
#include <array>
#include <unordered_map>
#include <atomic>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <map>
#include <set>
#include <memory>
#include <stdexcept>
#include <string>
#include <thread>

namespace hm {

namespace {
// worker() on the calling thread and on up to threads - 1 more (fewer if the system refuses
// to start them); returns when all have finished
template <class F>
void run_workers(int threads, F worker) {
  std::vector<std::thread> pool;
  for (int t = 1; t < threads; ++t) {
    try {
      pool.emplace_back(worker);
    } catch (...) {
      break;
    }
  }
  worker();
  for (auto& th : pool) th.join();
}
}  // namespace

namespace {
std::atomic<double> g_gemm_min_work{4096.0};
}  // namespace

void set_gemm_min_work(double w) { g_gemm_min_work.store(w > 0.0 ? w : 4096.0); }
double gemm_min_work() { return g_gemm_min_work.load(); }

void gemm_grid_to(const GemmOp* ops, int count, GemmOp* out, int& gy, int& gz) {
  // Dynamic sizes (ranks) are not known here: each micro-op carries an expected value in
  // `split` (0: 16). A CTA should get at least the tuned work (default 4096 FMAs, ~2k cycles of
  // one SM's FP64 pipe; set_gemm_min_work) and
  // about the launch's average work per CTA slot (three resident CTAs per SM). The split stored
  // is a budget of CTAs (grid y = the largest budget, z = 1); the kernel lowers it from the
  // actual sizes and divides it between C tiles and reduction slices.
  const double kMinWork = g_gemm_min_work.load();
  constexpr int kSlots = 3 * 152, kMaxSplit = 128, kTile = 1024, kSlice = 16;
  thread_local std::vector<double> w;
  thread_local std::vector<int> idx;
  w.resize(count);
  idx.resize(count);
  auto dims = [](const GemmOp& o, double& m, double& n, double& k) {
    const double dyn = o.split > 0 ? (double)o.split : 16.0;
    m = o.m + (o.md ? dyn : 0.0);
    n = o.n + (o.nd ? dyn : 0.0);
    k = o.k + (o.kd ? dyn : 0.0);
  };
  double total = 0.0;
  for (int q = 0; q < count; ++q) {
    double m, n, k;
    dims(ops[q], m, n, k);
    w[q] = m * n * k;
    total += w[q];
    idx[q] = q;
  }
  const double target = std::max(kMinWork, total / kSlots);
  std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) { return w[a] > w[b]; });
  gy = gz = 1;
  for (int t = 0; t < count; ++t) {
    const GemmOp& src = ops[idx[t]];
    double m, n, k;
    dims(src, m, n, k);
    const int want = std::min(kMaxSplit, std::max(1, (int)std::ceil(w[idx[t]] / target)));
    const int tiles = std::max(1, (int)((m * n + kTile - 1) / kTile));
    const int slices = (src.flags & GF_ATOMIC) ? std::max(1, (int)((k + kSlice - 1) / kSlice)) : 1;
    // a CTA budget: the kernel factors it into C tiles and reduction slices of the actual sizes
    const int budget = std::max(1, std::min(want, tiles * slices));
    out[t] = src;
    out[t].split = budget;
    gy = std::max(gy, budget);
  }
}

void gemm_grid(GemmOp* ops, int count, int& gy, int& gz) {
  std::vector<GemmOp> in(ops, ops + count);
  gemm_grid_to(in.data(), count, ops, gy, gz);
}

namespace {

constexpr int KMAX_STACK = 256;     // largest stacked rank of one rounded addition
constexpr int KMAX_ENTRIES = 256;   // largest number of pieces of one rounded addition (k_stack)
constexpr int GEMM_MCHUNK = 512;    // row chunk of a GEMM micro-op
constexpr int GEMM_KCHUNK = 512;    // reduction chunk of an accumulating GEMM micro-op
constexpr int TRSM_VCHUNK = 256;    // vectors of one triangular-solve micro-op
constexpr int TC_MIN_ROWS = 128;    // mixed precision: GEMM micro-ops with this many rows go to the tensor cores
constexpr int64_t ALIGN = 32;       // doubles (256 bytes)

inline int64_t align_up(int64_t x) { return (x + ALIGN - 1) / ALIGN * ALIGN; }

struct View {
  uint64_t ref;
  int64_t es, vs;   // element (row) stride, vector (column) stride
  View off(int64_t rows) const { return {ref + (uint64_t)(rows * es), es, vs}; }
};

struct Dim {
  int s;
  uint64_t d;
};

struct Piece {
  View W, Z;
  Dim k;
  int kmax;
  int ro, nrows, co, ncols;
  double alpha;
};

struct TargetEntries {
  int leaf;
  std::vector<std::pair<StackEntry, int>> e;   // entry, static max rank
};

struct Wave {
  std::vector<std::vector<GetrfOp>> getrf;
  std::vector<std::vector<TrsmOp>> trsm;
  std::vector<std::vector<GemmOp>> gemm;
  std::vector<std::vector<CopyOp>> copy;
  std::vector<std::vector<TruncOp>> stack, core;
  std::vector<std::vector<EvalOp>> eval;
  std::vector<std::vector<AcaOp>> aca;
  std::vector<std::vector<std::vector<StackEntry>>> stack_entries;   // per phase, per stack op
  int64_t sd = 0, si = 0;
  int nph = 0;
  void need(int ph) {
    if (ph + 1 > nph) nph = ph + 1;
    if ((int)gemm.size() <= ph) {
      getrf.resize(ph + 1);
      trsm.resize(ph + 1);
      gemm.resize(ph + 1);
      copy.resize(ph + 1);
      stack.resize(ph + 1);
      core.resize(ph + 1);
      eval.resize(ph + 1);
      aca.resize(ph + 1);
      stack_entries.resize(ph + 1);
    }
  }
  // empty every phase but keep the storage for the next wave
  void reset() {
    for (auto& v : getrf) v.clear();
    for (auto& v : trsm) v.clear();
    for (auto& v : gemm) v.clear();
    for (auto& v : copy) v.clear();
    for (auto& v : stack) v.clear();
    for (auto& v : core) v.clear();
    for (auto& v : eval) v.clear();
    for (auto& v : aca) v.clear();
    for (auto& v : stack_entries) v.clear();
    sd = si = 0;
    nph = 0;
  }
  int64_t alloc_d(int64_t n) {
    int64_t o = sd;
    sd += align_up(n);
    return o;
  }
  int64_t alloc_i(int64_t n) {
    int64_t o = si;
    si += (n + 7) / 8 * 8;
    return o;
  }
};

// Accumulator arena of an accumulator H-LU plan: blocks of doubles that live from the wave that
// allocates them to a release wave fixed at allocation (best fit among the free blocks, which
// coalesce; the top grows when none fits).
struct Arena {
  std::map<int64_t, int64_t> by_off;              // free blocks: offset -> size
  std::set<std::pair<int64_t, int64_t>> by_size;  // free blocks: (size, offset)
  std::multimap<int, std::pair<int64_t, int64_t>> later;   // release wave -> (offset, size)
  int64_t top = 0;
  int64_t alloc(int64_t n, int release_wave) {
    n = align_up(n);
    int64_t off;
    auto it = by_size.lower_bound({n, INT64_MIN});
    if (it != by_size.end()) {
      const int64_t sz = it->first;
      off = it->second;
      by_size.erase(it);
      by_off.erase(off);
      if (sz > n) {
        by_off[off + n] = sz - n;
        by_size.insert({sz - n, off + n});
      }
    } else {
      off = top;
      top += n;
    }
    later.insert({release_wave, {off, n}});
    return off;
  }
  void give_back(int64_t off, int64_t n) {
    auto nx = by_off.lower_bound(off);
    if (nx != by_off.end() && off + n == nx->first) {   // merge with the next free block
      n += nx->second;
      by_size.erase({nx->second, nx->first});
      nx = by_off.erase(nx);
    }
    if (nx != by_off.begin()) {   // merge with the previous one
      auto pv = std::prev(nx);
      if (pv->first + pv->second == off) {
        by_size.erase({pv->second, pv->first});
        off = pv->first;
        n += pv->second;
        by_off.erase(pv);
      }
    }
    by_off[off] = n;
    by_size.insert({n, off});
  }
  // the blocks whose release wave is <= wave become free
  void release_until(int wave) {
    while (!later.empty() && later.begin()->first <= wave) {
      give_back(later.begin()->second.first, later.begin()->second.second);
      later.erase(later.begin());
    }
  }
};

// For every leaf block, its events in the task graph sorted by level: (level, 1) where a task
// reads it (the leaf LU, a triangular solve, an operand of a product) and (level, 0) where a
// product updates it.
using LeafEvents = std::vector<std::vector<std::pair<int, int>>>;

struct Ctx {
  const ClusterTree& ct;
  const BlockTree& bt;
  const Layout& lay;
  Spaces sp;
  Plan& plan;
  Wave own;
  Wave& w;   // the wave being filled: this context's own, or one shared by several instances
  // offsets of this instance's values, ranks and pivots in their spaces (batched plans)
  int64_t base_d = 0, base_r = 0, base_p = 0;
  // mixed precision (0: FP64; 1: factor and rebuild products in FP32 (GF_F32); 2: those with at
  // least TC_MIN_ROWS rows on the tensor cores (GF_TF32), the others in FP32)
  int mixed = 0;
  // scratch spaces of the current wave (the odd waves of a plan with deferred rounded additions
  // use the second pair), the wave's level, and the first phase of its side launches
  int ss = SP_S, sis = IS_S;
  int level = -1;
  int side_from = 1 << 30;
  // pieces reaching low-rank leaves in the current wave, by leaf index
  std::map<int, int> target_index;
  std::vector<TargetEntries> targets;
  // accumulator H-LU: the leaves' events, the arena, the pieces held for each leaf until its
  // rounded addition, and the release wave of the pieces being formed (-1: wave scratch)
  const LeafEvents* events = nullptr;
  Arena* arena = nullptr;
  std::map<int, std::vector<std::pair<StackEntry, int>>> pending;
  int piece_release = -1;
  Ctx(const ClusterTree& c, const BlockTree& b, const Layout& l, Spaces s, Plan& p)
      : ct(c), bt(b), lay(l), sp(s), plan(p), w(own) {}
  Ctx(const ClusterTree& c, const BlockTree& b, const Layout& l, Spaces s, Plan& p, Wave& shared)
      : ct(c), bt(b), lay(l), sp(s), plan(p), w(shared) {}

  const Cluster& cl(int id) const { return ct.cl[id]; }
  const BlockNode& node(int id) const { return bt.nodes[id]; }
  const LeafStore& leaf_of(int nodeid) const { return lay.leaf[bt.nodes[nodeid].leaf]; }
  int find(int r, int c) const {
    int id = bt.find(r, c);
    if (id < 0) throw std::runtime_error("planner: block not in block tree");
    return id;
  }
  uint64_t dref(int64_t off) const { return mkref(sp.d, off + base_d); }
  uint64_t rref(const LeafStore& L) const { return mkref(sp.r, L.rank_idx + base_r); }
  uint64_t pref(const LeafStore& L) const { return mkref(IS_PIV, L.piv_off + base_p); }
  uint64_t sref(int64_t off) const { return mkref(ss, off); }
  // memory of an update piece: the wave's scratch, or the arena when the piece is held
  uint64_t palloc(int64_t n) {
    return piece_release >= 0 ? mkref(SP_ACC, arena->alloc(n, piece_release)) : sref(w.alloc_d(n));
  }
  // accumulator H-LU: the wave of the rounded addition of the pieces that an update at level lv
  // brings to leaf `leaf`: the last update level before the leaf's next read
  int flush_level(int leaf, int lv) const {
    const auto& ev = (*events)[leaf];
    auto it = std::upper_bound(ev.begin(), ev.end(), std::make_pair(lv, 1));
    int f = lv;
    for (; it != ev.end() && it->second == 0; ++it) f = it->first;
    return f;
  }
  // accumulator H-LU: the targets of this wave whose rounded addition comes later hand their
  // pieces to `pending`; the others take the pieces held for them (in arrival order) first
  void hold_pending(int lv) {
    std::vector<TargetEntries> keep;
    for (TargetEntries& T : targets) {
      if (flush_level(T.leaf, lv) > lv) {
        auto& P = pending[T.leaf];
        P.insert(P.end(), T.e.begin(), T.e.end());
        plan.accumulated_pieces += (int64_t)T.e.size();
        continue;
      }
      auto it = pending.find(T.leaf);
      if (it != pending.end()) {
        T.e.insert(T.e.begin(), it->second.begin(), it->second.end());
        pending.erase(it);
      }
      keep.push_back(std::move(T));
    }
    targets.swap(keep);
    target_index.clear();
    for (size_t q = 0; q < targets.size(); ++q) target_index[targets[q].leaf] = (int)q;
  }

  // ---------------------------------------------------------------- micro-op emitters
  // dhint: expected value of the dynamic sizes (a rank or a stacked rank), for the grid split
  void gemm(int ph, uint64_t A, int64_t ars, int64_t acs, uint64_t B, int64_t brs, int64_t bcs, uint64_t C,
            int64_t crs, int64_t ccs, Dim m, Dim n, Dim k, double alpha, int flags, int fclass, int dhint = 0) {
    w.need(ph);
    // mixed precision: the products of Alg 1 (FC_GEMM) and the rebuild products of a rounded
    // addition (overwrite, not symmetric) run in FP32; with tensor cores, those with at least
    // TC_MIN_ROWS static rows (a 128-row MMA tile mostly used) run on them. The Gram products
    // stay FP64 (their rounding sets the truncation's accuracy floor).
    if (mixed && !(flags & (GF_SYM_UPPER | GF_A_UPPER | GF_A_UNITLOWER)) &&
        (fclass == FC_GEMM || (fclass == FC_NONE && (flags & GF_OVERWRITE))))
      flags |= (mixed == 2 && !m.d && m.s >= TC_MIN_ROWS) ? GF_TF32 : GF_F32;
    // split static rows (always legal) and, for accumulating outputs, the static reduction
    int mstep = (m.d || m.s <= GEMM_MCHUNK) ? std::max(m.s, 1) : GEMM_MCHUNK;
    bool ksplit = (flags & GF_ATOMIC) && !k.d && k.s > GEMM_KCHUNK;
    int kstep = ksplit ? GEMM_KCHUNK : std::max(k.s, 1);
    for (int i0 = 0; i0 < std::max(m.s, 1); i0 += mstep) {
      int mi = m.d ? m.s : std::min(mstep, m.s - i0);
      for (int l0 = 0; l0 < std::max(k.s, 1); l0 += kstep) {
        int kl = k.d ? k.s : (ksplit ? std::min(kstep, k.s - l0) : k.s);
        GemmOp g;
        std::memset(&g, 0, sizeof(g));
        g.A = A + (uint64_t)(i0 * ars + l0 * acs);
        g.B = B + (uint64_t)(l0 * brs);
        g.C = C + (uint64_t)(i0 * crs);
        g.a_rs = ars;
        g.a_cs = acs;
        g.b_rs = brs;
        g.b_cs = bcs;
        g.c_rs = crs;
        g.c_cs = ccs;
        g.m = mi;
        g.md = m.d;
        g.n = n.s;
        g.nd = n.d;
        g.k = kl;
        g.kd = k.d;
        g.flags = flags;
        g.alpha = alpha;
        g.fclass = fclass;
        g.split = dhint;   // host-side hint until gemm_grid sets the split
        w.gemm[ph].push_back(g);
        if (k.d) break;
      }
      if (m.d) break;
    }
  }
  void copy(int ph, int mode, uint64_t src, int64_t srs, int64_t scs, uint64_t dst, int64_t drs, int64_t dcs,
            Dim m, Dim n, double alpha = 1.0) {
    w.need(ph);
    CopyOp c;
    std::memset(&c, 0, sizeof(c));
    c.src = src;
    c.s_rs = srs;
    c.s_cs = scs;
    c.dst = dst;
    c.d_rs = drs;
    c.d_cs = dcs;
    c.m = m.s;
    c.md = m.d;
    c.n = n.s;
    c.nd = n.d;
    c.mode = mode;
    c.alpha = alpha;
    w.copy[ph].push_back(c);
  }
  void trsm(int ph, int mode, const LeafStore& D, View X, Dim nv) {
    w.need(ph);
    int vstep = nv.d ? std::max(nv.s, 1) : TRSM_VCHUNK;
    for (int v0 = 0; v0 < std::max(nv.s, 1); v0 += vstep) {
      TrsmOp t;
      std::memset(&t, 0, sizeof(t));
      t.T = dref(D.off);
      t.piv = (mode == TM_L_PIV || mode == TM_MUL_PL) ? pref(D) : 0;
      t.X = X.ref + (uint64_t)(v0 * X.vs);
      t.x_es = X.es;
      t.x_vs = X.vs;
      t.nv = nv.d ? nv.s : std::min(vstep, nv.s - v0);
      t.nvd = nv.d;
      t.b = D.m;
      t.mode = mode;
      w.trsm[ph].push_back(t);
      if (nv.d) break;
    }
  }

  // Y[out] += alpha * op(M_node) X[in] for all leaves of the (sub-)block `nodeid`.
  // Phases: ph zero of temporaries, ph+1 partial products and dense leaves, ph+2 the
  // low-rank second factor. X must be final by ph+1; Y must be initialised by ph+1.
  // `filter`: 0 all leaves, 1 strictly upper, 2 strictly lower.
  int block_mv(int ph, int nodeid, View X, View Y, double alpha, bool trans, Dim nv, int nvmax,
               int filter = 0) {
    std::vector<int> leaves;
    collect_leaves(bt, nodeid, leaves);
    const BlockNode& N = node(nodeid);
    const int base_r = cl(N.row).lo, base_c = cl(N.col).lo;
    for (int lid : leaves) {
      const LeafStore& L = leaf_of(lid);
      const int r0 = cl(L.row).lo, c0 = cl(L.col).lo;
      if (filter == 1 && !(r0 < c0)) continue;
      if (filter == 2 && !(r0 > c0)) continue;
      const int ro = r0 - base_r, co = c0 - base_c;
      const View Xi = X.off(trans ? ro : co);
      const View Yo = Y.off(trans ? co : ro);
      if (!L.lr) {
        if (!trans)
          gemm(ph + 1, dref(L.off), 1, L.m, Xi.ref, Xi.es, Xi.vs, Yo.ref, Yo.es, Yo.vs, {L.m, 0}, nv, {L.n, 0},
               alpha, GF_ATOMIC, FC_GEMM);
        else
          gemm(ph + 1, dref(L.off), L.m, 1, Xi.ref, Xi.es, Xi.vs, Yo.ref, Yo.es, Yo.vs, {L.n, 0}, nv, {L.m, 0},
               alpha, GF_ATOMIC, FC_GEMM);
      } else {
        const int64_t T = w.alloc_d((int64_t)L.cap * nvmax);
        const Dim rk{0, rref(L)};
        // T = V^T X (or U^T X when transposed); a long reduction is split across CTAs and
        // accumulated atomically into a zeroed T, a short one is written directly
        const int64_t first = trans ? L.off : L.voff;
        const int ld1 = trans ? L.m : L.n;
        const bool split = ld1 > GEMM_KCHUNK;
        if (split) copy(ph, CM_ZERO, 0, 0, 0, sref(T), 1, L.cap, rk, nv);
        gemm(ph + 1, dref(first), ld1, 1, Xi.ref, Xi.es, Xi.vs, sref(T), 1, L.cap, rk, nv, {ld1, 0}, 1.0,
             split ? GF_ATOMIC : GF_OVERWRITE, FC_GEMM);
        const int64_t second = trans ? L.voff : L.off;
        const int ld2 = trans ? L.n : L.m;
        gemm(ph + 2, dref(second), 1, ld2, sref(T), 1, L.cap, Yo.ref, Yo.es, Yo.vs, {ld2, 0}, nv, rk, alpha,
             GF_ATOMIC, FC_GEMM);
      }
    }
    return ph + 3;
  }

  // ---------------------------------------------------------------- structured solves
  // X := L_tt^{-1} P^T X (rows of cluster t), block forward substitution (Alg 3 leaf case)
  int lsolve(int ph, int t, View X, Dim nv, int nvmax) {
    const int id = find(t, t);
    if (node(id).is_leaf()) {
      trsm(ph, TM_L_PIV, leaf_of(id), X, nv);
      return ph + 1;
    }
    const Cluster& C = cl(t);
    const int t0 = C.son0, t1 = C.son1;
    const int n0 = cl(t0).size();
    int p = lsolve(ph, t0, X, nv, nvmax);
    p = block_mv(p - 1, find(t1, t0), X, X.off(n0), -1.0, false, nv, nvmax);
    return lsolve(p, t1, X.off(n0), nv, nvmax);
  }
  // X := U_tt^{-T} X
  int utsolve(int ph, int t, View X, Dim nv, int nvmax) {
    const int id = find(t, t);
    if (node(id).is_leaf()) {
      trsm(ph, TM_UT, leaf_of(id), X, nv);
      return ph + 1;
    }
    const Cluster& C = cl(t);
    const int t0 = C.son0, t1 = C.son1;
    const int n0 = cl(t0).size();
    int p = utsolve(ph, t0, X, nv, nvmax);
    p = block_mv(p - 1, find(t0, t1), X, X.off(n0), -1.0, true, nv, nvmax);
    return utsolve(p, t1, X.off(n0), nv, nvmax);
  }
  // X := U_tt^{-1} X (backward substitution)
  int usolve(int ph, int t, View X, Dim nv, int nvmax) {
    const int id = find(t, t);
    if (node(id).is_leaf()) {
      trsm(ph, TM_U, leaf_of(id), X, nv);
      return ph + 1;
    }
    const Cluster& C = cl(t);
    const int t0 = C.son0, t1 = C.son1;
    const int n0 = cl(t0).size();
    int p = usolve(ph, t1, X.off(n0), nv, nvmax);
    p = block_mv(p - 1, find(t0, t1), X.off(n0), X, -1.0, false, nv, nvmax);
    return usolve(p, t0, X, nv, nvmax);
  }

  // ---------------------------------------------------------------- tasks
  void task_lu(int t) {
    const int id = find(t, t);
    const LeafStore& L = leaf_of(id);
    w.need(0);
    GetrfOp g;
    std::memset(&g, 0, sizeof(g));
    g.A = dref(L.off);
    g.piv = pref(L);
    g.b = L.m;
    w.getrf[0].push_back(g);
  }
  void task_trsl(int t, int s) {   // L_tt X_ts = M_ts, (t, s) a leaf block
    const LeafStore& M = leaf_of(find(t, s));
    if (M.lr)
      lsolve(0, t, View{dref(M.off), 1, M.m}, Dim{0, rref(M)}, M.cap);
    else
      lsolve(0, t, View{dref(M.off), 1, M.m}, Dim{M.n, 0}, M.n);
  }
  void task_trsu(int t, int s) {   // X_st U_tt = M_st, (s, t) a leaf block
    const LeafStore& M = leaf_of(find(s, t));
    if (M.lr)
      utsolve(0, t, View{dref(M.voff), 1, M.n}, Dim{0, rref(M)}, M.cap);
    else   // rows of M^T: element e (of t) of vector v (of s) is M[v + e*ld]
      utsolve(0, t, View{dref(M.off), M.m, 1}, Dim{M.m, 0}, M.m);
  }

  uint64_t identity(int k) {
    const uint64_t I = palloc((int64_t)k * k);
    copy(0, CM_IDENTITY, 0, 0, 0, I, 1, k, {k, 0}, {k, 0});
    return I;
  }

  // pieces of A_ab B_bc (relative offsets ro, co inside the target) -- phases 0..2
  void product_pieces(int An, int Bn, int ro, int co, std::vector<Piece>& out) {
    const BlockNode& A = node(An);
    const BlockNode& B = node(Bn);
    const int a = A.row, b = A.col, c = B.col;
    const int ma = cl(a).size(), mb = cl(b).size(), mc = cl(c).size();
    const bool Aleaf = A.is_leaf(), Bleaf = B.is_leaf();
    if (Aleaf && leaf_of(An).lr) {
      const LeafStore& LA = leaf_of(An);
      const uint64_t Z = palloc((int64_t)mc * LA.cap);
      copy(0, CM_ZERO, 0, 0, 0, Z, 1, mc, {mc, 0}, {LA.cap, 0});
      block_mv(0, Bn, View{dref(LA.voff), 1, mb}, View{Z, 1, mc}, 1.0, true, {0, rref(LA)}, LA.cap);
      out.push_back({View{dref(LA.off), 1, ma}, View{Z, 1, mc}, {0, rref(LA)}, LA.cap, ro, ma, co, mc, -1.0});
      return;
    }
    if (Bleaf && leaf_of(Bn).lr) {
      const LeafStore& LB = leaf_of(Bn);
      const uint64_t W = palloc((int64_t)ma * LB.cap);
      copy(0, CM_ZERO, 0, 0, 0, W, 1, ma, {ma, 0}, {LB.cap, 0});
      block_mv(0, An, View{dref(LB.off), 1, mb}, View{W, 1, ma}, 1.0, false, {0, rref(LB)}, LB.cap);
      out.push_back({View{W, 1, ma}, View{dref(LB.voff), 1, mc}, {0, rref(LB)}, LB.cap, ro, ma, co, mc, -1.0});
      return;
    }
    if (Aleaf && Bleaf) {
      const LeafStore& LA = leaf_of(An);
      const LeafStore& LB = leaf_of(Bn);
      if (mb <= std::min(ma, mc)) {
        out.push_back({View{dref(LA.off), 1, ma}, View{dref(LB.off), mb, 1}, {mb, 0}, mb, ro, ma, co, mc, -1.0});
        return;
      }
      const uint64_t P = palloc((int64_t)ma * mc);
      copy(0, CM_ZERO, 0, 0, 0, P, 1, ma, {ma, 0}, {mc, 0});
      gemm(1, dref(LA.off), 1, ma, dref(LB.off), 1, mb, P, 1, ma, {ma, 0}, {mc, 0}, {mb, 0}, 1.0, GF_ATOMIC,
           FC_GEMM);
      if (ma <= mc) {
        const uint64_t I = identity(ma);
        out.push_back({View{I, 1, ma}, View{P, ma, 1}, {ma, 0}, ma, ro, ma, co, mc, -1.0});
      } else {
        const uint64_t I = identity(mc);
        out.push_back({View{P, 1, ma}, View{I, 1, mc}, {mc, 0}, mc, ro, ma, co, mc, -1.0});
      }
      return;
    }
    if (Aleaf) {   // A dense with a leaf row cluster, B structured: (I, B^T A^T)
      const LeafStore& LA = leaf_of(An);
      const uint64_t S = palloc((int64_t)ma * mc);
      copy(0, CM_ZERO, 0, 0, 0, S, 1, ma, {ma, 0}, {mc, 0});
      block_mv(0, Bn, View{dref(LA.off), ma, 1}, View{S, ma, 1}, 1.0, true, {ma, 0}, ma);
      const uint64_t I = identity(ma);
      out.push_back({View{I, 1, ma}, View{S, ma, 1}, {ma, 0}, ma, ro, ma, co, mc, -1.0});
      return;
    }
    if (Bleaf) {   // B dense with a leaf column cluster, A structured: (A B, I)
      const LeafStore& LB = leaf_of(Bn);
      const uint64_t S = palloc((int64_t)ma * mc);
      copy(0, CM_ZERO, 0, 0, 0, S, 1, ma, {ma, 0}, {mc, 0});
      block_mv(0, An, View{dref(LB.off), 1, mb}, View{S, 1, ma}, 1.0, false, {mc, 0}, mc);
      const uint64_t I = identity(mc);
      out.push_back({View{S, 1, ma}, View{I, 1, mc}, {mc, 0}, mc, ro, ma, co, mc, -1.0});
      return;
    }
    const Cluster& Ca = cl(a);
    const Cluster& Cb = cl(b);
    const Cluster& Cc = cl(c);
    const int as[2] = {Ca.son0, Ca.son1}, bs[2] = {Cb.son0, Cb.son1}, cs[2] = {Cc.son0, Cc.son1};
    for (int i = 0; i < 2; ++i)
      for (int j = 0; j < 2; ++j)
        for (int l = 0; l < 2; ++l)
          product_pieces(find(as[i], bs[l]), find(bs[l], cs[j]), ro + cl(as[i]).lo - Ca.lo,
                         co + cl(cs[j]).lo - Cc.lo, out);
  }

  // dense target: C += alpha A B accumulated directly -- phases 0..3
  void product_dense(int An, int Bn, const LeafStore& C, double alpha) {
    const BlockNode& A = node(An);
    const BlockNode& B = node(Bn);
    const int a = A.row, b = A.col, c = B.col;
    const int ma = cl(a).size(), mb = cl(b).size(), mc = cl(c).size();
    const View Cv{dref(C.off), 1, C.m};
    if (A.is_leaf() && leaf_of(An).lr) {
      const LeafStore& LA = leaf_of(An);
      const int64_t Z = w.alloc_d((int64_t)mc * LA.cap);
      copy(0, CM_ZERO, 0, 0, 0, sref(Z), 1, mc, {mc, 0}, {LA.cap, 0});
      block_mv(0, Bn, View{dref(LA.voff), 1, mb}, View{sref(Z), 1, mc}, 1.0, true, {0, rref(LA)}, LA.cap);
      gemm(3, dref(LA.off), 1, ma, sref(Z), mc, 1, Cv.ref, 1, C.m, {ma, 0}, {mc, 0}, {0, rref(LA)}, alpha,
           GF_ATOMIC, FC_GEMM);
      return;
    }
    if (B.is_leaf() && leaf_of(Bn).lr) {
      const LeafStore& LB = leaf_of(Bn);
      const int64_t W = w.alloc_d((int64_t)ma * LB.cap);
      copy(0, CM_ZERO, 0, 0, 0, sref(W), 1, ma, {ma, 0}, {LB.cap, 0});
      block_mv(0, An, View{dref(LB.off), 1, mb}, View{sref(W), 1, ma}, 1.0, false, {0, rref(LB)}, LB.cap);
      gemm(3, sref(W), 1, ma, dref(LB.voff), mc, 1, Cv.ref, 1, C.m, {ma, 0}, {mc, 0}, {0, rref(LB)}, alpha,
           GF_ATOMIC, FC_GEMM);
      return;
    }
    if (A.is_leaf() && B.is_leaf()) {
      gemm(1, dref(leaf_of(An).off), 1, ma, dref(leaf_of(Bn).off), 1, mb, Cv.ref, 1, C.m, {ma, 0}, {mc, 0},
           {mb, 0}, alpha, GF_ATOMIC, FC_GEMM);
      return;
    }
    if (A.is_leaf()) {   // C^T += alpha B^T A^T
      const LeafStore& LA = leaf_of(An);
      block_mv(0, Bn, View{dref(LA.off), ma, 1}, View{Cv.ref, C.m, 1}, alpha, true, {ma, 0}, ma);
      return;
    }
    if (B.is_leaf()) {
      const LeafStore& LB = leaf_of(Bn);
      block_mv(0, An, View{dref(LB.off), 1, mb}, Cv, alpha, false, {mc, 0}, mc);
      return;
    }
    throw std::runtime_error("planner: dense target with two structured operands");
  }

  void add_entry(int leafidx, const Piece& p, int row_off, int nrows, int col_off, int ncols, int wrow,
                 int zrow) {
    StackEntry e;
    std::memset(&e, 0, sizeof(e));
    e.W = p.W.ref + (uint64_t)(wrow * p.W.es);
    e.w_rs = p.W.es;
    e.w_cs = p.W.vs;
    e.Z = p.Z.ref + (uint64_t)(zrow * p.Z.es);
    e.z_rs = p.Z.es;
    e.z_cs = p.Z.vs;
    e.k = p.k.s;
    e.kd = p.k.d;
    e.row_off = row_off;
    e.nrows = nrows;
    e.col_off = col_off;
    e.ncols = ncols;
    e.alpha = p.alpha;
    auto it = target_index.find(leafidx);
    int ti;
    if (it == target_index.end()) {
      ti = (int)targets.size();
      target_index[leafidx] = ti;
      targets.push_back({leafidx, {}});
    } else {
      ti = it->second;
    }
    targets[ti].e.push_back({e, p.kmax});
  }

  // apply the pieces (relative to the origin of block Cn) to the leaves of Cn -- phase 3
  void apply_pieces(int Cn, const std::vector<Piece>& pieces) {
    std::vector<int> leaves;
    collect_leaves(bt, Cn, leaves);
    const BlockNode& C = node(Cn);
    const int br = cl(C.row).lo, bc = cl(C.col).lo;
    for (int lid : leaves) {
      const LeafStore& L = leaf_of(lid);
      const int lr0 = cl(L.row).lo - br, lr1 = lr0 + L.m;
      const int lc0 = cl(L.col).lo - bc, lc1 = lc0 + L.n;
      for (const Piece& p : pieces) {
        const int ir0 = std::max(p.ro, lr0), ir1 = std::min(p.ro + p.nrows, lr1);
        const int ic0 = std::max(p.co, lc0), ic1 = std::min(p.co + p.ncols, lc1);
        if (ir0 >= ir1 || ic0 >= ic1) continue;
        if (!L.lr) {
          const View Wv = p.W.off(ir0 - p.ro), Zv = p.Z.off(ic0 - p.co);
          const uint64_t Cref = dref(L.off) + (uint64_t)((ir0 - lr0) + (int64_t)(ic0 - lc0) * L.m);
          gemm(3, Wv.ref, Wv.es, Wv.vs, Zv.ref, Zv.vs, Zv.es, Cref, 1, L.m, {ir1 - ir0, 0}, {ic1 - ic0, 0}, p.k,
               p.alpha, GF_ATOMIC, FC_GEMM);
        } else {
          add_entry(bt.nodes[lid].leaf, p, ir0 - lr0, ir1 - ir0, ic0 - lc0, ic1 - ic0, ir0 - p.ro, ic0 - p.co);
        }
      }
    }
  }

  void task_mul(int t, int r, int s) {
    const int An = find(t, r), Bn = find(r, s), Cn = find(t, s);
    const BlockNode& C = node(Cn);
    if (C.is_leaf() && !leaf_of(Cn).lr) {
      product_dense(An, Bn, leaf_of(Cn), -1.0);
      return;
    }
    std::vector<Piece> pieces;
    piece_release = -1;
    if (events) {   // accumulator H-LU: pieces held past this wave live in the arena
      std::vector<int> leaves;
      collect_leaves(bt, Cn, leaves);
      for (int lid : leaves) {
        const int leaf = bt.nodes[lid].leaf;
        if (!lay.leaf[leaf].lr) continue;
        const int f = flush_level(leaf, level);
        // the rounded addition of wave f may run beside wave f + 1: free from wave f + 2 on
        if (f > level) piece_release = std::max(piece_release, f + 2);
      }
    }
    product_pieces(An, Bn, 0, 0, pieces);
    piece_release = -1;
    apply_pieces(Cn, pieces);
  }

  // the targets whose rounded addition can wait for the side stream (defer(leaf) true) are
  // moved out of `targets` into `out`
  template <class F>
  void take_deferred(F defer, std::vector<TargetEntries>& out) {
    std::vector<TargetEntries> keep;
    for (TargetEntries& T : targets) (defer(T.leaf) ? out : keep).push_back(std::move(T));
    targets.swap(keep);
    target_index.clear();
    for (size_t q = 0; q < targets.size(); ++q) target_index[targets[q].leaf] = (int)q;
  }

  // rounded additions of all pieces that reached low-rank leaves in this wave. A target whose
  // pieces and own factors fit one stack (KMAX_STACK columns by static rank bounds) is one
  // rounded addition. A larger one is either updated in sequential rounds (chunk r + 1 stacked
  // on the result of chunk r) or, when that takes more levels, as a tree: stacks of pieces are
  // rounded in parallel into temporary low-rank sums (groups: stacks without the target's own
  // factors, TF_NOSELF), those are combined the same way level by level, and the last level adds
  // the target's own factors and at most the remaining sums; rounded additions of one level are
  // independent. The rounded additions of one level run in batches whose scratch fits `budget`;
  // every batch reuses the same scratch region (they are sequential phases), so a wave's scratch
  // is its product temporaries, the groups' sums and one batch.
  void emit_truncations(int ph0, double eps, bool target_rank_zero = false, int64_t budget = (int64_t)1 << 29) {
    plan.scratch_products_max = std::max(plan.scratch_products_max, w.sd);
    struct Group {
      uint64_t U, V, rank;   // the temporary sum (ld m and n, cap columns) and its rank
    };
    struct Job {
      int target;            // index into targets: the leaf whose shape the stack has
      bool self;             // the stack starts with the output's own factors
      int out;               // -1: the leaf; else a group
      std::vector<std::pair<StackEntry, int>> e;   // pieces with static rank bounds
      int sum;               // static stacked rank
    };
    std::vector<Group> groups;
    std::vector<std::vector<Job>> levels;
    auto level = [&](size_t lv) -> std::vector<Job>& {
      if (levels.size() <= lv) levels.resize(lv + 1);
      return levels[lv];
    };
    // greedy chunks of es with static sums <= room and at most KMAX_ENTRIES pieces
    auto chunks = [&](const std::vector<std::pair<StackEntry, int>>& es, int room) {
      std::vector<std::pair<size_t, size_t>> out;
      size_t e0 = 0;
      while (e0 < es.size()) {
        int sum = 0;
        size_t e1 = e0;
        while (e1 < es.size() && e1 - e0 < (size_t)KMAX_ENTRIES && (e1 == e0 || sum + es[e1].second <= room)) {
          sum += es[e1].second;
          ++e1;
        }
        if (sum > room) throw std::runtime_error("planner: piece rank exceeds the stack limit");
        out.push_back({e0, e1});
        e0 = e1;
      }
      return out;
    };
    // a temporary sum as a piece of the next level's stacks
    auto group_entry = [&](const Group& g, const LeafStore& L) {
      StackEntry e;
      std::memset(&e, 0, sizeof(e));
      e.W = g.U;
      e.w_rs = 1;
      e.w_cs = L.m;
      e.Z = g.V;
      e.z_rs = 1;
      e.z_cs = L.n;
      e.k = 0;
      e.kd = g.rank;
      e.row_off = 0;
      e.nrows = L.m;
      e.col_off = 0;
      e.ncols = L.n;
      e.alpha = 1.0;
      return std::make_pair(e, L.cap);
    };
    for (size_t ti = 0; ti < targets.size(); ++ti) {
      const TargetEntries& T = targets[ti];
      const LeafStore& L = lay.leaf[T.leaf];
      // sequential rounds: the first with the target's static rank (0 for an empty target)
      std::vector<std::pair<size_t, size_t>> seq;
      std::vector<int> seq_sum;
      {
        size_t e0 = 0;
        for (int round = 0; e0 < T.e.size(); ++round) {
          const int selfmax = (target_rank_zero && round == 0) ? 0 : L.cap;
          int sum = selfmax;
          size_t e1 = e0;
          while (e1 < T.e.size() && e1 - e0 < (size_t)KMAX_ENTRIES &&
                 (e1 == e0 || sum + T.e[e1].second <= KMAX_STACK)) {
            sum += T.e[e1].second;
            ++e1;
          }
          if (sum > KMAX_STACK) throw std::runtime_error("planner: piece rank exceeds the stack limit");
          seq.push_back({e0, e1});
          seq_sum.push_back(sum);
          e0 = e1;
        }
      }
      // tree: the groups of the pieces, the levels that combine sums, the last stack
      const int capk = std::max(1, L.cap);
      const int per = std::max(1, std::min(KMAX_ENTRIES, KMAX_STACK / capk));
      const int last = std::max(0, (KMAX_STACK - (target_rank_zero ? 0 : L.cap)) / capk);
      int tree = 2;
      {
        int r = (int)chunks(T.e, KMAX_STACK).size();
        while (r > last) {
          r = (r + per - 1) / per;
          ++tree;
        }
      }
      if ((int)seq.size() <= tree || last < 1) {
        for (size_t q = 0; q < seq.size(); ++q) {
          Job j{(int)ti, true, -1, {T.e.begin() + seq[q].first, T.e.begin() + seq[q].second}, seq_sum[q]};
          level(q).push_back(std::move(j));
        }
        continue;
      }
      std::vector<std::pair<StackEntry, int>> cur = T.e;
      size_t lv = 0;
      for (;;) {
        const auto ch = chunks(cur, KMAX_STACK);
        std::vector<std::pair<StackEntry, int>> next;
        for (const auto& c : ch) {
          Group g;
          g.U = sref(w.alloc_d((int64_t)L.m * L.cap));
          g.V = sref(w.alloc_d((int64_t)L.n * L.cap));
          g.rank = mkref(sis, w.alloc_i(1));
          Job j{(int)ti, false, (int)groups.size(), {cur.begin() + c.first, cur.begin() + c.second}, 0};
          for (const auto& pe : j.e) j.sum += pe.second;
          groups.push_back(g);
          level(lv).push_back(std::move(j));
          next.push_back(group_entry(groups.back(), L));
        }
        cur.swap(next);
        ++lv;
        if ((int)cur.size() <= last) break;
      }
      Job j{(int)ti, true, -1, cur, target_rank_zero ? 0 : L.cap};
      for (const auto& pe : cur) j.sum += pe.second;
      level(lv).push_back(std::move(j));
    }
    const int64_t base = w.sd;   // after the groups' sums, which live through all levels
    int batch = 0;
    int64_t peak = 0;
    for (const auto& rd : levels) {
      w.sd = base;
      bool opened = false;
      for (const Job& jb : rd) {
        const LeafStore& L = lay.leaf[targets[jb.target].leaf];
        const int Kc = std::max(2, (jb.sum + 1) / 2 * 2);
        const int64_t need = (int64_t)(L.m + L.n) * Kc + 4 * (int64_t)Kc * Kc + 2 * (int64_t)Kc * L.cap + 8 * ALIGN;
        if (opened && w.sd + need - base > budget) {
          ++batch;
          w.sd = base;
        }
        opened = true;
        const int ph = ph0 + 4 * batch;
        w.need(ph + 3);
        TruncOp op;
        std::memset(&op, 0, sizeof(op));
        if (jb.out < 0) {
          op.U = dref(L.off);
          op.V = dref(L.voff);
          op.rank = rref(L);
        } else {
          op.U = groups[jb.out].U;
          op.V = groups[jb.out].V;
          op.rank = groups[jb.out].rank;
          op.flags = TF_NOSELF;
        }
        op.m = L.m;
        op.n = L.n;
        op.cap = L.cap;
        op.Kcap = Kc;
        op.Wst = sref(w.alloc_d((int64_t)L.m * Kc));
        op.Zst = sref(w.alloc_d((int64_t)L.n * Kc));
        op.Gw = sref(w.alloc_d((int64_t)Kc * Kc));
        op.Gz = sref(w.alloc_d((int64_t)Kc * Kc));
        op.Tw = sref(w.alloc_d((int64_t)Kc * L.cap));
        op.Tz = sref(w.alloc_d((int64_t)Kc * L.cap));
        op.work = sref(w.alloc_d(2 * (int64_t)Kc * Kc));
        op.Kd = mkref(sis, w.alloc_i(1));
        op.eps = eps;
        peak = std::max(peak, w.sd);
        std::vector<StackEntry> es;
        for (const auto& pe : jb.e) es.push_back(pe.first);
        w.stack[ph].push_back(op);
        w.stack_entries[ph].push_back(es);
        const Dim Kd{0, op.Kd};
        for (int i0 = 0; i0 < L.m; i0 += GEMM_KCHUNK) {
          int mi = std::min(GEMM_KCHUNK, L.m - i0);
          gemm(ph + 1, op.Wst + (uint64_t)i0, L.m, 1, op.Wst + (uint64_t)i0, 1, L.m, op.Gw, 1, Kc, Kd, Kd,
               {mi, 0}, 1.0, GF_ATOMIC | GF_SYM_UPPER, FC_NONE, Kc);
        }
        for (int i0 = 0; i0 < L.n; i0 += GEMM_KCHUNK) {
          int ni = std::min(GEMM_KCHUNK, L.n - i0);
          gemm(ph + 1, op.Zst + (uint64_t)i0, L.n, 1, op.Zst + (uint64_t)i0, 1, L.n, op.Gz, 1, Kc, Kd, Kd,
               {ni, 0}, 1.0, GF_ATOMIC | GF_SYM_UPPER, FC_NONE, Kc);
        }
        w.core[ph + 2].push_back(op);
        const Dim rk{0, op.rank};
        gemm(ph + 3, op.Wst, 1, L.m, op.Tw, 1, Kc, op.U, 1, L.m, {L.m, 0}, rk, Kd, 1.0, GF_OVERWRITE, FC_NONE, Kc);
        gemm(ph + 3, op.Zst, 1, L.n, op.Tz, 1, Kc, op.V, 1, L.n, {L.n, 0}, rk, Kd, 1.0, GF_OVERWRITE, FC_NONE, Kc);
        plan.ntrunc++;
      }
      if (opened) ++batch;
    }
    w.sd = std::max(base, peak);
    plan.scratch_trunc_max = std::max(plan.scratch_trunc_max, w.sd - base);
    targets.clear();
    target_index.clear();
  }

  // append the wave's phases to the plan in execution order
  void flush() {
    std::unordered_map<uint64_t, std::pair<int, int>> entry_range;
    for (int ph = 0; ph < w.nph; ++ph) {
      if ((int)w.gemm.size() <= ph) break;
      bool first = true;   // the next launch put is the phase's first
      auto put = [&](int kind, int count, int begin) {
        if (count > 0) {
          Launch L{kind, begin, count};
          L.first = first ? 1 : 0;
          L.wave = level;
          L.side = ph >= side_from ? 1 : 0;
          first = false;
          plan.launches.push_back(L);
        }
      };
      put(K_GETRF, (int)w.getrf[ph].size(), (int)plan.getrf.size());
      plan.getrf.insert(plan.getrf.end(), w.getrf[ph].begin(), w.getrf[ph].end());
      put(K_EVAL, (int)w.eval[ph].size(), (int)plan.eval.size());
      plan.eval.insert(plan.eval.end(), w.eval[ph].begin(), w.eval[ph].end());
      put(K_ACA, (int)w.aca[ph].size(), (int)plan.aca.size());
      plan.aca.insert(plan.aca.end(), w.aca[ph].begin(), w.aca[ph].end());
      put(K_COPY, (int)w.copy[ph].size(), (int)plan.copy.size());
      plan.copy.insert(plan.copy.end(), w.copy[ph].begin(), w.copy[ph].end());
      put(K_TRSM, (int)w.trsm[ph].size(), (int)plan.trsm.size());
      if (!w.trsm[ph].empty()) {
        // CTAs per micro-op along its vectors (chunks of 32; a dynamic count is taken as 64)
        int most = 0;
        for (const TrsmOp& op : w.trsm[ph]) most = std::max(most, op.nv + (op.nvd ? 64 : 0));
        plan.launches.back().gy = std::min(16, std::max(1, (most + 31) / 32));
      }
      plan.trsm.insert(plan.trsm.end(), w.trsm[ph].begin(), w.trsm[ph].end());
      {
        // FP64 micro-ops, then FP32, then tensor-core ones (independent: same phase)
        std::vector<GemmOp>& g = w.gemm[ph];
        const auto m32 = std::stable_partition(g.begin(), g.end(),
                                               [](const GemmOp& o) { return !(o.flags & (GF_TF32 | GF_F32)); });
        const auto mid = std::stable_partition(m32, g.end(), [](const GemmOp& o) { return !(o.flags & GF_TF32); });
        const int n64 = (int)(m32 - g.begin()), n32 = (int)(mid - m32), ntc = (int)(g.end() - mid);
        put(K_GEMM, n64, (int)plan.gemm.size());
        if (n64 > 0) {
          GemmOp* out = plan.gemm.extend(n64);
          gemm_grid_to(g.data(), n64, out, plan.launches.back().gy, plan.launches.back().gz);
        }
        put(K_GEMM32, n32, (int)plan.gemm.size());
        if (n32 > 0) {
          GemmOp* out = plan.gemm.extend(n32);
          gemm_grid_to(&*m32, n32, out, plan.launches.back().gy, plan.launches.back().gz);
        }
        if (ntc > 0) {
          // one persistent launch: every CTA computes whole micro-ops (all their C tiles)
          put(K_GEMM_TC, ntc, (int)plan.gemm.size());
          plan.gemm.append(&*mid, ntc);
        }
      }
      if (!w.stack[ph].empty()) {
        put(K_STACK, (int)w.stack[ph].size(), (int)plan.trunc.size());
        // CTAs per rounded addition along the rows: ~16k copied doubles each, at most 32
        int64_t most = 0;
        for (const TruncOp& op : w.stack[ph]) most = std::max(most, (int64_t)(op.m + op.n) * op.Kcap);
        plan.launches.back().gy = (int)std::min<int64_t>(32, std::max<int64_t>(1, most / 16384));
        for (size_t q = 0; q < w.stack[ph].size(); ++q) {
          TruncOp op = w.stack[ph][q];
          op.first_entry = (int)plan.entries.size();
          op.n_entries = (int)w.stack_entries[ph][q].size();
          entry_range[op.Kd] = {op.first_entry, op.n_entries};
          plan.entries.insert(plan.entries.end(), w.stack_entries[ph][q].begin(), w.stack_entries[ph][q].end());
          plan.trunc.push_back(op);
        }
      }
      // the core of a rounded addition reads its pieces' ranks (flop model): same entry range as
      // its stack record (a later phase of this wave; the stacked-rank slot Kd identifies it)
      for (TruncOp& op : w.core[ph]) {
        const auto it = entry_range.find(op.Kd);
        if (it != entry_range.end()) {
          op.first_entry = it->second.first;
          op.n_entries = it->second.second;
        }
      }
      // the cores of a launch are independent: largest stacked-rank bound first, so that the
      // longest ones start first
      std::stable_sort(w.core[ph].begin(), w.core[ph].end(),
                       [](const TruncOp& a, const TruncOp& b) { return a.Kcap > b.Kcap; });
      put(K_CORE, (int)w.core[ph].size(), (int)plan.trunc.size());
      plan.trunc.insert(plan.trunc.end(), w.core[ph].begin(), w.core[ph].end());
    }
    plan.nphases += w.nph;
    side_from = 1 << 30;
    plan.scratch_doubles = std::max(plan.scratch_doubles, w.sd);
    plan.scratch_ints = std::max(plan.scratch_ints, w.si);
    plan.nwaves++;
    w.reset();
    targets.clear();
    target_index.clear();
  }
};

}  // namespace

// ------------------------------------------------------------------------------ layout
void build_layout(const ClusterTree& ct, const BlockTree& bt, int rank_cap, Layout& lay) {
  lay = Layout();
  lay.rank_cap = rank_cap;
  lay.leaf.resize(bt.leaves.size());
  int64_t off = 0;
  for (size_t q = 0; q < bt.leaves.size(); ++q) {
    const BlockNode& b = bt.nodes[bt.leaves[q]];
    LeafStore& L = lay.leaf[q];
    L.node = bt.leaves[q];
    L.row = b.row;
    L.col = b.col;
    L.m = ct.cl[b.row].size();
    L.n = ct.cl[b.col].size();
    L.lr = b.adm;
    if (L.lr) {
      L.cap = std::min(rank_cap, std::min(L.m, L.n));
      L.off = off;
      off += align_up((int64_t)L.m * L.cap);
      L.voff = off;
      off += align_up((int64_t)L.n * L.cap);
      L.rank_idx = lay.nranks++;
    } else {
      L.off = off;
      off += align_up((int64_t)L.m * L.n);
      if (b.row == b.col) {
        L.piv_off = lay.npiv;
        lay.npiv += L.m;
      }
    }
  }
  lay.nvalues = off;
}

// ------------------------------------------------------------------------------ H-LU
namespace {
void expand_task(Ctx& c, const Task& t) {
  switch (t.type) {
    case T_LU: c.task_lu(t.a); break;
    case T_TRSL: c.task_trsl(t.a, t.b); break;
    case T_TRSU: c.task_trsu(t.a, t.b); break;
    default: c.task_mul(t.a, t.b, t.c); break;
  }
  c.plan.ntasks++;
}
std::vector<std::vector<int>> by_level(const TaskGraph& g) {
  std::vector<std::vector<int>> byl(g.nlevels);
  for (size_t i = 0; i < g.nodes.size(); ++i) byl[g.level[i]].push_back((int)i);
  return byl;
}

// Appends the plans of consecutive wave ranges to `plan` in order: launch begins and the
// entry ranges of stack records are made global, counters summed, scratch sizes maximised.
// The copies of the parts run in parallel (each part has its own destination range).
void concat_plans(std::vector<Plan>& parts, Plan& plan, int threads) {
  const size_t np = parts.size();
  struct Off {
    size_t getrf, trsm, gemm, copy, trunc, entries, eval, aca, launches;
  };
  std::vector<Off> off(np + 1);
  off[0] = {plan.getrf.size(), plan.trsm.size(), plan.gemm.size(), plan.copy.size(), plan.trunc.size(),
            plan.entries.size(), plan.eval.size(), plan.aca.size(), plan.launches.size()};
  for (size_t k = 0; k < np; ++k) {
    const Plan& q = parts[k];
    off[k + 1] = {off[k].getrf + q.getrf.size(), off[k].trsm + q.trsm.size(),     off[k].gemm + q.gemm.size(),
                  off[k].copy + q.copy.size(),   off[k].trunc + q.trunc.size(),   off[k].entries + q.entries.size(),
                  off[k].eval + q.eval.size(),   off[k].aca + q.aca.size(),       off[k].launches + q.launches.size()};
  }
  const Off& end = off[np];
  plan.getrf.extend(end.getrf - off[0].getrf);
  plan.trsm.extend(end.trsm - off[0].trsm);
  plan.gemm.extend(end.gemm - off[0].gemm);
  plan.copy.extend(end.copy - off[0].copy);
  plan.trunc.extend(end.trunc - off[0].trunc);
  plan.entries.extend(end.entries - off[0].entries);
  plan.eval.extend(end.eval - off[0].eval);
  plan.aca.extend(end.aca - off[0].aca);
  plan.launches.resize(end.launches);
  auto put = [&](size_t k) {
    const Plan& q = parts[k];
    const Off& o = off[k];
    auto cp = [](auto& dst, size_t at, const auto& src) {
      if (src.size()) std::memcpy(static_cast<void*>(dst.data() + at), src.data(), src.size() * sizeof(*src.data()));
    };
    cp(plan.getrf, o.getrf, q.getrf);
    cp(plan.trsm, o.trsm, q.trsm);
    cp(plan.gemm, o.gemm, q.gemm);
    cp(plan.copy, o.copy, q.copy);
    cp(plan.trunc, o.trunc, q.trunc);
    cp(plan.entries, o.entries, q.entries);
    cp(plan.eval, o.eval, q.eval);
    cp(plan.aca, o.aca, q.aca);
    for (size_t l = 0; l < q.launches.size(); ++l) {
      Launch L = q.launches[l];
      size_t base = 0;
      switch (L.kind) {
        case K_GETRF: base = o.getrf; break;
        case K_TRSM: base = o.trsm; break;
        case K_GEMM:
        case K_GEMM32:
        case K_GEMM_TC: base = o.gemm; break;
        case K_COPY: base = o.copy; break;
        case K_STACK:
        case K_CORE: base = o.trunc; break;
        case K_EVAL: base = o.eval; break;
        default: base = o.aca; break;
      }
      if (L.kind == K_STACK || L.kind == K_CORE)
        for (int r = 0; r < L.count; ++r) plan.trunc[base + L.begin + r].first_entry += (int)o.entries;
      L.begin += (int)base;
      plan.launches[o.launches + l] = L;
    }
  };
  std::atomic<size_t> next{0};
  run_workers(threads, [&]() {   // only copies: nothing here throws
    for (size_t k; (k = next.fetch_add(1)) < np;) put(k);
  });
  for (const Plan& q : parts) {
    plan.scratch_doubles = std::max(plan.scratch_doubles, q.scratch_doubles);
    plan.scratch_ints = std::max(plan.scratch_ints, q.scratch_ints);
    plan.scratch_products_max = std::max(plan.scratch_products_max, q.scratch_products_max);
    plan.scratch_trunc_max = std::max(plan.scratch_trunc_max, q.scratch_trunc_max);
    plan.nwaves += q.nwaves;
    plan.nphases += q.nphases;
    plan.ntasks += q.ntasks;
    plan.ntrunc += q.ntrunc;
    plan.deferred_truncations += q.deferred_truncations;
  }
}

int plan_threads(int threads) {
  if (threads > 0) return threads;
  const unsigned h = std::thread::hardware_concurrency();
  return (int)std::max(1u, std::min(h, 64u));
}

// Plans waves [0, nlev) with plan_range(part, lv0, lv1), which plans the waves [lv0, lv1) into
// `part` in order. Waves are planned independently (scratch and rounded-addition targets are
// per wave), so consecutive ranges, balanced by the tasks per wave, are planned on several
// threads and concatenated in order: the result equals planning all waves in one range.
template <class F>
void plan_wave_ranges(int nlev, const std::vector<size_t>& tasks_per_wave, int threads, F plan_range, Plan& plan) {
  threads = plan_threads(threads);
  if (threads == 1 || nlev < 64) {
    plan_range(plan, 0, nlev);
    return;
  }
  size_t total = 0;
  for (size_t t : tasks_per_wave) total += t;
  const int nparts = std::min(nlev, 8 * threads);
  std::vector<int> first(nparts + 1, nlev);
  {
    const double per = (double)total / nparts;
    int lv = 0;
    size_t done = 0;
    for (int k = 0; k < nparts; ++k) {
      first[k] = lv;
      while (lv < nlev && (done < (size_t)((k + 1) * per) || lv == first[k])) done += tasks_per_wave[lv++];
    }
    first[nparts] = nlev;
  }
  std::vector<Plan> parts(nparts);
  std::vector<std::string> errors(nparts);
  std::atomic<int> next{0};
  run_workers(threads, [&]() {
    for (int k; (k = next.fetch_add(1)) < nparts;) {
      try {
        plan_range(parts[k], first[k], first[k + 1]);
      } catch (const std::exception& ex) {
        errors[k] = ex.what();
      } catch (...) {
        errors[k] = "unknown error";
      }
    }
  });
  for (const std::string& e : errors)
    if (!e.empty()) throw std::runtime_error(e);
  concat_plans(parts, plan, threads);
}
}  // namespace

static LeafEvents leaf_events(const BlockTree& bt, const Layout& lay, const TaskGraph& g, int threads) {
  // ranges of tasks on the host threads, each into its own (leaf, level, read) list; the lists
  // are then gathered per leaf and sorted (the result does not depend on the thread count)
  const int nt = plan_threads(threads);
  const size_t N = g.nodes.size();
  const int nchunk = (int)std::max<size_t>(1, std::min<size_t>((size_t)nt * 4, N / 2048 + 1));
  std::vector<std::vector<std::array<int, 3>>> part(nchunk);
  std::atomic<int> next{0};
  run_workers(std::min(nt, nchunk), [&]() {
    std::vector<int> leaves;
    for (int k; (k = next.fetch_add(1)) < nchunk;) {
      auto& out = part[k];
      auto mark = [&](int r, int c, int lv, int read) {
        const int id = bt.find(r, c);
        if (id < 0) return;
        leaves.clear();
        collect_leaves(bt, id, leaves);
        for (int lid : leaves) out.push_back({bt.nodes[lid].leaf, lv, read});
      };
      for (size_t i = N * k / nchunk; i < N * (k + 1) / nchunk; ++i) {
        const Task& t = g.nodes[i];
        const int lv = g.level[i];
        switch (t.type) {
          case T_LU: mark(t.a, t.a, lv, 1); break;
          case T_TRSL: mark(t.a, t.b, lv, 1); break;
          case T_TRSU: mark(t.b, t.a, lv, 1); break;
          case T_SHIFT:
          case T_APPLY: mark(t.a, t.b, lv, 1); break;
          default:
            mark(t.a, t.b, lv, 1);
            mark(t.b, t.c, lv, 1);
            mark(t.a, t.c, lv, 0);
            break;
        }
      }
    }
  });
  LeafEvents out(lay.leaf.size());
  {
    std::vector<size_t> cnt(lay.leaf.size(), 0);
    for (const auto& p : part)
      for (const auto& e : p) ++cnt[e[0]];
    for (size_t l = 0; l < out.size(); ++l) out[l].reserve(cnt[l]);
    for (const auto& p : part)
      for (const auto& e : p) out[e[0]].push_back({e[1], e[2]});
  }
  for (auto& v : out) {
    std::sort(v.begin(), v.end());
    v.erase(std::unique(v.begin(), v.end()), v.end());
  }
  return out;
}

void plan_lu(const ClusterTree& ct, const BlockTree& bt, const Layout& lay, const TaskGraph& g, double eps,
             Plan& plan, int threads, int precision, bool defer, bool accumulate) {
  plan = Plan();
  const auto byl = by_level(g);
  std::vector<size_t> per(g.nlevels);
  for (int lv = 0; lv < g.nlevels; ++lv) per[lv] = byl[lv].size();
  LeafEvents events;
  if (defer || accumulate) events = leaf_events(bt, lay, g, threads);
  // a leaf is touched at a level when any task of that level reads or updates it
  auto touched_at = [&](int leaf, int lv) {
    const auto& v = events[leaf];
    auto it = std::lower_bound(v.begin(), v.end(), std::make_pair(lv, 0));
    return it != v.end() && it->first == lv;
  };
  Arena arena;
  plan_wave_ranges(
      g.nlevels, per, accumulate ? 1 : threads,
      [&](Plan& part, int lv0, int lv1) {
        Ctx c(ct, bt, lay, Spaces{SP_F, IS_RANK}, part);
        c.mixed = precision;
        if (accumulate) {
          c.events = &events;
          c.arena = &arena;
        }
        for (int lv = lv0; lv < lv1; ++lv) {
          c.level = lv;
          if (defer) {
            c.ss = (lv & 1) ? SP_S2 : SP_S;
            c.sis = (lv & 1) ? IS_S2 : IS_S;
          }
          if (accumulate) arena.release_until(lv);
          for (int ti : byl[lv]) expand_task(c, g.nodes[ti]);
          if (accumulate) c.hold_pending(lv);
          std::vector<TargetEntries> later;
          if (defer)   // not touched by the next wave: its rounded addition can overlap that wave
            c.take_deferred([&](int leaf) { return !touched_at(leaf, lv + 1); }, later);
          c.emit_truncations(3, eps);
          if (!later.empty()) {
            c.targets.swap(later);
            for (size_t q = 0; q < c.targets.size(); ++q) c.target_index[c.targets[q].leaf] = (int)q;
            c.side_from = c.w.nph;
            part.deferred_truncations += (int64_t)c.targets.size();
            c.emit_truncations(c.side_from, eps);
          }
          c.flush();
        }
        if (!c.pending.empty()) throw std::runtime_error("planner: accumulated updates never reached their leaf");
      },
      plan);
  plan.two_scratch = defer;
  plan.arena_doubles = arena.top;
}

void plan_lu_batch(const std::vector<LuInstance>& inst, double eps, Plan& plan, int threads, int precision) {
  plan = Plan();
  if (inst.empty()) return;
  std::vector<std::vector<std::vector<int>>> byl;
  int nlev = 0;
  for (const LuInstance& I : inst) {
    byl.push_back(by_level(*I.g));
    nlev = std::max(nlev, I.g->nlevels);
  }
  std::vector<size_t> per(nlev, 0);
  for (size_t i = 0; i < inst.size(); ++i)
    for (int lv = 0; lv < inst[i].g->nlevels; ++lv) per[lv] += byl[i][lv].size();
  plan_wave_ranges(
      nlev, per, threads,
      [&](Plan& part, int lv0, int lv1) {
        Wave w;
        std::vector<std::unique_ptr<Ctx>> cs;
        for (const LuInstance& I : inst) {
          cs.emplace_back(new Ctx(*I.ct, *I.bt, *I.lay, Spaces{SP_F, IS_RANK}, part, w));
          cs.back()->base_d = I.base_d;
          cs.back()->base_r = I.base_r;
          cs.back()->base_p = I.base_p;
          cs.back()->mixed = precision;
        }
        for (int lv = lv0; lv < lv1; ++lv) {
          for (size_t i = 0; i < inst.size(); ++i)
            if (lv < inst[i].g->nlevels)
              for (int ti : byl[i][lv]) expand_task(*cs[i], inst[i].g->nodes[ti]);
          // every instance's rounded additions of this wave share the phases after the products
          for (auto& c : cs) c->emit_truncations(3, eps);
          cs[0]->level = lv;
          cs[0]->flush();
        }
      },
      plan);
}

// ------------------------------------------------------------------------------ build
void plan_build(const ClusterTree& ct, const BlockTree& bt, const Layout& lay, double eps, int aca_kmax,
                int64_t scratch_budget, Plan& plan) {
  plan = Plan();
  Ctx c(ct, bt, lay, Spaces{SP_A, IS_ARANK}, plan);
  // dense leaves: one wave
  for (const LeafStore& L : lay.leaf)
    if (!L.lr) {
      c.w.need(0);
      EvalOp e{mkref(SP_A, L.off), ct.cl[L.row].lo, ct.cl[L.col].lo, L.m, L.n};
      c.w.eval[0].push_back(e);
    }
  c.flush();
  // admissible leaves: ACA into scratch, then a rounded truncation into the leaf; waves are
  // cut so that each stays within the scratch budget
  for (size_t q = 0; q < lay.leaf.size(); ++q) {
    const LeafStore& L = lay.leaf[q];
    if (!L.lr) continue;
    const int kmax = std::min(aca_kmax, std::min(L.m, L.n));
    const int Kc = (kmax + 1) / 2 * 2;
    int64_t need = (int64_t)(L.m + L.n) * kmax * 2 + 8 * (int64_t)Kc * Kc + 2 * (int64_t)Kc * L.cap + 256;
    if (c.w.sd > 0 && c.w.sd + need > scratch_budget) {
      c.emit_truncations(1, eps, true);
      c.flush();
    }
    c.w.need(0);
    AcaOp a;
    std::memset(&a, 0, sizeof(a));
    a.r0 = ct.cl[L.row].lo;
    a.c0 = ct.cl[L.col].lo;
    a.m = L.m;
    a.n = L.n;
    a.U = mkref(SP_S, c.w.alloc_d((int64_t)L.m * kmax));
    a.V = mkref(SP_S, c.w.alloc_d((int64_t)L.n * kmax));
    a.used = mkref(IS_S, c.w.alloc_i(L.m));
    a.kd = mkref(IS_S, c.w.alloc_i(1));
    a.kmax = kmax;
    a.tol = eps / 10.0;
    c.w.aca[0].push_back(a);
    Piece p{View{a.U, 1, L.m}, View{a.V, 1, L.n}, Dim{0, a.kd}, kmax, 0, L.m, 0, L.n, 1.0};
    c.add_entry((int)q, p, 0, L.m, 0, L.n, 0, 0);
  }
  if (!c.targets.empty() || c.w.nph > 0) {
    c.emit_truncations(1, eps, true);
    c.flush();
  }
}

// ------------------------------------------------------------------------------ solve
void plan_solve(const ClusterTree& ct, const BlockTree& bt, const Layout& lay, int nrhs_max, Plan& plan) {
  plan = Plan();
  Ctx c(ct, bt, lay, Spaces{SP_F, IS_RANK}, plan);
  const int n = ct.cl[0].size();
  const Dim nv{0, mkref(IS_S, c.w.alloc_i(1))};   // scratch int 0: number of right-hand sides
  const View X{mkref(SP_X, 0), 1, n};
  int p = c.lsolve(0, 0, X, nv, nrhs_max);
  c.usolve(p, 0, X, nv, nrhs_max);
  c.flush();
}

// ------------------------------------------------------------------------------ matvec
void plan_matvec(const ClusterTree& ct, const BlockTree& bt, const Layout& lay, int op, int nrhs_max,
                 Plan& plan) {
  plan = Plan();
  const int n = ct.cl[0].size();
  Ctx c(ct, bt, lay, op == 0 ? Spaces{SP_A, IS_ARANK} : Spaces{SP_F, IS_RANK}, plan);
  const Dim nv{0, mkref(IS_S, c.w.alloc_i(1))};
  auto col = [&](int blk) { return View{mkref(SP_X, (int64_t)blk * nrhs_max * n), 1, n}; };
  const View X = col(0), Y = col(1), Z = col(2), V = col(3);
  auto diag_apply = [&](int ph, int mode, View T) {
    for (const LeafStore& L : lay.leaf)
      if (!L.lr && L.row == L.col) c.trsm(ph, mode, L, T.off(ct.cl[L.row].lo), nv);
  };
  // out = tri(M) in: strictly-triangular leaves plus the diagonal leaves applied in place
  auto tri = [&](int ph, View in, View out, int mode, int filter) {
    c.copy(ph, CM_ZERO, 0, 0, 0, out.ref, 1, n, {n, 0}, nv);
    c.copy(ph, CM_COPY, in.ref, 1, n, V.ref, 1, n, {n, 0}, nv);
    diag_apply(ph + 1, mode, V);
    int p = c.block_mv(ph, 0, in, out, 1.0, false, nv, nrhs_max, filter);
    c.copy(p, CM_ADD, V.ref, 1, n, out.ref, 1, n, {n, 0}, nv);
    return p + 1;
  };
  if (op == 0) {
    c.copy(0, CM_ZERO, 0, 0, 0, Y.ref, 1, n, {n, 0}, nv);
    c.block_mv(0, 0, X, Y, 1.0, false, nv, nrhs_max);
  } else if (op == 1) {
    tri(0, X, Y, TM_MUL_PL, 2);
  } else if (op == 2) {
    tri(0, X, Y, TM_MUL_U, 1);
  } else {
    int p = tri(0, X, Z, TM_MUL_U, 1);
    tri(p, Z, Y, TM_MUL_PL, 2);
  }
  c.flush();
}

}  // namespace hm
