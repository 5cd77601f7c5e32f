// Cluster tree, block tree and the semi-automatic H-LU task graphs (host side).
// Paper: Def 2.1 (cluster tree), Def 2.2 (block tree), §5.1 (standard admissibility),
// Table 1 (task data dependencies), Def 3.2 (task relation), Alg 9-11 (refinement), Alg 13
// (its parallel loops), Alg 12 (edge sparsification), Table 2 and §4.3 (accumulator graphs).
#include "structure.h"

#include <algorithm>
#include <atomic>
#include <chrono>
#include <deque>
#include <exception>
#include <functional>
#include <mutex>
#include <thread>

namespace hm {

// ------------------------------------------------------------------ cluster tree (Def 2.1)
namespace {

struct CtBuilder {
  const double* p;
  int leaf_size;
  ClusterTree* ct;
  std::vector<int64_t> idx;   // working permutation; each cluster owns a contiguous range

  int build(int64_t lo, int64_t hi, int level, int parent) {
    int id = (int)ct->cl.size();
    ct->cl.emplace_back();
    {
      Cluster& c = ct->cl[id];
      c.lo = (int)lo;
      c.hi = (int)hi;
      c.level = level;
      c.parent = parent;
      for (int a = 0; a < 3; ++a) {
        c.bmin[a] = p[3 * idx[lo] + a];
        c.bmax[a] = p[3 * idx[lo] + a];
      }
      for (int64_t k = lo + 1; k < hi; ++k)
        for (int a = 0; a < 3; ++a) {
          double v = p[3 * idx[k] + a];
          if (v < c.bmin[a]) c.bmin[a] = v;
          if (v > c.bmax[a]) c.bmax[a] = v;
        }
    }
    if (level > ct->depth) ct->depth = level;
    if (hi - lo <= leaf_size) return id;
    double ext[3];
    int axis = 0;
    double mid;
    {
      const Cluster& c = ct->cl[id];
      for (int a = 0; a < 3; ++a) ext[a] = c.bmax[a] - c.bmin[a];
      for (int a = 1; a < 3; ++a)
        if (ext[a] > ext[axis]) axis = a;
      mid = 0.5 * (c.bmin[axis] + c.bmax[axis]);
    }
    auto first = idx.begin() + lo, last = idx.begin() + hi;
    auto split = std::stable_partition(first, last, [&](int64_t i) { return p[3 * i + axis] < mid; });
    int64_t nleft = split - first;
    if (nleft == 0 || nleft == hi - lo) {
      // median split in (coordinate, original index) order; each half in ascending index
      std::sort(first, last, [&](int64_t x, int64_t y) {
        double cx = p[3 * x + axis], cy = p[3 * y + axis];
        return cx < cy || (cx == cy && x < y);
      });
      nleft = (hi - lo) / 2;
      std::sort(first, first + nleft);
      std::sort(first + nleft, last);
    }
    int s0 = build(lo, lo + nleft, level + 1, id);
    int s1 = build(lo + nleft, hi, level + 1, id);
    ct->cl[id].son0 = s0;
    ct->cl[id].son1 = s1;
    return id;
  }
};

}  // namespace

void build_cluster_tree(const double* pts, int64_t n, int leaf_size, ClusterTree& ct) {
  ct = ClusterTree();
  ct.leaf_size = leaf_size;
  CtBuilder b{pts, leaf_size, &ct, {}};
  b.idx.resize(n);
  for (int64_t i = 0; i < n; ++i) b.idx[i] = i;
  if (n > 0) b.build(0, n, 0, -1);
  ct.perm = b.idx;
}

// ------------------------------------------------------------------ admissibility (§5.1)
static double diam2(const Cluster& c) {
  double e0 = c.bmax[0] - c.bmin[0];
  double e1 = c.bmax[1] - c.bmin[1];
  double e2 = c.bmax[2] - c.bmin[2];
  return e0 * e0 + e1 * e1 + e2 * e2;
}

static double dist2(const Cluster& t, const Cluster& s) {
  double d[3];
  for (int a = 0; a < 3; ++a) {
    double g = std::max(s.bmin[a] - t.bmax[a], t.bmin[a] - s.bmax[a]);
    d[a] = g > 0.0 ? g : 0.0;
  }
  return d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
}

bool admissible(const Cluster& t, const Cluster& s, double eta) {
  double dd = dist2(t, s);
  if (!(dd > 0.0)) return false;
  return std::min(diam2(t), diam2(s)) <= (eta * eta) * dd;
}

// ------------------------------------------------------------------ block tree (Def 2.2)
void build_block_tree(const ClusterTree& ct, double eta, BlockTree& bt) {
  bt = BlockTree();
  bt.ncl = (int)ct.cl.size();
  if (ct.cl.empty()) return;
  std::function<int(int, int)> rec = [&](int r, int c) -> int {
    int id = (int)bt.nodes.size();
    bt.nodes.emplace_back();
    bt.index[(uint64_t)r * (uint64_t)bt.ncl + (uint64_t)c] = id;
    const Cluster& t = ct.cl[r];
    const Cluster& s = ct.cl[c];
    bool adm = admissible(t, s, eta);
    bt.nodes[id].row = r;
    bt.nodes[id].col = c;
    bt.nodes[id].adm = adm;
    if (!adm && !t.leaf() && !s.leaf()) {
      int tr[2] = {t.son0, t.son1}, sc[2] = {s.son0, s.son1};
      for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j) {
          int child = rec(tr[i], sc[j]);
          bt.nodes[id].sons[2 * i + j] = child;
        }
    } else {
      bt.nodes[id].leaf = (int)bt.leaves.size();
      bt.leaves.push_back(id);
    }
    return id;
  };
  rec(0, 0);
}

void collect_leaves(const BlockTree& bt, int node, std::vector<int>& out) {
  const BlockNode& b = bt.nodes[node];
  if (b.is_leaf()) {
    out.push_back(node);
    return;
  }
  for (int q = 0; q < 4; ++q) collect_leaves(bt, b.sons[q], out);
}

// ------------------------------------------------------------------ task graph (§3.1, §3.2)
namespace {

// Matrix identifiers of H-LU; the accumulator of block-tree node b has identifier ID_ACC + b.
enum { ID_A = 0, ID_L = 1, ID_U = 2, ID_ACC = 3 };

struct Dep {
  int id, r, c;
};

struct DagBuilder {
  const ClusterTree& ct;
  const BlockTree& bt;
  const bool accu;               // accumulator H-LU (§3.2, Table 2) instead of Table 1
  std::vector<Task> tasks;
  std::vector<std::vector<int>> succ;
  std::vector<int> sub_first, sub_count;
  std::vector<int> acc_self, acc_par;   // accumulator ids of a task's block and of its parent block
  std::vector<int> parent_node;         // block-tree parent of each node, -1 at the root

  DagBuilder(const ClusterTree& c, const BlockTree& b, bool accumulators) : ct(c), bt(b), accu(accumulators) {
    range.reserve(ct.cl.size());
    for (const Cluster& x : ct.cl) range.emplace_back(x.lo, x.hi);
    if (accu) {
      parent_node.assign(bt.nodes.size(), -1);
      for (size_t i = 0; i < bt.nodes.size(); ++i)
        for (int q = 0; q < 4; ++q)
          if (bt.nodes[i].sons[q] >= 0) parent_node[bt.nodes[i].sons[q]] = (int)i;
    }
  }

  // Table 1 (and Table 2 in accumulator mode) with the identifiers H-LU passes (Alg 2 / Alg 3
  // and Alg 7 / Alg 8 arguments). T_MUL stands for hmul, or for add_upd in accumulator mode.
  int ins(int k, Dep* d) const {
    const Task& t = tasks[k];
    int n = 0;
    switch (t.type) {
      case T_LU: d[n++] = {ID_A, t.a, t.a}; break;
      case T_TRSL: d[n++] = {ID_L, t.a, t.a}; d[n++] = {ID_A, t.a, t.b}; break;
      case T_TRSU: d[n++] = {ID_U, t.a, t.a}; d[n++] = {ID_A, t.b, t.a}; break;
      case T_MUL: d[n++] = {ID_L, t.a, t.b}; d[n++] = {ID_U, t.b, t.c}; return n;
      default: d[n++] = {ID_ACC + acc_self[k], t.a, t.b}; break;   // shift_upd, apply_upd
    }
    if (accu && acc_par[k] >= 0) {
      int r = t.type == T_TRSU ? t.b : t.a, c = t.type == T_TRSU ? t.a : t.b;
      d[n++] = {ID_ACC + acc_par[k], r, c};
    }
    return n;
  }
  int outs(int k, Dep* d) const {
    const Task& t = tasks[k];
    switch (t.type) {
      case T_LU: d[0] = {ID_L, t.a, t.a}; d[1] = {ID_U, t.a, t.a}; return 2;
      case T_TRSL: d[0] = {ID_U, t.a, t.b}; return 1;
      case T_TRSU: d[0] = {ID_L, t.b, t.a}; return 1;
      case T_MUL:
        d[0] = {ID_A, t.a, t.c};
        if (!accu) return 1;
        d[1] = {ID_ACC + acc_self[k], t.a, t.c};
        return 2;
      case T_SHIFT: d[0] = {ID_ACC + acc_self[k], t.a, t.b}; return 1;
      default: d[0] = {ID_A, t.a, t.b}; return 1;   // apply_upd
    }
  }
  std::vector<std::pair<int, int>> range;   // [lo, hi) of every cluster, compact for the overlap tests
  bool overlap(int x, int y) const { return range[x].first < range[y].second && range[y].first < range[x].second; }
  // Def 3.2
  bool precedes(int i, int j) const {
    if (i == j) return false;
    Dep o[2], in[3];
    int no = outs(i, o), ni = ins(j, in);
    for (int p = 0; p < no; ++p)
      for (int q = 0; q < ni; ++q)
        if (o[p].id == in[q].id && overlap(o[p].r, in[q].r) && overlap(o[p].c, in[q].c)) return true;
    return false;
  }
  bool leaf_block(int r, int c) const {
    int id = bt.find(r, c);
    return bt.nodes[id].is_leaf();
  }
  // recursive bodies of Alg 2, Alg 3, its upper mirror and Alg 1 (Alg 7, Alg 8 and its mirror,
  // Alg 4 in accumulator mode), in program order: the sub-tasks of task g (none for a task on
  // leaves); at most MAX_SUB
  static constexpr int MAX_SUB = 12;
  int list_subtasks(int g, Task* out) const {
    const Task t = tasks[g];
    if (t.type == T_SHIFT || t.type == T_APPLY) return 0;
    int n = 0;
    auto put = [&](int type, int a, int b, int c) { out[n++] = {type, a, b, c}; };
    // accumulator mode: apply_upd of a leaf before the task that factorises or solves with it
    auto sub = [&](int type, int a, int b, int c) {
      if (accu && type != T_MUL) {
        int r = type == T_TRSU ? b : a, q = type == T_TRSU ? a : b;
        if (leaf_block(r, q)) put(T_APPLY, r, q, -1);
      }
      put(type, a, b, c);
    };
    const Cluster& A = ct.cl[t.a];
    if (t.type == T_LU) {
      if (leaf_block(t.a, t.a)) return 0;
      int t0 = A.son0, t1 = A.son1;
      if (accu) put(T_SHIFT, t.a, t.a, -1);
      sub(T_LU, t0, t0, -1);
      sub(T_TRSU, t0, t1, -1);
      sub(T_TRSL, t0, t1, -1);
      sub(T_MUL, t1, t0, t1);
      sub(T_LU, t1, t1, -1);
    } else if (t.type == T_TRSL) {
      if (leaf_block(t.a, t.b)) return 0;
      const Cluster& S = ct.cl[t.b];
      int t0 = A.son0, t1 = A.son1, s0 = S.son0, s1 = S.son1;
      if (accu) put(T_SHIFT, t.a, t.b, -1);
      sub(T_TRSL, t0, s0, -1);
      sub(T_TRSL, t0, s1, -1);
      sub(T_MUL, t1, t0, s0);
      sub(T_MUL, t1, t0, s1);
      sub(T_TRSL, t1, s0, -1);
      sub(T_TRSL, t1, s1, -1);
    } else if (t.type == T_TRSU) {
      if (leaf_block(t.b, t.a)) return 0;
      const Cluster& S = ct.cl[t.b];
      int t0 = A.son0, t1 = A.son1, s0 = S.son0, s1 = S.son1;
      if (accu) put(T_SHIFT, t.b, t.a, -1);
      sub(T_TRSU, t0, s0, -1);
      sub(T_TRSU, t0, s1, -1);
      sub(T_MUL, s0, t0, t1);
      sub(T_MUL, s1, t0, t1);
      sub(T_TRSU, t1, s0, -1);
      sub(T_TRSU, t1, s1, -1);
    } else {
      if (leaf_block(t.a, t.b) || leaf_block(t.b, t.c) || leaf_block(t.a, t.c)) return 0;
      const Cluster& R = ct.cl[t.b];
      const Cluster& C = ct.cl[t.c];
      int ai[2] = {A.son0, A.son1}, bl[2] = {R.son0, R.son1}, cj[2] = {C.son0, C.son1};
      for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j)
          for (int l = 0; l < 2; ++l) put(T_MUL, ai[i], bl[l], cj[j]);
    }
    return n;
  }
  // the accumulator identifiers of task k's block and of its parent block
  void set_acc(int k) {
    const Task& t = tasks[k];
    int r = t.a, q = t.b;
    if (t.type == T_TRSU) r = t.b, q = t.a;
    if (t.type == T_MUL) q = t.c;
    const int node = bt.find(r, q);
    acc_self[k] = node;
    acc_par[k] = parent_node[node];
  }
  // writes the cnt sub-tasks of g at indices [first, first + cnt) (already allocated) with the
  // automatic local edges t_i -> t_j for i < j whenever Def 3.2 holds
  void place(int g, int first, const Task* sub, int cnt) {
    for (int i = 0; i < cnt; ++i) {
      tasks[first + i] = sub[i];
      if (accu) set_acc(first + i);
    }
    if (cnt == 0) return;
    sub_first[g] = first;
    sub_count[g] = cnt;
    for (int i = 0; i < cnt; ++i)
      for (int j = i + 1; j < cnt; ++j)
        if (precedes(first + i, first + j)) succ[first + i].push_back(first + j);
  }
  // room for `extra` more tasks
  void grow(size_t extra) {
    const size_t n = tasks.size() + extra;
    tasks.resize(n);
    succ.resize(n);
    sub_first.resize(n, -1);
    sub_count.resize(n, 0);
    if (accu) {
      acc_self.resize(n, -1);
      acc_par.resize(n, -1);
    }
  }
  // Alg 9 / Alg 10 for task w of the current work list: returns 0 if w retires, 1 if it stays
  // (an unrefined task whose successors were refined), 2 if it was refined
  int refine(int w, std::vector<int>& newsucc) {
    if (sub_count[w] == 0) {
      // Alg 10: refine the dependencies of an unrefined task
      bool changed = false;
      newsucc.clear();
      for (int x : succ[w]) {
        if (sub_count[x] > 0) {
          changed = true;
          for (int s = sub_first[x]; s < sub_first[x] + sub_count[x]; ++s)
            if (precedes(w, s)) newsucc.push_back(s);
        } else if (precedes(w, x)) {
          newsucc.push_back(x);
        }
      }
      succ[w] = newsucc;
      return changed ? 1 : 0;
    }
    // Alg 9: inherit the dependencies on the sub-tasks
    const int f = sub_first[w], cnt = sub_count[w];
    for (int x : succ[w]) {
      int xf = x, xc = 1;
      if (sub_count[x] > 0) {
        xf = sub_first[x];
        xc = sub_count[x];
      }
      for (int tp = f; tp < f + cnt; ++tp)
        for (int q = xf; q < xf + xc; ++q)
          if (precedes(tp, q)) succ[tp].push_back(q);
    }
    return 2;
  }

  // §4.1, Alg 12 for task t of the current work set: the neighbourhood N is t's sub-tasks (or t)
  // and, for every successor, its sub-tasks (or the successor); every edge (t', s) of t's
  // sub-tasks (or of t) whose target is also reached by a path of length >= 2 inside N goes.
  std::vector<int> in_n, seen, stack_;
  int stamp_n = 0, stamp_s = 0;
  void sparsify(int t) {
    if (in_n.size() < tasks.size()) {
      in_n.resize(tasks.size(), 0);
      seen.resize(tasks.size(), 0);
    }
    ++stamp_n;
    auto add_n = [&](int x) {
      if (sub_count[x] > 0)
        for (int q = sub_first[x]; q < sub_first[x] + sub_count[x]; ++q) in_n[q] = stamp_n;
      else
        in_n[x] = stamp_n;
    };
    add_n(t);
    for (int s : succ[t]) add_n(s);
    const int f = sub_count[t] > 0 ? sub_first[t] : t, cnt = sub_count[t] > 0 ? sub_count[t] : 1;
    for (int tp = f; tp < f + cnt; ++tp) {
      ++stamp_s;
      stack_.clear();
      auto visit_from = [&](int v) {
        for (int u : succ[v])
          if (in_n[u] == stamp_n && seen[u] != stamp_s) {
            seen[u] = stamp_s;
            stack_.push_back(u);
          }
      };
      for (int s : succ[tp])
        if (in_n[s] == stamp_n) visit_from(s);
      if (stack_.empty()) continue;
      while (!stack_.empty()) {
        const int v = stack_.back();
        stack_.pop_back();
        visit_from(v);
      }
      auto& S = succ[tp];
      S.erase(std::remove_if(S.begin(), S.end(), [&](int x) { return seen[x] == stamp_s; }), S.end());
    }
  }
};

// fn(i) for i in [0, n) on `threads` threads (chunks handed out in order; serial when small);
// an exception of any worker is rethrown on the calling thread after all have stopped
template <class F>
void parallel_for(size_t n, int threads, F fn) {
  if (threads <= 1 || n < 2048) {
    for (size_t i = 0; i < n; ++i) fn(i);
    return;
  }
  const size_t chunk = std::max<size_t>(256, n / ((size_t)threads * 8));
  std::atomic<size_t> next{0};
  std::exception_ptr err;
  std::mutex err_mu;
  auto worker = [&]() {
    try {
      for (size_t b; (b = next.fetch_add(chunk)) < n;)
        for (size_t i = b; i < std::min(n, b + chunk); ++i) fn(i);
    } catch (...) {
      std::lock_guard<std::mutex> lk(err_mu);
      if (!err) err = std::current_exception();
      next.store(n);
    }
  };
  std::vector<std::thread> pool;
  for (int t = 1; t < threads; ++t) {
    try {
      pool.emplace_back(worker);
    } catch (...) {   // no more threads: the ones started and the caller share the work
      break;
    }
  }
  worker();
  for (auto& th : pool) th.join();
  if (err) std::rethrow_exception(err);
}

}  // namespace

// Alg 11 with the parallel loops of Alg 13: in every iteration the sub-tasks of all work tasks
// are generated (sizes first, then places by a prefix sum, so that task indices do not depend on
// the thread count), then the dependencies of every work task are refined; each step writes only
// data of its own task and its sub-tasks. The result equals the serial construction.
void build_task_graph(const ClusterTree& ct, const BlockTree& bt, TaskGraph& g, bool accumulators, int threads,
                      bool sparsify) {
  auto t0 = std::chrono::steady_clock::now();
  g = TaskGraph();
  if (ct.cl.empty()) return;
  if (threads <= 0) threads = (int)std::max(1u, std::min(std::thread::hardware_concurrency(), 64u));
  DagBuilder b(ct, bt, accumulators);
  b.tasks.reserve(1 << 16);
  b.grow(1);
  b.tasks[0] = {T_LU, 0, 0, -1};
  if (accumulators) b.set_acc(0);
  std::vector<int> work{0}, next, retired, cnt, first, flag;
  std::vector<Task> lists;
  while (!work.empty()) {
    const size_t nw = work.size();
    cnt.assign(nw, 0);
    lists.resize(nw * DagBuilder::MAX_SUB);
    parallel_for(nw, threads, [&](size_t i) { cnt[i] = b.list_subtasks(work[i], &lists[i * DagBuilder::MAX_SUB]); });
    first.resize(nw);
    size_t total = 0;
    const int base = (int)b.tasks.size();
    for (size_t i = 0; i < nw; ++i) {
      first[i] = base + (int)total;
      total += cnt[i];
    }
    b.grow(total);
    parallel_for(nw, threads,
                 [&](size_t i) { b.place(work[i], first[i], &lists[i * DagBuilder::MAX_SUB], cnt[i]); });
    flag.assign(nw, 0);
    parallel_for(nw, threads, [&](size_t i) {
      thread_local std::vector<int> scratch;
      flag[i] = b.refine(work[i], scratch);
    });
    // Alg 12 in work order (each step sees the removals of the previous ones)
    if (sparsify)
      for (size_t i = 0; i < nw; ++i) b.sparsify(work[i]);
    next.clear();
    for (size_t i = 0; i < nw; ++i) {
      const int w = work[i];
      if (flag[i] == 0)
        retired.push_back(w);
      else if (flag[i] == 1)
        next.push_back(w);
      else
        for (int tp = b.sub_first[w]; tp < b.sub_first[w] + b.sub_count[w]; ++tp) next.push_back(tp);
    }
    // refined tasks leave the graph; sub-task counts only describe refinement within one
    // iteration of Alg 11
    for (size_t i = 0; i < nw; ++i)
      if (flag[i] == 2) {
        std::vector<int>().swap(b.succ[work[i]]);
        b.sub_count[work[i]] = -1;
      }
    work.swap(next);
  }
  // compact the retired tasks into the output graph
  std::vector<int> remap(b.tasks.size(), -1);
  g.nodes.reserve(retired.size());
  for (int r : retired) {
    remap[r] = (int)g.nodes.size();
    g.nodes.push_back(b.tasks[r]);
  }
  std::vector<size_t> eoff(retired.size() + 1, 0);
  for (size_t i = 0; i < retired.size(); ++i) eoff[i + 1] = eoff[i] + b.succ[retired[i]].size();
  g.edges.resize(eoff.back());
  parallel_for(retired.size(), threads, [&](size_t i) {
    const int r = retired[i];
    size_t e = eoff[i];
    for (int q : b.succ[r]) g.edges[e++] = {remap[r], remap[q]};
  });
  g.build_seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
}

void build_merged_accumulator_graph(const ClusterTree& ct, const BlockTree& bt, TaskGraph& g, int threads) {
  auto t0 = std::chrono::steady_clock::now();
  build_task_graph(ct, bt, g, false, threads);
  if (g.nodes.empty()) return;
  const int nlu = (int)g.nodes.size();
  // the accumulator handling alone: one task per block-tree node, parent -> sons
  std::vector<int> acc_task(bt.nodes.size());
  for (size_t i = 0; i < bt.nodes.size(); ++i) {
    const BlockNode& b = bt.nodes[i];
    acc_task[i] = (int)g.nodes.size();
    g.nodes.push_back({b.is_leaf() ? T_APPLY : T_SHIFT, b.row, b.col, -1});
  }
  for (size_t i = 0; i < bt.nodes.size(); ++i)
    for (int q = 0; q < 4; ++q)
      if (bt.nodes[i].sons[q] >= 0) g.edges.emplace_back(acc_task[i], acc_task[bt.nodes[i].sons[q]]);
  // links: add_upd -> accumulator task of its destination; apply_upd of a leaf -> its leaf task
  for (int k = 0; k < nlu; ++k) {
    const Task& t = g.nodes[k];
    if (t.type == T_MUL) {
      g.edges.emplace_back(k, acc_task[bt.find(t.a, t.c)]);
    } else {
      int r = t.type == T_TRSU ? t.b : t.a, c = t.type == T_TRSU ? t.a : t.b;
      g.edges.emplace_back(acc_task[bt.find(r, c)], k);
    }
  }
  g.build_seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
}

bool compute_levels(TaskGraph& g) {
  size_t n = g.nodes.size();
  std::vector<int> indeg(n, 0), start(n + 1, 0), adj(g.edges.size());
  for (auto& e : g.edges) {
    indeg[e.second]++;
    start[e.first + 1]++;
  }
  for (size_t i = 0; i < n; ++i) start[i + 1] += start[i];
  std::vector<int> fill(start.begin(), start.end() - 1);
  for (auto& e : g.edges) adj[fill[e.first]++] = e.second;
  g.level.assign(n, 0);
  std::deque<int> q;
  for (size_t i = 0; i < n; ++i)
    if (indeg[i] == 0) q.push_back((int)i);
  size_t seen = 0;
  int maxl = -1;
  while (!q.empty()) {
    int t = q.front();
    q.pop_front();
    ++seen;
    if (g.level[t] > maxl) maxl = g.level[t];
    for (int k = start[t]; k < start[t + 1]; ++k) {
      int s = adj[k];
      if (g.level[t] + 1 > g.level[s]) g.level[s] = g.level[t] + 1;
      if (--indeg[s] == 0) q.push_back(s);
    }
  }
  g.nlevels = maxl + 1;
  return seen == n;
}

}  // namespace hm
