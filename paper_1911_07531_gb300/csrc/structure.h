// Host-side structure of an H-matrix and of its H-LU task graph.
//
//  * cluster tree by geometric bisection (Def 2.1), standard admissibility (§5.1),
//    block tree (Def 2.2);
//  * the H-LU task graph built by semi-automatic refinement (§3.1: Table 1, Def 3.2,
//    Alg 9, Alg 10, Alg 11) and its longest-path levels (the waves the GPU executes), and the
//    task graph of the accumulator-based H-LU (§3.2, Table 2).
//
// All of it is integer and comparison work in FP64 with a fixed operation order; it is
// compiled without floating-point contraction so that the admissibility decisions are
// reproducible bit for bit.
#pragma once

#include <cstdint>
#include <string>
#include <unordered_map>
#include <vector>

namespace hm {

struct Cluster {
  int lo = 0, hi = 0;          // permuted index range [lo, hi)
  int son0 = -1, son1 = -1;    // depth-first pre-order ids
  int level = 0;
  int parent = -1;
  double bmin[3] = {0, 0, 0}, bmax[3] = {0, 0, 0};
  int size() const { return hi - lo; }
  bool leaf() const { return son0 < 0; }
};

struct ClusterTree {
  std::vector<Cluster> cl;
  std::vector<int64_t> perm;   // perm[k] = original index of permuted position k
  int leaf_size = 64;
  int depth = 0;
};

// Block tree node; sons[2*i + j] = (row son i, col son j), or -1 for a leaf.
struct BlockNode {
  int row = -1, col = -1;
  bool adm = false;
  int sons[4] = {-1, -1, -1, -1};
  int leaf = -1;               // index into BlockTree::leaves, or -1 for inner nodes
  bool is_leaf() const { return sons[0] < 0; }
};

struct BlockTree {
  std::vector<BlockNode> nodes;
  std::vector<int> leaves;     // node ids of the leaves, in creation (pre-) order
  std::unordered_map<uint64_t, int> index;
  int ncl = 0;
  int find(int r, int c) const {
    auto it = index.find((uint64_t)r * (uint64_t)ncl + (uint64_t)c);
    return it == index.end() ? -1 : it->second;
  }
};

enum TaskType : int { T_LU = 0, T_MUL = 1, T_TRSL = 2, T_TRSU = 3, T_SHIFT = 4, T_APPLY = 5 };

struct Task {
  int type;
  int a, b, c;   // lu: (t,t,-1); trsl: (t,s,-1) L_tt X_ts = M_ts; trsu: (t,s,-1) X_st U_tt = M_st;
                 // mul: (t,r,s) C_ts -= A_tr B_rs (add_upd in the accumulator graph);
                 // shift / apply: (t,s,-1) shift_upd / apply_upd of the block (t,s)
};

struct TaskGraph {
  std::vector<Task> nodes;
  std::vector<std::pair<int, int>> edges;   // (src, dst) indices into nodes
  std::vector<int> level;                   // longest-path level of each node
  int nlevels = 0;
  double build_seconds = 0.0;
};

void build_cluster_tree(const double* pts, int64_t n, int leaf_size, ClusterTree& ct);
bool admissible(const Cluster& t, const Cluster& s, double eta);
void build_block_tree(const ClusterTree& ct, double eta, BlockTree& bt);
void collect_leaves(const BlockTree& bt, int node, std::vector<int>& out);

// Alg 11 started from hlu(A, L, U) on the root cluster. accumulators: the task graph of the
// accumulator-based H-LU (§3.2, Table 2) -- a refined hlu / htrsl / htrsu starts with
// shift_upd of its block, apply_upd of a leaf precedes the task that factorises or solves with
// it, add_upd is refined like hmul and writes the block and its accumulator.
// threads: host threads of the parallel loops of Alg 13 (0: all hardware threads); the graph
// does not depend on it. sparsify: every iteration ends with the removal of redundant edges of
// Alg 12 (§4.1) for each task of the work set, in order.
void build_task_graph(const ClusterTree& ct, const BlockTree& bt, TaskGraph& g, bool accumulators = false,
                      int threads = 0, bool sparsify = false);
// The accumulator task graph built in two parts (§4.3): the standard graph (hmul tasks stand for
// add_upd) plus one shift_upd / apply_upd task per block-tree node, linked by edges parent ->
// son, add_upd -> accumulator task of its destination, apply_upd of a leaf -> its leaf task.
void build_merged_accumulator_graph(const ClusterTree& ct, const BlockTree& bt, TaskGraph& g, int threads = 0);
// longest-path levels; returns false if the graph has a cycle
bool compute_levels(TaskGraph& g);

}  // namespace hm
