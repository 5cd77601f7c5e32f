// Planner: turns the H-LU task graph (or a solve / matvec) into batched micro-op launches.
#pragma once

#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <new>
#include <type_traits>
#include <vector>

#include "ops.h"
#include "structure.h"

namespace hm {

// Storage of one leaf block in a value arena (column-major).
struct LeafStore {
  int node = -1, row = -1, col = -1;
  int m = 0, n = 0;
  bool lr = false;
  int cap = 0;          // low-rank capacity (columns of U and V)
  int64_t off = 0;      // dense: D (ld m); low-rank: U (ld m)
  int64_t voff = 0;     // low-rank: V (ld n)
  int rank_idx = -1;    // low-rank: index into the rank array
  int64_t piv_off = -1; // diagonal dense leaf: offset into the pivot array
};

struct Layout {
  std::vector<LeafStore> leaf;   // indexed by BlockTree leaf index
  int64_t nvalues = 0;
  int nranks = 0;
  int64_t npiv = 0;
  int rank_cap = 64;
};

void build_layout(const ClusterTree& ct, const BlockTree& bt, int rank_cap, Layout& lay);

struct Launch {
  int kind, begin, count;
  int gy = 1, gz = 1;   // GEMM launches: CTAs per micro-op along C tiles / reduction slices
  int first = 0;        // 1: the first launch of a phase; the launches of one phase are independent
  int wave = -1;        // H-LU plans: the wave (task-graph level) the launch belongs to
  int side = 0;         // 1: a deferred rounded addition of `wave`, run on a side stream after the
                        // wave's other launches and before wave + 2 (its scratch is reused there)
};

// Grid of a GEMM launch: orders the (independent) micro-ops by estimated work, largest first,
// and gives each micro-op whose work is well above its share of the GPU several CTAs (tiles of
// C along y, reduction slices of accumulating micro-ops along z, recorded in GemmOp::split);
// gy, gz are the launch's maxima.
void gemm_grid(GemmOp* ops, int count, int& gy, int& gz);
// FMAs per CTA that the GEMM split aims at (process-wide; default 16384): the planner's split
// bound and, through Bases::gemm_work, the kernels' own lowering of it.
void set_gemm_min_work(double fmas_per_cta);
double gemm_min_work();
// The same, writing the ordered micro-ops with their splits to out (count entries, not
// overlapping ops).
void gemm_grid_to(const GemmOp* ops, int count, GemmOp* out, int& gy, int& gz);

// Growable array of trivially copyable records that grows in place (realloc): the micro-op
// arrays of a large plan reach gigabytes, and a std::vector would copy and zero-fill them on
// every doubling.
template <class T>
class PodVec {
  static_assert(std::is_trivially_copyable<T>::value, "PodVec holds trivially copyable records");
  T* p_ = nullptr;
  size_t n_ = 0, cap_ = 0;
  void grow(size_t want) {
    if (want <= cap_) return;
    size_t c = cap_ ? cap_ : 64;
    while (c < want) c *= 2;
    void* q = std::realloc(p_, c * sizeof(T));
    if (!q) throw std::bad_alloc();
    p_ = static_cast<T*>(q);
    cap_ = c;
  }

 public:
  PodVec() = default;
  PodVec(const PodVec& o) { append(o.p_, o.n_); }
  PodVec(PodVec&& o) noexcept : p_(o.p_), n_(o.n_), cap_(o.cap_) { o.p_ = nullptr, o.n_ = o.cap_ = 0; }
  PodVec& operator=(const PodVec& o) {
    if (this != &o) {
      n_ = 0;
      append(o.p_, o.n_);
    }
    return *this;
  }
  PodVec& operator=(PodVec&& o) noexcept {
    if (this != &o) {
      std::free(p_);
      p_ = o.p_, n_ = o.n_, cap_ = o.cap_;
      o.p_ = nullptr, o.n_ = o.cap_ = 0;
    }
    return *this;
  }
  ~PodVec() { std::free(p_); }
  size_t size() const { return n_; }
  bool empty() const { return n_ == 0; }
  T* data() { return p_; }
  const T* data() const { return p_; }
  T* begin() { return p_; }
  T* end() { return p_ + n_; }
  const T* begin() const { return p_; }
  const T* end() const { return p_ + n_; }
  T& operator[](size_t i) { return p_[i]; }
  const T& operator[](size_t i) const { return p_[i]; }
  T& back() { return p_[n_ - 1]; }
  void clear() { n_ = 0; }
  void push_back(const T& v) {
    grow(n_ + 1);
    p_[n_++] = v;
  }
  void append(const T* src, size_t k) {
    if (!k) return;
    grow(n_ + k);
    std::memcpy(static_cast<void*>(p_ + n_), src, k * sizeof(T));
    n_ += k;
  }
  template <class It>
  void insert(T* /* at the end only */, It first, It last) {
    append(&*first, (size_t)(last - first));
  }
  // k uninitialised records at the end, to be written by the caller
  T* extend(size_t k) {
    grow(n_ + k);
    T* r = p_ + n_;
    n_ += k;
    return r;
  }
};

struct Plan {
  PodVec<GetrfOp> getrf;
  PodVec<TrsmOp> trsm;
  PodVec<GemmOp> gemm;
  PodVec<CopyOp> copy;
  PodVec<TruncOp> trunc;      // shared by K_STACK and K_CORE launches
  PodVec<StackEntry> entries;
  PodVec<EvalOp> eval;
  PodVec<AcaOp> aca;
  std::vector<Launch> launches;    // execution order
  int64_t scratch_doubles = 0;
  int64_t scratch_ints = 0;
  int nwaves = 0;
  int nphases = 0;
  int ntasks = 0;
  int64_t ntrunc = 0;
  int64_t scratch_products_max = 0;   // largest product / solve scratch of one wave (doubles)
  int64_t scratch_trunc_max = 0;      // largest truncation scratch of one wave (doubles)
  bool two_scratch = false;           // odd waves use SP_S2 / IS_S2 (deferred rounded additions)
  int64_t deferred_truncations = 0;   // rounded additions on the side stream
  int64_t arena_doubles = 0;          // accumulator arena (SP_ACC) of an accumulator H-LU plan
  int64_t accumulated_pieces = 0;     // update pieces kept in the arena across waves
};

// Memory spaces the planner addresses (factor vs. matrix storage).
struct Spaces {
  int d;   // SP_F or SP_A
  int r;   // IS_RANK or IS_ARANK
};

// H-LU: every wave of the levelled task graph expanded into phases of micro-ops. threads: host
// threads that plan ranges of waves in parallel (0: all hardware threads); any value gives the
// same plan.
// precision 0: all FP64. 1 (mixed): the products of Alg 1 and the rebuild products of the rounded
// additions are K_GEMM32 micro-ops (FP32 FMAs); 2 (mixed, tensor cores): those with at least 128
// static rows are K_GEMM_TC micro-ops (split TF32 on tcgen05, FP32 accumulation), the rest K_GEMM32.
// defer: rounded additions whose target leaf is not touched by the next wave (no task of the
// next level reads it, no product of the next level updates it) become side launches of their
// wave (Launch::side), overlapping the next wave; odd waves then use the second scratch space.
// accumulate: the accumulator H-LU of §2.3 (Alg 4-8) with its accumulators held as lists of
// pieces: the product pieces that reach a low-rank leaf are not truncated in the wave that forms
// them but kept (in the arena SP_ACC when they outlive their wave) and added in one rounded
// addition in the wave of the leaf's last update before the leaf is read (apply_upd before the
// solve, the leaf LU or a product that uses it). Planned on one thread.
void plan_lu(const ClusterTree& ct, const BlockTree& bt, const Layout& lay, const TaskGraph& g,
             double eps, Plan& plan, int threads = 0, int precision = 0, bool defer = false,
             bool accumulate = false);
// Independent H-LU instances in one plan: wave w of every instance is expanded into the same
// phases, so that one launch per kind and phase serves all of them (their task graphs have no
// edges between each other). Instance i addresses its values, ranks and pivots at the given
// offsets of one concatenated space each; scratch is shared wave by wave.
struct LuInstance {
  const ClusterTree* ct;
  const BlockTree* bt;
  const Layout* lay;
  const TaskGraph* g;
  int64_t base_d, base_r, base_p;
};
void plan_lu_batch(const std::vector<LuInstance>& inst, double eps, Plan& plan, int threads = 0,
                   int precision = 0);
// hm_build: dense leaf assembly, ACA + rounded truncation of the admissible leaves.
void plan_build(const ClusterTree& ct, const BlockTree& bt, const Layout& lay, double eps, int aca_kmax,
                int64_t scratch_budget_doubles, Plan& plan);
// forward / backward substitution with the factors for up to nrhs_max right-hand sides in
// the SP_X work buffer (n x nrhs_max, permuted order); the dynamic count is scratch int 0.
void plan_solve(const ClusterTree& ct, const BlockTree& bt, const Layout& lay, int nrhs_max, Plan& plan);
// y = op(M) x on the SP_X buffer: columns [0, nrhs_max) hold x, [nrhs_max, 2 nrhs_max) get y.
// op: 0 = the H-matrix A (SP_A), 1 = L (unit lower incl. pivots), 2 = U, 3 = P L U.
void plan_matvec(const ClusterTree& ct, const BlockTree& bt, const Layout& lay, int op, int nrhs_max,
                 Plan& plan);

}  // namespace hm
