// Batched micro-op descriptors shared by the host planner and the CUDA kernels.
//
// The H-LU task graph (Alg 11) is executed wave by wave; every task of a wave is expanded
// into micro-ops of a few kinds (dense leaf LU, triangular solves, small GEMMs, copies,
// stacked rounded truncation), and all micro-ops of one kind in one phase of a wave are
// launched as one batched kernel, one CTA per micro-op.
//
// Addresses are stored as 64-bit references into a handful of memory spaces so that one
// plan can be replayed on any factor / scratch / right-hand-side buffers:
//   ref = ((space + 1) << 60) | element_offset,   ref == 0 means "none".
// Dimensions are a static part plus an optional dynamic part read from device memory
// (the rank of a low-rank block, known only on the device).
#pragma once

#include <cstdint>

namespace hm {

enum DSpace : int { SP_F = 0, SP_S = 1, SP_X = 2, SP_A = 3, SP_P = 4, SP_S2 = 5, SP_ACC = 6, NDSPACE = 7 };
// SP_F factor values, SP_S scratch, SP_X right-hand-side work buffer,
// SP_A matrix values, SP_P permuted points (n x 3, row-major), SP_S2 the scratch of the odd waves
// of an H-LU plan whose truncations overlap the next wave (same size as SP_S), SP_ACC the
// accumulator arena of an accumulator H-LU plan (update pieces kept across waves)
enum ISpace : int { IS_RANK = 0, IS_PIV = 1, IS_S = 2, IS_ARANK = 3, IS_S2 = 4, NISPACE = 5 };

constexpr uint64_t REF_MASK = (1ull << 60) - 1;
inline uint64_t mkref(int space, int64_t off) { return ((uint64_t)(space + 1) << 60) | (uint64_t)off; }

struct Bases {
  double* d[NDSPACE];
  int* i[NISPACE];
  unsigned long long* flops;   // [0, NFC): model flops per class; [NFC, NFC+NKIND): algorithmic
                               // flops executed by each kernel kind
  float gemm_work;             // GEMM split: FMAs per CTA the kernels aim at (0: 16384)
  int* status;                 // [0] singular pivot count, [1] rank-cap hits, [2] aca non-converged,
                               // [3] row interchanges of the leaf LUs, [4] bounded device waits
                               // that gave up (8 ints)
};

// flop accounting classes (model of the truncation counts QR + core + SVD + rebuild)
enum FlopClass : int { FC_GETRF = 0, FC_TRSM = 1, FC_GEMM = 2, FC_TRUNC = 3, FC_NONE = 4, NFC = 5 };

// GF_SYM_UPPER: C is symmetric (a Gram matrix A^T A); only the entries i <= j are computed and
// written, the consumer mirrors them
// GF_TF32 / GF_F32: the micro-op runs in a K_GEMM_TC / K_GEMM32 launch (mixed-precision plans)
enum GemmFlags : int { GF_ATOMIC = 1, GF_OVERWRITE = 2, GF_A_UPPER = 4, GF_A_UNITLOWER = 8, GF_SYM_UPPER = 16,
                       GF_TF32 = 32, GF_F32 = 64 };

// C(i,j) (+)= alpha * sum_l A(i,l) B(l,j),  X(i,j) = X[i*rs + j*cs]
struct GemmOp {
  uint64_t A, B, C;
  int64_t a_rs, a_cs, b_rs, b_cs, c_rs, c_cs;
  uint64_t md, nd, kd;   // dynamic dimension adders (int refs)
  int m, n, k;
  int flags;
  double alpha;
  int fclass;
  int split;   // CTA budget of this micro-op: (split & 0xffff) * max(1, split >> 16); the kernel
               // divides it between C tiles and (atomic micro-ops) reduction slices
               // slices (0 = one CTA); CTAs of the launch grid beyond them exit
};

// batched vector triangular kernels on the packed LU of a diagonal leaf (b x b, ld = b)
enum TrsmMode : int {
  TM_L_PIV = 0,    // x := L^{-1} P^T x   (unit lower, pivots)
  TM_UT = 1,       // x := U^{-T} x
  TM_U = 2,        // x := U^{-1} x
  TM_MUL_U = 3,    // x := U x
  TM_MUL_PL = 4    // x := P L x
};
struct TrsmOp {
  uint64_t T;      // packed LU, col-major b x b
  uint64_t piv;    // int ref to b pivots (0-based, LAPACK order)
  uint64_t X;      // vectors: element e of vector v at X[e*x_es + v*x_vs]
  int64_t x_es, x_vs;
  uint64_t nvd;    // dynamic vector count adder
  int nv, b, mode, pad;
};

struct GetrfOp {
  uint64_t A;      // b x b col-major (ld = b), factored in place
  uint64_t piv;    // int ref
  int b, pad;
};

enum CopyMode : int { CM_ZERO = 0, CM_IDENTITY = 1, CM_COPY = 2, CM_ADD = 3 };
struct CopyOp {
  uint64_t src; int64_t s_rs, s_cs;
  uint64_t dst; int64_t d_rs, d_cs;
  uint64_t md, nd;
  int m, n, mode, pad;
  double alpha;
};

// one stacked piece of a rounded addition: alpha * W Z^T on rows [row_off, row_off+nrows),
// cols [col_off, col_off+ncols) of the target; W(i,l) = W[i*w_rs + l*w_cs], Z likewise.
struct StackEntry {
  uint64_t W; int64_t w_rs, w_cs;
  uint64_t Z; int64_t z_rs, z_cs;
  uint64_t kd;     // dynamic rank adder
  int k;
  int row_off, nrows, col_off, ncols, pad;
  double alpha;
};

// rounded addition of a group of pieces into one low-rank leaf U V^T (m x n, cap)
struct TruncOp {
  uint64_t U, V;       // target factors, ld m and n, cap columns
  uint64_t rank;       // int ref
  int m, n, cap, Kcap;
  int first_entry, n_entries;
  uint64_t Wst, Zst;   // m x Kcap and n x Kcap stacks
  uint64_t Gw, Gz;     // Kcap x Kcap Gram matrices (ld Kcap)
  uint64_t Tw, Tz;     // Kcap x cap coefficient matrices (ld Kcap)
  uint64_t work;       // 2 * Kcap * Kcap doubles (Gw and Gz are reused by the core)
  uint64_t Kd;         // int ref: stacked rank
  double eps;
  int flags;           // TF_NOSELF: the stack leaves out U, V (a temporary sum: its rank is not read)
  int pad_;
};
enum TruncFlags : int { TF_NOSELF = 1 };

// dense leaf assembly: D(i,j) = 1 / (4 pi (|p_{r0+i} - p_{c0+j}| + h)), permuted points
struct EvalOp {
  uint64_t D;
  int r0, c0, m, n;
};

// adaptive cross approximation of an admissible leaf into scratch factors
struct AcaOp {
  int r0, c0, m, n;
  uint64_t U, V;       // m x kmax and n x kmax (ld m, n)
  uint64_t used;       // int ref: m row flags
  uint64_t kd;         // int ref: resulting rank
  int kmax, pad;
  double tol;
};

// Mixed-precision GEMM micro-ops, in the same GemmOp array as K_GEMM:
// K_GEMM_TC (flag GF_TF32): tensor cores, split-TF32 operands, FP32 accumulation;
// K_GEMM32 (flag GF_F32): the FP64 kernel's tiling with FP32 FMAs and accumulators.
enum OpKind : int { K_GETRF = 0, K_TRSM = 1, K_GEMM = 2, K_COPY = 3, K_STACK = 4, K_CORE = 5,
                    K_EVAL = 6, K_ACA = 7, K_GEMM_TC = 8, K_GEMM32 = 9, NKIND = 10 };

}  // namespace hm
