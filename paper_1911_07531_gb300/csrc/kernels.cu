// Batched FP64 kernels of the H-LU hot path (one CTA per micro-op).
//
// GB300 has very little FP64 throughput (about 2 DFMA per clock per SM), so every kernel
// here is FP64-issue bound once the operands sit in shared memory or L1/L2; the design
// goal is to keep the DFMA pipe of all 152 SMs busy: 64x64 register-blocked tiles with
// 16 independent accumulators per thread for the small GEMMs, one CTA per task so that
// a wave with hundreds of tasks fills the machine, and no host round trip inside a wave.
//
//   k_getrf  dense leaf LU with partial pivoting (Alg 2, leaf case)
//   k_trsm   triangular solves / multiplies of a diagonal leaf on many vectors (Alg 3 leaf)
//   k_gemm   C (+)= alpha A B with strided operands and dynamic sizes (Alg 1 leaf products)
//   k_copy   zero / identity / copy / add of strided blocks
//   k_stack  stacking of the pieces of a rounded addition into [U, W_1, ...], [V, Z_1, ...]
//   k_core   rounded truncation core: Gram matrices -> pivoted Cholesky -> Jacobi -> factors
//   k_eval   dense leaf assembly a_ij = 1/(4 pi (|x_i - x_j| + h))
//   k_aca    adaptive cross approximation of an admissible leaf
#include <cuda_runtime.h>

#include <cmath>

#include "kernels.h"

namespace hm {

__device__ __forceinline__ double* dptr(const Bases& B, uint64_t r) {
  return r ? B.d[(r >> 60) - 1] + (r & REF_MASK) : nullptr;
}
__device__ __forceinline__ int* iptr(const Bases& B, uint64_t r) {
  return r ? B.i[(r >> 60) - 1] + (r & REF_MASK) : nullptr;
}
__device__ __forceinline__ int dimv(const Bases& B, int s, uint64_t d) {
  return s + (d ? *iptr(B, d) : 0);
}

__device__ __forceinline__ double block_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  double s = 0.0;
  for (int i = 0; i < nw; ++i) s += red[i];
  __syncthreads();
  return s;
}

__device__ __forceinline__ double block_max(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  double s = red[0];
  for (int i = 1; i < nw; ++i) s = fmax(s, red[i]);
  __syncthreads();
  return s;
}

// argmax of |value| with the smallest index among ties; returns the index (or -1)
__device__ __forceinline__ int block_argmax(double v, int idx, double* redv, int* redi) {
  for (int o = 16; o > 0; o >>= 1) {
    double ov = __shfl_xor_sync(0xffffffffu, v, o);
    int oi = __shfl_xor_sync(0xffffffffu, idx, o);
    if (ov > v || (ov == v && oi >= 0 && (idx < 0 || oi < idx))) {
      v = ov;
      idx = oi;
    }
  }
  int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
  __syncthreads();
  if (l == 0) {
    redv[w] = v;
    redi[w] = idx;
  }
  __syncthreads();
  double bv = redv[0];
  int bi = redi[0];
  for (int i = 1; i < nw; ++i)
    if (redv[i] > bv || (redv[i] == bv && redi[i] >= 0 && (bi < 0 || redi[i] < bi))) {
      bv = redv[i];
      bi = redi[i];
    }
  __syncthreads();
  return bi;
}

// ------------------------------------------------------------------------------ GEMM
// One CTA (256 threads) per micro-op. The output is covered by TM x TN tiles; S groups of
// threads split the reduction of each tile and are summed in shared memory at the end. The
// tile shape is chosen per micro-op from its (dynamic) sizes so that few DFMAs are spent on
// zero padding: the micro-ops are mostly thin (a rank-sized side of 10-60) or have a small
// output with a long reduction (Gram matrices, V^T X).
constexpr int GK = 16;                 // reduction slice
constexpr int GEMM_SMEM_DOUBLES = 5248;

template <int TM, int TN, int RM, int RN, int S>
__device__ __forceinline__ void gemm_tiles(const GemmOp& op, int m, int n, int k, const double* __restrict__ A,
                                           const double* __restrict__ Bm, double* C, double* sm) {
  constexpr int TX = TN / RN, TY = TM / RM, G = TX * TY;
  static_assert(G * S == 256, "256 threads");
  static_assert(S * GK * (TM + 1) + S * GK * (TN + 1) + (S > 1 ? TM * TN : 0) <= GEMM_SMEM_DOUBLES, "smem");
  double* As = sm;                                  // [S][GK][TM+1]
  double* Bs = sm + S * GK * (TM + 1);              // [S][GK][TN+1]
  double* red = Bs + S * GK * (TN + 1);             // [TM*TN] when S > 1
  const int tid = threadIdx.x, g = tid / G, t = tid % G, tx = t % TX, ty = t / TX;
  const bool a_i_fast = op.a_rs <= op.a_cs;
  const bool b_j_fast = op.b_cs <= op.b_rs;
  const bool upper = op.flags & GF_A_UPPER, unitlower = op.flags & GF_A_UNITLOWER;
  for (int i0 = 0; i0 < m; i0 += TM)
    for (int j0 = 0; j0 < n; j0 += TN) {
      double acc[RM][RN];
#pragma unroll
      for (int p = 0; p < RM; ++p)
#pragma unroll
        for (int q = 0; q < RN; ++q) acc[p][q] = 0.0;
      for (int L0 = 0; L0 < k; L0 += S * GK) {
        // every group stages its own slice l0 = L0 + g*GK
        for (int e = tid; e < S * GK * TM; e += 256) {
          int gg = e / (GK * TM), r = e % (GK * TM);
          int i, l;
          if (a_i_fast) { i = r % TM; l = r / TM; } else { l = r % GK; i = r / GK; }
          int gi = i0 + i, gl = L0 + gg * GK + l;
          double v = 0.0;
          if (gi < m && gl < k) {
            if (unitlower) v = gi > gl ? A[gi * op.a_rs + gl * op.a_cs] : (gi == gl ? 1.0 : 0.0);
            else if (upper) v = gl >= gi ? A[gi * op.a_rs + gl * op.a_cs] : 0.0;
            else v = A[gi * op.a_rs + gl * op.a_cs];
          }
          As[(gg * GK + l) * (TM + 1) + i] = v;
        }
        for (int e = tid; e < S * GK * TN; e += 256) {
          int gg = e / (GK * TN), r = e % (GK * TN);
          int j, l;
          if (b_j_fast) { j = r % TN; l = r / TN; } else { l = r % GK; j = r / GK; }
          int gj = j0 + j, gl = L0 + gg * GK + l;
          Bs[(gg * GK + l) * (TN + 1) + j] = (gj < n && gl < k) ? Bm[gl * op.b_rs + gj * op.b_cs] : 0.0;
        }
        __syncthreads();
        const double* Ag = As + g * GK * (TM + 1);
        const double* Bg = Bs + g * GK * (TN + 1);
#pragma unroll 4
        for (int l = 0; l < GK; ++l) {
          double a[RM], b[RN];
#pragma unroll
          for (int p = 0; p < RM; ++p) a[p] = Ag[l * (TM + 1) + ty + TY * p];
#pragma unroll
          for (int q = 0; q < RN; ++q) b[q] = Bg[l * (TN + 1) + tx + TX * q];
#pragma unroll
          for (int p = 0; p < RM; ++p)
#pragma unroll
            for (int q = 0; q < RN; ++q) acc[p][q] = fma(a[p], b[q], acc[p][q]);
        }
        __syncthreads();
      }
      if (S > 1) {
        for (int e = tid; e < TM * TN; e += 256) red[e] = 0.0;
        __syncthreads();
#pragma unroll
        for (int p = 0; p < RM; ++p)
#pragma unroll
          for (int q = 0; q < RN; ++q) atomicAdd(&red[(ty + TY * p) * TN + tx + TX * q], acc[p][q]);
        __syncthreads();
      }
      if (S == 1 || g == 0) {
#pragma unroll
        for (int p = 0; p < RM; ++p)
#pragma unroll
          for (int q = 0; q < RN; ++q) {
            const int il = ty + TY * p, jl = tx + TX * q;
            const int i = i0 + il, j = j0 + jl;
            if (i < m && j < n) {
              double* c = C + (int64_t)i * op.c_rs + (int64_t)j * op.c_cs;
              const double v = op.alpha * (S > 1 ? red[il * TN + jl] : acc[p][q]);
              if (op.flags & GF_ATOMIC) atomicAdd(c, v);
              else if (op.flags & GF_OVERWRITE) *c = v;
              else *c += v;
            }
          }
      }
      if (S > 1) __syncthreads();
    }
}

__global__ void __launch_bounds__(256) k_gemm(const GemmOp* __restrict__ ops, Bases B) {
  const GemmOp op = ops[blockIdx.x];
  const int m = dimv(B, op.m, op.md), n = dimv(B, op.n, op.nd), k = dimv(B, op.k, op.kd);
  if (m <= 0 || n <= 0) return;
  if (k <= 0 && !(op.flags & GF_OVERWRITE)) return;
  __shared__ double sm[GEMM_SMEM_DOUBLES];
  const double* A = dptr(B, op.A);
  const double* Bm = dptr(B, op.B);
  double* C = dptr(B, op.C);
  if (m <= 16 && n <= 16) gemm_tiles<16, 16, 2, 2, 4>(op, m, n, k, A, Bm, C, sm);
  else if (m <= 32 && n <= 32) gemm_tiles<32, 32, 4, 4, 4>(op, m, n, k, A, Bm, C, sm);
  else if (n <= 16) gemm_tiles<256, 16, 16, 1, 1>(op, m, n, k, A, Bm, C, sm);
  else if (n <= 32) gemm_tiles<128, 32, 8, 2, 1>(op, m, n, k, A, Bm, C, sm);
  else if (m <= 32) gemm_tiles<32, 128, 2, 8, 1>(op, m, n, k, A, Bm, C, sm);
  else gemm_tiles<64, 64, 4, 4, 1>(op, m, n, k, A, Bm, C, sm);
  if (threadIdx.x == 0) {
    const unsigned long long f = (unsigned long long)(2.0 * m * n * (double)(k > 0 ? k : 0));
    if (op.fclass < FC_NONE) atomicAdd(&B.flops[op.fclass], f);
    atomicAdd(&B.flops[NFC + K_GEMM], f);
  }
}

// ------------------------------------------------------------------------------ TRSM
__global__ void __launch_bounds__(256) k_trsm(const TrsmOp* __restrict__ ops, Bases B) {
  const TrsmOp op = ops[blockIdx.x];
  const int nv = dimv(B, op.nv, op.nvd), b = op.b;
  if (nv <= 0 || b <= 0) return;
  extern __shared__ double trsm_smem[];   // T[64][65] then X[64][65]
  double(*T)[65] = reinterpret_cast<double(*)[65]>(trsm_smem);
  double(*X)[65] = reinterpret_cast<double(*)[65]>(trsm_smem + 64 * 65);
  __shared__ int piv[64];
  __shared__ double dinv[64];
  const int tid = threadIdx.x;
  const double* Tg = dptr(B, op.T);
  double* Xg = dptr(B, op.X);
  for (int e = tid; e < b * b; e += 256) T[e % b][e / b] = Tg[e];
  if (op.piv)
    for (int e = tid; e < b; e += 256) piv[e] = iptr(B, op.piv)[e];
  __syncthreads();
  if (op.mode == TM_UT || op.mode == TM_U)
    for (int e = tid; e < b; e += 256) dinv[e] = 1.0 / T[e][e];
  __syncthreads();
  const bool e_fast = op.x_es == 1;
  for (int v0 = 0; v0 < nv; v0 += 64) {
    const int nc = min(64, nv - v0);
    for (int e = tid; e < b * nc; e += 256) {
      int ee, v;
      if (e_fast) { ee = e % b; v = e / b; } else { v = e % nc; ee = e / nc; }
      X[ee][v] = Xg[(int64_t)ee * op.x_es + (int64_t)(v0 + v) * op.x_vs];
    }
    __syncthreads();
    if (op.mode == TM_L_PIV) {
      if (tid < nc)
        for (int i = 0; i < b; ++i) {
          int p = piv[i];
          if (p != i) {
            double t = X[i][tid];
            X[i][tid] = X[p][tid];
            X[p][tid] = t;
          }
        }
      __syncthreads();
      for (int j = 0; j < b - 1; ++j) {
        int cnt = (b - 1 - j) * nc;
        for (int e = tid; e < cnt; e += 256) {
          int i = j + 1 + e / nc, v = e % nc;
          X[i][v] = fma(-T[i][j], X[j][v], X[i][v]);
        }
        __syncthreads();
      }
    } else if (op.mode == TM_UT) {
      for (int j = 0; j < b; ++j) {
        if (tid < nc) X[j][tid] = X[j][tid] * dinv[j];
        __syncthreads();
        int cnt = (b - 1 - j) * nc;
        for (int e = tid; e < cnt; e += 256) {
          int i = j + 1 + e / nc, v = e % nc;
          X[i][v] = fma(-T[j][i], X[j][v], X[i][v]);
        }
        __syncthreads();
      }
    } else if (op.mode == TM_U) {
      for (int j = b - 1; j >= 0; --j) {
        if (tid < nc) X[j][tid] = X[j][tid] * dinv[j];
        __syncthreads();
        int cnt = j * nc;
        for (int e = tid; e < cnt; e += 256) {
          int i = e / nc, v = e % nc;
          X[i][v] = fma(-T[i][j], X[j][v], X[i][v]);
        }
        __syncthreads();
      }
    } else {
      // multiplies: each thread keeps its results in registers until all reads are done
      double y[16];
      int cnt = b * nc;
      int q = 0;
      for (int e = tid; e < cnt; e += 256, ++q) {
        int i = e / nc, v = e % nc;
        double s = 0.0;
        if (op.mode == TM_MUL_U) {
          for (int j = i; j < b; ++j) s = fma(T[i][j], X[j][v], s);
        } else {
          s = X[i][v];
          for (int j = 0; j < i; ++j) s = fma(T[i][j], X[j][v], s);
        }
        y[q] = s;
      }
      __syncthreads();
      q = 0;
      for (int e = tid; e < cnt; e += 256, ++q) X[e / nc][e % nc] = y[q];
      __syncthreads();
      if (op.mode == TM_MUL_PL && tid < nc)
        for (int i = b - 1; i >= 0; --i) {
          int p = piv[i];
          if (p != i) {
            double t = X[i][tid];
            X[i][tid] = X[p][tid];
            X[p][tid] = t;
          }
        }
      __syncthreads();
    }
    for (int e = tid; e < b * nc; e += 256) {
      int ee, v;
      if (e_fast) { ee = e % b; v = e / b; } else { v = e % nc; ee = e / nc; }
      Xg[(int64_t)ee * op.x_es + (int64_t)(v0 + v) * op.x_vs] = X[ee][v];
    }
    __syncthreads();
  }
  if (tid == 0) {
    atomicAdd(&B.flops[FC_TRSM], (unsigned long long)nv * b * b);
    atomicAdd(&B.flops[NFC + K_TRSM], (unsigned long long)nv * b * b);
  }
}

// ------------------------------------------------------------------------------ GETRF
__global__ void __launch_bounds__(256) k_getrf(const GetrfOp* __restrict__ ops, Bases B) {
  const GetrfOp op = ops[blockIdx.x];
  const int b = op.b;
  if (b <= 0) return;
  __shared__ double S[64][65];
  __shared__ int sp;
  double* A = dptr(B, op.A);
  int* piv = iptr(B, op.piv);
  const int tid = threadIdx.x;
  for (int e = tid; e < b * b; e += 256) S[e % b][e / b] = A[e];
  __syncthreads();
  for (int j = 0; j < b; ++j) {
    if (tid < 32) {
      double bv = -1.0;
      int bi = -1;
      for (int i = j + tid; i < b; i += 32) {
        double v = fabs(S[i][j]);
        if (v > bv) { bv = v; bi = i; }
      }
      for (int o = 16; o > 0; o >>= 1) {
        double ov = __shfl_xor_sync(0xffffffffu, bv, o);
        int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ov > bv || (ov == bv && oi >= 0 && (bi < 0 || oi < bi))) { bv = ov; bi = oi; }
      }
      if (tid == 0) {
        sp = bi;
        piv[j] = bi;
      }
    }
    __syncthreads();
    const int p = sp;
    if (p != j)
      for (int c = tid; c < b; c += 256) {
        double t = S[j][c];
        S[j][c] = S[p][c];
        S[p][c] = t;
      }
    __syncthreads();
    const double d = S[j][j];
    if (d == 0.0) {
      if (tid == 0) atomicAdd(&B.status[0], 1);
    } else {
      const double dinv = 1.0 / d;
      for (int i = j + 1 + tid; i < b; i += 256) S[i][j] = S[i][j] * dinv;
    }
    __syncthreads();
    const int r = b - 1 - j;
    for (int e = tid; e < r * r; e += 256) {
      int i = j + 1 + e % r, c = j + 1 + e / r;
      S[i][c] = fma(-S[i][j], S[j][c], S[i][c]);
    }
    __syncthreads();
  }
  for (int e = tid; e < b * b; e += 256) A[e] = S[e % b][e / b];
  if (tid == 0) {
    atomicAdd(&B.flops[FC_GETRF], (unsigned long long)(2.0 * b * b * b / 3.0));
    atomicAdd(&B.flops[NFC + K_GETRF], (unsigned long long)(2.0 * b * b * b / 3.0));
  }
}

// ------------------------------------------------------------------------------ COPY
__global__ void __launch_bounds__(256) k_copy(const CopyOp* __restrict__ ops, Bases B) {
  const CopyOp op = ops[blockIdx.x];
  const int m = dimv(B, op.m, op.md), n = dimv(B, op.n, op.nd);
  if (m <= 0 || n <= 0) return;
  const double* src = dptr(B, op.src);
  double* dst = dptr(B, op.dst);
  const int64_t tot = (int64_t)m * n;
  const bool i_fast = op.d_rs <= op.d_cs;
  for (int64_t e = threadIdx.x; e < tot; e += blockDim.x) {
    int i, j;
    if (i_fast) { i = (int)(e % m); j = (int)(e / m); } else { j = (int)(e % n); i = (int)(e / n); }
    double* d = dst + (int64_t)i * op.d_rs + (int64_t)j * op.d_cs;
    switch (op.mode) {
      case CM_ZERO: *d = 0.0; break;
      case CM_IDENTITY: *d = (i == j) ? 1.0 : 0.0; break;
      case CM_COPY: *d = op.alpha * src[(int64_t)i * op.s_rs + (int64_t)j * op.s_cs]; break;
      default: *d += op.alpha * src[(int64_t)i * op.s_rs + (int64_t)j * op.s_cs]; break;
    }
  }
}

// ------------------------------------------------------------------------------ STACK
__global__ void __launch_bounds__(256) k_stack(const TruncOp* __restrict__ ops,
                                               const StackEntry* __restrict__ ent, Bases B) {
  const TruncOp op = ops[blockIdx.x];
  const int m = op.m, n = op.n, Kc = op.Kcap;
  int* rk = iptr(B, op.rank);
  const int kself = *rk;
  __shared__ int s_k[1];
  if (threadIdx.x == 0) {
    int K = kself;
    for (int e = 0; e < op.n_entries; ++e) {
      const StackEntry& se = ent[op.first_entry + e];
      int ke = dimv(B, se.k, se.kd);
      if (ke < 0) ke = 0;
      K += ke;
    }
    if (K > Kc) K = Kc;   // the planner sizes Kcap from static maxima; never taken
    s_k[0] = K;
    *iptr(B, op.Kd) = K;
  }
  __syncthreads();
  const int K = s_k[0];
  double* Wst = dptr(B, op.Wst);
  double* Zst = dptr(B, op.Zst);
  double* Gw = dptr(B, op.Gw);
  double* Gz = dptr(B, op.Gz);
  for (int e = threadIdx.x; e < K * K; e += blockDim.x) {
    int i = e % K, j = e / K;
    Gw[i + (int64_t)j * Kc] = 0.0;
    Gz[i + (int64_t)j * Kc] = 0.0;
  }
  const double* U = dptr(B, op.U);
  const double* V = dptr(B, op.V);
  int col = min(kself, K);
  for (int64_t e = threadIdx.x; e < (int64_t)m * col; e += blockDim.x) Wst[e] = U[e];
  for (int64_t e = threadIdx.x; e < (int64_t)n * col; e += blockDim.x) Zst[e] = V[e];
  for (int q = 0; q < op.n_entries && col < K; ++q) {
    const StackEntry se = ent[op.first_entry + q];
    int ke = dimv(B, se.k, se.kd);
    if (ke > K - col) ke = K - col;
    if (ke <= 0) continue;
    const double* W = dptr(B, se.W);
    const double* Z = dptr(B, se.Z);
    for (int64_t e = threadIdx.x; e < (int64_t)m * ke; e += blockDim.x) {
      int i = (int)(e % m), c = (int)(e / m);
      double v = 0.0;
      if (i >= se.row_off && i < se.row_off + se.nrows)
        v = se.alpha * W[(int64_t)(i - se.row_off) * se.w_rs + (int64_t)c * se.w_cs];
      Wst[(int64_t)(col + c) * m + i] = v;
    }
    for (int64_t e = threadIdx.x; e < (int64_t)n * ke; e += blockDim.x) {
      int j = (int)(e % n), c = (int)(e / n);
      double v = 0.0;
      if (j >= se.col_off && j < se.col_off + se.ncols)
        v = Z[(int64_t)(j - se.col_off) * se.z_rs + (int64_t)c * se.z_cs];
      Zst[(int64_t)(col + c) * n + j] = v;
    }
    col += ke;
  }
}

// ------------------------------------------------------------------------------ CORE
// Cyclic parallel Jacobi for a symmetric K x K matrix (K even): A <- J^T A J until no
// off-diagonal entry is significant, V <- V J.  The rotation of each pair is the classical
// one that annihilates A_pq (Golub & Van Loan, "Matrix Computations", symmetric Schur
// decomposition); the K/2 disjoint pairs of one round of a round-robin tournament are rotated
// together.  FP64 division and square root are long FMA sequences on this GPU, so the angle
// t = tan(theta) is computed in FP32 from exactly formed FP64 differences (its relative
// error only slows convergence from quadratic to a factor 1e-7 per sweep), and
// c = 1/sqrt(1 + t^2), s = t c are then made orthogonal to FP64 accuracy by two Newton steps.
// An entry is significant if A_pq^2 > u^2 |A_pp A_qq| and |A_pq| > abs_tol (the absolute
// floor keeps noise-level eigenvalues from being chased to the sweep limit).
template <typename T>
__device__ void jacobi_eigen(T* A, int lda, T* V, int ldv, int K, T* cs, T* sn, int* pa, int* pb, int* flag,
                             T abs_tol, int max_sweeps) {
  const int tid = threadIdx.x, nt = blockDim.x;
  const int half = K / 2;
  const T rel2 = sizeof(T) == 8 ? (T)4.9e-32 : (T)1.5e-14;   // (unit roundoff)^2
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    if (tid == 0) *flag = 0;
    __syncthreads();
    for (int r = 0; r < K - 1; ++r) {
      for (int q = tid; q < half; q += nt) {
        int x = q == 0 ? 0 : 1 + (q - 1 + r) % (K - 1);
        int yq = K - 1 - q;
        int y = 1 + (yq - 1 + r) % (K - 1);
        int a = min(x, y), b = max(x, y);
        pa[q] = a;
        pb[q] = b;
        const T app = A[a + (int64_t)a * lda], aqq = A[b + (int64_t)b * lda], apq = A[a + (int64_t)b * lda];
        T c = 1, s = 0;
        const T aa = apq < 0 ? -apq : apq;
        if (aa > abs_tol && aa * aa > rel2 * (app * aqq < 0 ? -app * aqq : app * aqq)) {
          if (sizeof(T) == 8) {
            // FP32 angle from exactly formed FP64 operands scaled into FP32 range, then an
            // exactly orthogonal FP64 pair (c, s) by two Newton steps for 1/sqrt(1 + t^2)
            const double num = (double)aqq - (double)app, den = 2.0 * (double)apq;
            int e;
            frexp(fmax(fabs(num), fabs(den)), &e);
            const float th = (float)ldexp(num, -e) / (float)ldexp(den, -e);
            float tf;
            if (!(fabsf(th) < 1e18f)) tf = 0.0f;
            else tf = copysignf(1.0f, th) / (fabsf(th) + sqrtf(fmaf(th, th, 1.0f)));
            const double t = (double)tf;
            const double x2 = fma(t, t, 1.0);
            double yv = (double)rsqrtf((float)x2);
            yv = yv * fma(-0.5 * x2, yv * yv, 1.5);
            yv = yv * fma(-0.5 * x2, yv * yv, 1.5);
            c = (T)yv;
            s = (T)(t * yv);
          } else {
            const float th = ((float)aqq - (float)app) / (2.0f * (float)apq);
            float tf;
            if (!(fabsf(th) < 1e18f)) tf = 0.0f;
            else tf = copysignf(1.0f, th) / (fabsf(th) + sqrtf(fmaf(th, th, 1.0f)));
            const float cf = rsqrtf(fmaf(tf, tf, 1.0f));
            c = (T)cf;
            s = (T)(tf * cf);
          }
          if (s != 0) *flag = 1;
        }
        cs[q] = c;
        sn[q] = s;
      }
      __syncthreads();
      for (int e = tid; e < half * K; e += nt) {   // rows a, b of A
        int q = e / K, j = e % K;
        T c = cs[q], s = sn[q];
        if (s == 0) continue;
        int a = pa[q], b = pb[q];
        T xa = A[a + (int64_t)j * lda], xb = A[b + (int64_t)j * lda];
        A[a + (int64_t)j * lda] = c * xa - s * xb;
        A[b + (int64_t)j * lda] = s * xa + c * xb;
      }
      __syncthreads();
      for (int e = tid; e < half * K; e += nt) {   // columns a, b of A and V
        int q = e / K, j = e % K;
        T c = cs[q], s = sn[q];
        if (s == 0) continue;
        int a = pa[q], b = pb[q];
        T xa = A[j + (int64_t)a * lda], xb = A[j + (int64_t)b * lda];
        A[j + (int64_t)a * lda] = c * xa - s * xb;
        A[j + (int64_t)b * lda] = s * xa + c * xb;
        T va = V[j + (int64_t)a * ldv], vb = V[j + (int64_t)b * ldv];
        V[j + (int64_t)a * ldv] = c * va - s * vb;
        V[j + (int64_t)b * ldv] = s * va + c * vb;
      }
      __syncthreads();
    }
    if (*flag == 0) break;
    __syncthreads();
  }
}

// C (n x n, ldc) = op(A) B for n x n operands (op(A) = A or A^T), one output element per
// thread iteration; used for the small products of the eigen-solver polish.
__device__ void small_mm(double* C, int ldc, const double* A, int lda, bool transA, const double* B, int ldb,
                         int n) {
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
    const int i = e % n, j = e / n;
    double s = 0.0;
    if (transA)
      for (int l = 0; l < n; ++l) s = fma(A[l + (int64_t)i * lda], B[l + (int64_t)j * ldb], s);
    else
      for (int l = 0; l < n; ++l) s = fma(A[i + (int64_t)l * lda], B[l + (int64_t)j * ldb], s);
    C[i + (int64_t)j * ldc] = s;
  }
}

constexpr int KMAX = 256;       // largest stacked rank of one rounded addition
constexpr int JSM = 64;         // Jacobi problems up to this size run in shared memory

__global__ void __launch_bounds__(512) k_core(const TruncOp* __restrict__ ops, Bases B) {
  const TruncOp op = ops[blockIdx.x];
  extern __shared__ double smem[];            // 2 * JSM * (JSM + 1) doubles
  __shared__ double d[KMAX], dinv[KMAX], rdinv[KMAX], lam[KMAX], cs[KMAX / 2], sn[KMAX / 2], red[32];
  __shared__ int perm[KMAX], pa[KMAX / 2], pb[KMAX / 2], order[KMAX], s_int[4];
  const int tid = threadIdx.x, nt = blockDim.x;
  const int K = *iptr(B, op.Kd);
  int* rk = iptr(B, op.rank);
  const int m = op.m, n = op.n, Kc = op.Kcap;
  if (K <= 0) {
    if (tid == 0) *rk = 0;
    return;
  }
  double* Gw = dptr(B, op.Gw);
  double* Gz = dptr(B, op.Gz);
  double* work = dptr(B, op.work);
  double* R = Gw;                              // K x K (ld Kc): equilibrated Gram -> Cholesky, in place
  double* Bm = work;                           // K x r
  double* T1 = work + (int64_t)Kc * Kc;        // K x r
  double* M = Gz;                              // r x r (global fallback for Jacobi; Gz is dead by then)
  // 1. equilibrate the Gram matrix of the stacked left factor
  for (int i = tid; i < K; i += nt) {
    double g = Gw[i + (int64_t)i * Kc];
    d[i] = g > 0.0 ? sqrt(g) : 1.0;
    dinv[i] = 1.0 / d[i];
    perm[i] = i;
  }
  __syncthreads();
  for (int e = tid; e < K * K; e += nt) {
    int i = e % K, j = e / K;
    R[i + (int64_t)j * Kc] = R[i + (int64_t)j * Kc] * (dinv[i] * dinv[j]);
  }
  __syncthreads();
  // 2. pivoted Cholesky G = Pi R^T R Pi^T (upper R in pivoted order, stored in place);
  //    stop when the largest remaining diagonal is below the noise level of the Gram.
  const double tolc = 4.0 * K * 2.2e-16;
  int r = 0;
  for (int j = 0; j < K; ++j) {
    if (tid < 32) {
      double bv = -1.0;
      int bi = -1;
      for (int i = j + tid; i < K; i += 32) {
        double v = R[perm[i] + (int64_t)perm[i] * Kc];
        if (v > bv) { bv = v; bi = i; }
      }
      for (int o = 16; o > 0; o >>= 1) {
        double ov = __shfl_xor_sync(0xffffffffu, bv, o);
        int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ov > bv || (ov == bv && oi >= 0 && (bi < 0 || oi < bi))) { bv = ov; bi = oi; }
      }
      if (tid == 0) {
        s_int[0] = bi;
        red[0] = bv;
      }
    }
    __syncthreads();
    const double piv = red[0];
    if (!(piv > tolc)) break;
    if (tid == 0) {
      int t = perm[j];
      perm[j] = perm[s_int[0]];
      perm[s_int[0]] = t;
    }
    __syncthreads();
    // R is kept in original index space: row pj of the factor is stored in column pj
    const int pj = perm[j];
    const double rjj = sqrt(piv);
    const double rinv = 1.0 / rjj;
    // column j of R^T in pivoted order: l_i = G(pi_i, pj) / rjj for i > j
    for (int i = j + 1 + tid; i < K; i += nt) {
      int pi = perm[i];
      R[pi + (int64_t)pj * Kc] = R[pi + (int64_t)pj * Kc] * rinv;
    }
    if (tid == 0) R[pj + (int64_t)pj * Kc] = rjj;
    __syncthreads();
    const int rem = K - 1 - j;
    for (int e = tid; e < rem * rem; e += nt) {
      int ii = j + 1 + e % rem, jj = j + 1 + e / rem;
      if (jj < ii) continue;   // update the lower triangle (pi_ii, pi_jj), ii <= jj, symmetric use
      int pi = perm[ii], pk = perm[jj];
      double v = R[pi + (int64_t)pk * Kc] - R[pi + (int64_t)pj * Kc] * R[pk + (int64_t)pj * Kc];
      R[pi + (int64_t)pk * Kc] = v;
      R[pk + (int64_t)pi * Kc] = v;
    }
    __syncthreads();
    ++r;
  }
  // factor entries: Rf(q, l) for q < r, l >= q in pivoted positions = R[perm[l] + perm[q]*Kc]
  // (diagonal: R[perm[q] + perm[q]*Kc]).
  if (r == 0) {
    if (tid == 0) *rk = 0;
    return;
  }
  // 3. Bm = D Pi Rf^T  (K x r): Bm(perm[l], q) = d[perm[l]] * Rf(q, l) for l >= q
  for (int e = tid; e < K * r; e += nt) {
    int l = e % K, q = e / K;
    int pl = perm[l];
    double v = 0.0;
    if (l >= q) v = d[pl] * R[pl + (int64_t)perm[q] * Kc];
    Bm[pl + (int64_t)q * Kc] = v;
  }
  __syncthreads();
  // 4. M = Bm^T Gz Bm  (r x r)
  for (int e = tid; e < K * r; e += nt) {
    int i = e % K, q = e / K;
    double s = 0.0;
    for (int l = 0; l < K; ++l) s = fma(Gz[i + (int64_t)l * Kc], Bm[l + (int64_t)q * Kc], s);
    T1[i + (int64_t)q * Kc] = s;
  }
  __syncthreads();
  const int rp = r + (r & 1);                  // even size for the round-robin ordering
  double* Mj;
  double* Yj;
  int ldj;
  if (rp <= JSM) {
    Mj = smem;
    Yj = smem + JSM * (JSM + 1);
    ldj = JSM + 1;
  } else {
    Mj = M;
    Yj = T1 + 0;   // T1 is free again after M is formed; reuse below
    ldj = Kc;
  }
  // M into registers-then-store to allow Yj to alias T1 in the global fallback
  for (int e = tid; e < rp * rp; e += nt) {
    int p = e % rp, q = e / rp;
    double s = 0.0;
    if (p < r && q < r) {
      for (int i = 0; i < K; ++i) s = fma(Bm[i + (int64_t)p * Kc], T1[i + (int64_t)q * Kc], s);
    }
    if (rp > JSM) M[p + (int64_t)q * Kc] = s;
    else Mj[p + q * ldj] = s;
  }
  __syncthreads();
  if (rp > JSM) {
    // symmetrise in place
    for (int e = tid; e < rp * rp; e += nt) {
      int p = e % rp, q = e / rp;
      if (p < q) {
        double v = 0.5 * (M[p + (int64_t)q * Kc] + M[q + (int64_t)p * Kc]);
        M[p + (int64_t)q * Kc] = v;
        M[q + (int64_t)p * Kc] = v;
      }
    }
  } else {
    for (int e = tid; e < rp * rp; e += nt) {
      int p = e % rp, q = e / rp;
      if (p < q) {
        double v = 0.5 * (Mj[p + q * ldj] + Mj[q + p * ldj]);
        Mj[p + q * ldj] = v;
        Mj[q + p * ldj] = v;
      }
    }
  }
  __syncthreads();
  for (int e = tid; e < rp * rp; e += nt) {
    int p = e % rp, q = e / rp;
    Yj[p + (int64_t)q * ldj] = (p == q) ? 1.0 : 0.0;
  }
  __syncthreads();
  // 5. eigen-decomposition of M = Y S Y^T (S = sigma^2 of the stacked product); entries
  //    below 1e-17 trace(M) are noise of the Gram formation and are not rotated away
  if (tid == 0) {
    double tr = 0.0;
    for (int q = 0; q < r; ++q) tr += fabs(Mj[q + (int64_t)q * ldj]);
    red[1] = tr;
  }
  __syncthreads();
  const double tr = red[1];
  if (rp <= JSM && tr > 0.0) {
    // Mixed precision: sweeps in FP32 on M / trace(M) (FP32 runs ~64x faster than FP64 on
    // this GPU), then in FP64: orthogonalise the FP32 eigenvectors by one Newton-Schulz step
    // Y <- Y (3 I - Y^T Y) / 2, form M1 = Y^T M Y (nearly diagonal) and finish with FP64
    // sweeps that accumulate onto Y. The eigenvalues come from the FP64 sweeps, so they keep
    // full accuracy; the FP32 stage only supplies a starting basis.
    double* Mg = T1;                     // global copy of M (ld Kc)
    double* G = Gz;                      // global temporary (ld Kc); Gz is dead here
    float* Mf = reinterpret_cast<float*>(Mj);            // two FP32 matrices inside Mj's buffer
    float* Yf = Mf + JSM * (JSM + 1);
    const int ldf = JSM + 1;
    __shared__ float csf[KMAX / 2], snf[KMAX / 2];
    for (int e = tid; e < rp * rp; e += nt) {
      const int p = e % rp, q = e / rp;
      Mg[p + (int64_t)q * Kc] = Mj[p + q * ldj];
    }
    __syncthreads();
    const double itr = 1.0 / tr;
    for (int e = tid; e < rp * rp; e += nt) {
      const int p = e % rp, q = e / rp;
      Mf[p + q * ldf] = (float)(Mg[p + (int64_t)q * Kc] * itr);
      Yf[p + q * ldf] = (p == q) ? 1.0f : 0.0f;
    }
    __syncthreads();
    jacobi_eigen<float>(Mf, ldf, Yf, ldf, rp, csf, snf, pa, pb, &s_int[1], 1e-12f, 12);
    __syncthreads();
    for (int e = tid; e < rp * rp; e += nt) {
      const int p = e % rp, q = e / rp;
      Yj[p + q * ldj] = (double)Yf[p + q * ldf];
    }
    __syncthreads();
    small_mm(Mj, ldj, Yj, ldj, true, Yj, ldj, rp);            // P = Y^T Y
    __syncthreads();
    small_mm(G, Kc, Yj, ldj, false, Mj, ldj, rp);             // Y P
    __syncthreads();
    for (int e = tid; e < rp * rp; e += nt) {
      const int p = e % rp, q = e / rp;
      Yj[p + q * ldj] = 1.5 * Yj[p + q * ldj] - 0.5 * G[p + (int64_t)q * Kc];
    }
    __syncthreads();
    small_mm(Mj, ldj, Mg, Kc, false, Yj, ldj, rp);            // T = M Y
    __syncthreads();
    small_mm(G, Kc, Yj, ldj, true, Mj, ldj, rp);              // M1 = Y^T T
    __syncthreads();
    for (int e = tid; e < rp * rp; e += nt) {
      const int p = e % rp, q = e / rp;
      Mj[p + q * ldj] = 0.5 * (G[p + (int64_t)q * Kc] + G[q + (int64_t)p * Kc]);
    }
    __syncthreads();
    jacobi_eigen<double>(Mj, ldj, Yj, ldj, rp, cs, sn, pa, pb, &s_int[1], 1e-17 * tr, 40);
  } else {
    jacobi_eigen<double>(Mj, ldj, Yj, ldj, rp, cs, sn, pa, pb, &s_int[1], 1e-17 * tr, 40);
  }
  __syncthreads();
  for (int q = tid; q < r; q += nt) lam[q] = Mj[q + (int64_t)q * ldj];
  __syncthreads();
  // 6. order the eigenvalues (descending, ties by index) and choose the rank; the order
  //    array is first the identity so that it stays a valid index list even with NaNs
  for (int q = tid; q < r; q += nt) order[q] = q;
  __syncthreads();
  for (int q = tid; q < r; q += nt) {
    int pos = 0;
    double v = lam[q];
    for (int p = 0; p < r; ++p)
      if (lam[p] > v || (lam[p] == v && p < q)) ++pos;
    order[pos] = q;
  }
  __syncthreads();
  const double smax = lam[order[0]];
  const double thr = op.eps * op.eps * smax;
  int kk = 0;
  if (smax > 0.0)
    for (int p = 0; p < r; ++p)
      if (lam[order[p]] > thr) ++kk;
  if (kk > op.cap) {
    if (tid == 0) atomicAdd(&B.status[1], 1);
    kk = op.cap;
  }
  // 7. coefficient matrices: Tz = Bm Y_k S_k^{-1/2}, Tw = D^{-1} Pi_r Rf11^{-1} Y_k S_k^{1/2}
  double* Tw = dptr(B, op.Tw);
  double* Tz = dptr(B, op.Tz);
  __syncthreads();
  if (tid < kk) {
    const double sg = sqrt(lam[order[tid]]);
    cs[tid] = sg;          // sigma of the c-th kept direction
    sn[tid] = 1.0 / sg;
  }
  __syncthreads();
  for (int e = tid; e < K * kk; e += nt) {
    int i = e % K, c = e / K;
    int q = order[c];
    double s = 0.0;
    for (int p = 0; p < r; ++p) s = fma(Bm[i + (int64_t)p * Kc], Yj[p + (int64_t)q * ldj], s);
    Tz[i + (int64_t)c * Kc] = s * sn[c];
  }
  // back substitution Rf11 x = Y_k S^{1/2} (Rf11 upper r x r in pivoted order); x lives in
  // rows perm[0..r) of Tw, the other rows of Tw are zero.
  for (int e = tid; e < K * kk; e += nt) {
    int i = e % K, c = e / K;
    Tw[i + (int64_t)c * Kc] = 0.0;
  }
  __syncthreads();
  // reciprocals of the Cholesky diagonal
  for (int l = tid; l < r; l += nt) rdinv[l] = 1.0 / R[perm[l] + (int64_t)perm[l] * Kc];
  __syncthreads();
  for (int c = tid; c < kk; c += nt) {
    int q = order[c];
    double sig = cs[c];
    for (int l = r - 1; l >= 0; --l) {
      double s = Yj[l + (int64_t)q * ldj] * sig;
      for (int p = l + 1; p < r; ++p)
        s = fma(-R[perm[p] + (int64_t)perm[l] * Kc], Tw[perm[p] + (int64_t)c * Kc], s);
      Tw[perm[l] + (int64_t)c * Kc] = s * rdinv[l];
    }
  }
  __syncthreads();
  // undo the equilibration: rows of Tw scale by 1/d_i
  for (int e = tid; e < K * kk; e += nt) {
    int i = e % K, c = e / K;
    Tw[i + (int64_t)c * Kc] *= dinv[i];
  }
  __syncthreads();
  if (tid == 0) {
    *rk = kk;
    double Kd = K;
    auto qr = [](double mm, double kq) {
      return mm >= kq ? 2.0 * mm * kq * kq - 2.0 * kq * kq * kq / 3.0
                      : 2.0 * kq * mm * mm - 2.0 * mm * mm * mm / 3.0;
    };
    double f = qr(m, Kd) + qr(n, Kd) + 23.0 * Kd * Kd * Kd + 2.0 * (m + n) * Kd * kk;
    atomicAdd(&B.flops[FC_TRUNC], (unsigned long long)f);
    // the core's own share of the model: product of the triangular factors + SVD of K x K
    atomicAdd(&B.flops[NFC + K_CORE], (unsigned long long)(23.0 * Kd * Kd * Kd));
  }
}

// ------------------------------------------------------------------------------ assembly
__device__ __forceinline__ double kernel_entry(const double* P, int i, int j, double h) {
  double dx = P[3 * i] - P[3 * j], dy = P[3 * i + 1] - P[3 * j + 1], dz = P[3 * i + 2] - P[3 * j + 2];
  double r = sqrt(dx * dx + dy * dy + dz * dz);
  return 1.0 / (4.0 * M_PI * (r + h));
}

__global__ void __launch_bounds__(256) k_eval(const EvalOp* __restrict__ ops, Bases B, double h) {
  const EvalOp op = ops[blockIdx.x];
  const double* P = B.d[SP_P];
  double* D = dptr(B, op.D);
  const int64_t tot = (int64_t)op.m * op.n;
  for (int64_t e = threadIdx.x; e < tot; e += blockDim.x) {
    int i = (int)(e % op.m), j = (int)(e / op.m);
    D[e] = kernel_entry(P, op.r0 + i, op.c0 + j, h);
  }
}

// Adaptive cross approximation with partial pivoting (Bebendorf 2000): rank-one cross
// terms u v^T of the residual, chosen by the largest residual entry of a row, stopped when
// |u||v| <= tol |S_k|_F.
__global__ void __launch_bounds__(256) k_aca(const AcaOp* __restrict__ ops, Bases B, double h) {
  const AcaOp op = ops[blockIdx.x];
  const int m = op.m, n = op.n, tid = threadIdx.x, nt = blockDim.x;
  const double* P = B.d[SP_P];
  double* U = dptr(B, op.U);
  double* V = dptr(B, op.V);
  int* used = iptr(B, op.used);
  __shared__ double coef[256], red[32], dots[2 * 256];
  __shared__ int redi[32];
  __shared__ double s_norm2;
  __shared__ int s_i, s_k;
  for (int i = tid; i < m; i += nt) used[i] = 0;
  if (tid == 0) {
    s_i = 0;
    s_k = 0;
    s_norm2 = 0.0;
  }
  __syncthreads();
  const int kmax = min(op.kmax, 256);
  for (int guard = 0; guard < kmax + m; ++guard) {
    const int k = s_k;
    if (k >= kmax) break;
    const int i = s_i;
    for (int l = tid; l < k; l += nt) coef[l] = U[i + (int64_t)l * m];
    __syncthreads();
    double* v = V + (int64_t)k * n;
    double bv = -1.0;
    int bj = -1;
    for (int j = tid; j < n; j += nt) {
      double x = kernel_entry(P, op.r0 + i, op.c0 + j, h);
      for (int l = 0; l < k; ++l) x = fma(-coef[l], V[j + (int64_t)l * n], x);
      v[j] = x;
      double ax = fabs(x);
      if (ax > bv) { bv = ax; bj = j; }
    }
    if (tid == 0) used[i] = 1;
    const int jstar = block_argmax(bv, bj, red, redi);
    const double pivot = v[jstar];
    if (pivot == 0.0) {
      // zero residual row: continue with the first unused row, if any
      int cand = m;
      for (int q = tid; q < m; q += nt)
        if (!used[q]) { cand = q; break; }
      for (int o = 16; o > 0; o >>= 1) cand = min(cand, __shfl_xor_sync(0xffffffffu, cand, o));
      if ((tid & 31) == 0) redi[tid >> 5] = cand;
      __syncthreads();
      if (tid == 0) {
        int c = m;
        for (int w = 0; w < nt / 32; ++w) c = min(c, redi[w]);
        s_i = c;
      }
      __syncthreads();
      if (s_i >= m) break;
      continue;
    }
    for (int j = tid; j < n; j += nt) v[j] = v[j] / pivot;
    for (int l = tid; l < k; l += nt) coef[l] = V[jstar + (int64_t)l * n];
    __syncthreads();
    double* u = U + (int64_t)k * m;
    for (int q = tid; q < m; q += nt) {
      double x = kernel_entry(P, op.r0 + q, op.c0 + jstar, h);
      for (int l = 0; l < k; ++l) x = fma(-coef[l], U[q + (int64_t)l * m], x);
      u[q] = x;
    }
    __syncthreads();
    // dot products with the previous terms and the new norms, one pass, warp partials
    for (int l = tid; l < 2 * (k + 1); l += nt) dots[l] = 0.0;
    __syncthreads();
    for (int l = 0; l <= k; ++l) {
      double su = 0.0, sv = 0.0;
      for (int q = tid; q < m; q += nt) su = fma(U[q + (int64_t)l * m], u[q], su);
      for (int q = tid; q < n; q += nt) sv = fma(V[q + (int64_t)l * n], v[q], sv);
      for (int o = 16; o > 0; o >>= 1) {
        su += __shfl_xor_sync(0xffffffffu, su, o);
        sv += __shfl_xor_sync(0xffffffffu, sv, o);
      }
      if ((tid & 31) == 0) {
        atomicAdd(&dots[2 * l], su);
        atomicAdd(&dots[2 * l + 1], sv);
      }
    }
    __syncthreads();
    // next pivot row: largest |u| among unused rows
    double bu = -1.0;
    int bi = -1;
    for (int q = tid; q < m; q += nt)
      if (!used[q]) {
        double a = fabs(u[q]);
        if (a > bu) { bu = a; bi = q; }
      }
    const int inext = block_argmax(bu, bi, red, redi);
    if (tid == 0) {
      double cross = 0.0;
      for (int l = 0; l < k; ++l) cross += dots[2 * l] * dots[2 * l + 1];
      double uu = dots[2 * k], vv = dots[2 * k + 1];
      s_norm2 = s_norm2 + 2.0 * cross + uu * vv;
      s_k = k + 1;
      bool stop = sqrt(uu * vv) <= op.tol * sqrt(fabs(s_norm2));
      s_i = (stop || inext < 0) ? -1 : inext;
    }
    __syncthreads();
    if (s_i < 0) break;
  }
  __syncthreads();
  if (tid == 0) {
    *iptr(B, op.kd) = s_k;
    if (s_k >= kmax) atomicAdd(&B.status[2], 1);
  }
}

// ------------------------------------------------------------------------------ misc
// nearest-neighbour squared distance of every point (brute force, tiled through smem)
__global__ void __launch_bounds__(256) k_nn2(const double* __restrict__ P, int n, double* out) {
  __shared__ double tile[256 * 3];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  double xi = 0, yi = 0, zi = 0;
  if (i < n) { xi = P[3 * i]; yi = P[3 * i + 1]; zi = P[3 * i + 2]; }
  double best = INFINITY;
  for (int t0 = 0; t0 < n; t0 += 256) {
    int j = t0 + threadIdx.x;
    if (j < n) {
      tile[3 * threadIdx.x] = P[3 * j];
      tile[3 * threadIdx.x + 1] = P[3 * j + 1];
      tile[3 * threadIdx.x + 2] = P[3 * j + 2];
    }
    __syncthreads();
    int cnt = min(256, n - t0);
    for (int q = 0; q < cnt; ++q) {
      double dx = xi - tile[3 * q], dy = yi - tile[3 * q + 1], dz = zi - tile[3 * q + 2];
      double d2 = dx * dx + dy * dy + dz * dz;
      if (t0 + q != i && d2 < best) best = d2;
    }
    __syncthreads();
  }
  if (i < n) out[i] = best;
}

// y(:, c) (+)= alpha * A_exact x(:, c): kernel entries evaluated on the fly, in ORIGINAL order
__global__ void __launch_bounds__(256) k_exact_mv(const double* __restrict__ P, int n, double h,
                                                  const double* __restrict__ x, int64_t ldx,
                                                  double* y, int64_t ldy, int nrhs) {
  __shared__ double tile[256 * 3];
  __shared__ double xs[256 * 8];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  double xi = 0, yi = 0, zi = 0;
  if (i < n) { xi = P[3 * i]; yi = P[3 * i + 1]; zi = P[3 * i + 2]; }
  for (int c0 = 0; c0 < nrhs; c0 += 8) {
    const int nc = min(8, nrhs - c0);
    double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int t0 = 0; t0 < n; t0 += 256) {
      int j = t0 + threadIdx.x;
      if (j < n) {
        tile[3 * threadIdx.x] = P[3 * j];
        tile[3 * threadIdx.x + 1] = P[3 * j + 1];
        tile[3 * threadIdx.x + 2] = P[3 * j + 2];
        for (int c = 0; c < nc; ++c) xs[c * 256 + threadIdx.x] = x[j + (int64_t)(c0 + c) * ldx];
      }
      __syncthreads();
      int cnt = min(256, n - t0);
      for (int q = 0; q < cnt; ++q) {
        double dx = xi - tile[3 * q], dy = yi - tile[3 * q + 1], dz = zi - tile[3 * q + 2];
        double a = 1.0 / (4.0 * M_PI * (sqrt(dx * dx + dy * dy + dz * dz) + h));
        for (int c = 0; c < nc; ++c) acc[c] = fma(a, xs[c * 256 + q], acc[c]);
      }
      __syncthreads();
    }
    if (i < n)
      for (int c = 0; c < nc; ++c) y[i + (int64_t)(c0 + c) * ldy] = acc[c];
  }
}

// dst(k, c) = src(perm[k], c) (gather) or dst(perm[k], c) = src(k, c) (scatter), with
// dst = alpha * value + beta * dst when beta_mode is set
__global__ void k_permute(const double* __restrict__ src, int64_t lds, double* dst, int64_t ldd,
                          const int64_t* __restrict__ perm, int n, int nrhs, int scatter,
                          double alpha, double beta, int accumulate) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)n * nrhs) return;
  int k = (int)(e % n), c = (int)(e / n);
  int64_t p = perm[k];
  double v;
  double* d;
  if (scatter) {
    v = src[k + c * lds];
    d = dst + p + c * ldd;
  } else {
    v = src[p + c * lds];
    d = dst + k + c * ldd;
  }
  *d = accumulate ? alpha * v + (beta == 0.0 ? 0.0 : beta * *d) : v;
}

__global__ void k_set_int(int* p, int v) { *p = v; }

__global__ void k_permute_points(const double* __restrict__ P, const int64_t* __restrict__ perm,
                                 int n, double* out) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  int64_t p = perm[k];
  out[3 * k] = P[3 * p];
  out[3 * k + 1] = P[3 * p + 1];
  out[3 * k + 2] = P[3 * p + 2];
}

// ------------------------------------------------------------------------------ launchers
static bool g_attr_set = false;
constexpr int TRSM_SMEM = 2 * 64 * 65 * (int)sizeof(double);
constexpr int CORE_SMEM = 2 * JSM * (JSM + 1) * (int)sizeof(double);

static void set_attributes() {
  if (g_attr_set) return;
  cudaFuncSetAttribute(k_trsm, cudaFuncAttributeMaxDynamicSharedMemorySize, TRSM_SMEM);
  cudaFuncSetAttribute(k_core, cudaFuncAttributeMaxDynamicSharedMemorySize, CORE_SMEM);
  g_attr_set = true;
}

void prepare_kernels() { set_attributes(); }

cudaError_t launch_kind(int kind, const void* ops, int count, const StackEntry* entries, const Bases& B,
                        double h, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  set_attributes();
  switch (kind) {
    case K_GETRF: k_getrf<<<count, 256, 0, s>>>((const GetrfOp*)ops, B); break;
    case K_TRSM: k_trsm<<<count, 256, TRSM_SMEM, s>>>((const TrsmOp*)ops, B); break;
    case K_GEMM: k_gemm<<<count, 256, 0, s>>>((const GemmOp*)ops, B); break;
    case K_COPY: k_copy<<<count, 256, 0, s>>>((const CopyOp*)ops, B); break;
    case K_STACK: k_stack<<<count, 256, 0, s>>>((const TruncOp*)ops, entries, B); break;
    case K_CORE: k_core<<<count, 512, CORE_SMEM, s>>>((const TruncOp*)ops, B); break;
    case K_EVAL: k_eval<<<count, 256, 0, s>>>((const EvalOp*)ops, B, h); break;
    case K_ACA: k_aca<<<count, 256, 0, s>>>((const AcaOp*)ops, B, h); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_nn2(const double* P, int n, double* out, cudaStream_t s) {
  k_nn2<<<(n + 255) / 256, 256, 0, s>>>(P, n, out);
  return cudaGetLastError();
}

cudaError_t launch_exact_mv(const double* P, int n, double h, const double* x, int64_t ldx, double* y,
                            int64_t ldy, int nrhs, cudaStream_t s) {
  k_exact_mv<<<(n + 255) / 256, 256, 0, s>>>(P, n, h, x, ldx, y, ldy, nrhs);
  return cudaGetLastError();
}

cudaError_t launch_permute(const double* src, int64_t lds, double* dst, int64_t ldd, const int64_t* perm,
                           int n, int nrhs, int scatter, double alpha, double beta, int accumulate,
                           cudaStream_t s) {
  int64_t tot = (int64_t)n * nrhs;
  if (tot == 0) return cudaSuccess;
  k_permute<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(src, lds, dst, ldd, perm, n, nrhs, scatter, alpha,
                                                          beta, accumulate);
  return cudaGetLastError();
}

cudaError_t launch_set_int(int* p, int v, cudaStream_t s) {
  k_set_int<<<1, 1, 0, s>>>(p, v);
  return cudaGetLastError();
}

cudaError_t launch_permute_points(const double* P, const int64_t* perm, int n, double* out, cudaStream_t s) {
  k_permute_points<<<(n + 255) / 256, 256, 0, s>>>(P, perm, n, out);
  return cudaGetLastError();
}

}  // namespace hm

namespace hm {

// squared 2-norm of every column (one CTA per column)
__global__ void __launch_bounds__(256) k_colnorm2(const double* __restrict__ x, int64_t ld, int n, double* out) {
  __shared__ double red[32];
  const double* c = x + (int64_t)blockIdx.x * ld;
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s = fma(c[i], c[i], s);
  s = block_sum(s, red);
  if (threadIdx.x == 0) out[blockIdx.x] = s;
}

// y(:, c) = alpha x(:, c) + beta y(:, c)
__global__ void k_axpby(const double* __restrict__ x, int64_t ldx, double* y, int64_t ldy, int n, int nrhs,
                        double alpha, double beta) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)n * nrhs) return;
  int i = (int)(e % n), c = (int)(e / n);
  double* d = y + i + c * ldy;
  *d = alpha * x[i + c * ldx] + (beta == 0.0 ? 0.0 : beta * *d);
}

cudaError_t launch_colnorm2(const double* x, int64_t ld, int n, int nrhs, double* out, cudaStream_t s) {
  if (nrhs <= 0) return cudaSuccess;
  k_colnorm2<<<nrhs, 256, 0, s>>>(x, ld, n, out);
  return cudaGetLastError();
}

cudaError_t launch_axpby(const double* x, int64_t ldx, double* y, int64_t ldy, int n, int nrhs, double alpha,
                         double beta, cudaStream_t s) {
  int64_t tot = (int64_t)n * nrhs;
  if (tot == 0) return cudaSuccess;
  k_axpby<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(x, ldx, y, ldy, n, nrhs, alpha, beta);
  return cudaGetLastError();
}

}  // namespace hm
