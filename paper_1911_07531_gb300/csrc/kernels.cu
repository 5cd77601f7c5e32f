// Batched FP64 kernels of the H-LU hot path (one CTA per micro-op).
//
// GB300 has very little FP64 throughput (about 2 DFMA per clock per SM, ~64 cycles of latency
// per dependent FP64 operation), so every kernel here is FP64-issue bound once the operands sit
// in shared memory or L1/L2, and serial FP64 chains dominate the small factorisations. The
// design keeps the DFMA pipes busy without padding (exact-size GEMM tiles, large micro-ops
// spread over several CTAs), moves decisions and iterations that tolerate it to FP32 or the
// integer pipe, and keeps a whole wave on the device with no host round trip.
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

// FP64 reciprocal and reciprocal square root by Newton-Raphson iteration from FP32 seeds
// (x = m 2^e with m in [0.5, 2); two Newton steps take the ~1e-7 seed to full precision).
// FP64 division and square root are long dependent instruction sequences on this GPU; these
// serve the serial paths (pivots of LU and Cholesky), where their latency is exposed.
__device__ __forceinline__ double nr_rcp(double x) {
  int e;
  const double m = frexp(x, &e);
  double y = (double)(1.0f / (float)m);
  double r = fma(-m, y, 1.0);
  y = fma(y, r, y);
  r = fma(-m, y, 1.0);
  y = fma(y, r, y);
  return ldexp(y, -e);
}

__device__ __forceinline__ double nr_rsqrt(double x) {
  int e;
  double m = frexp(x, &e);
  if (e & 1) {
    m *= 2.0;
    e -= 1;
  }
  double y = (double)rsqrtf((float)m);
  y = y * fma(-0.5 * m, y * y, 1.5);
  y = y * fma(-0.5 * m, y * y, 1.5);
  return ldexp(y, -e / 2);
}

// Reciprocal of x in [1e-30, 1e30] to full FP64 accuracy with three dependent FP64 operations:
// r0 = 1/x from the FP32 approximate reciprocal (the FP32 operand and the FP64 seed are formed
// by integer moves of the exponent and the leading mantissa bits, not by conversion
// instructions), e = 1 - x r0 (|e| < 2^-21), 1/x = r0 (1 + e + e^2 + ...); the truncated series
// leaves r0 e^3 ~ 2^-63 r0.
// GB300 spends ~64 cycles on each dependent FP64 operation, so this is for serial sections.
__device__ __forceinline__ double fast_rcp(double x) {
  constexpr long long kBias = (long long)(1023 - 127) << 23;   // exponent rebias, FP32 bit position
  const long long xb = __double_as_longlong(x);
  const float xf = __int_as_float((int)((xb >> 29) - kBias));
  float rf;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(rf) : "f"(xf));   // ~1 ulp; the series absorbs it
  const double r0 = __longlong_as_double(((long long)__float_as_int(rf) + kBias) << 29);
  const double e = fma(-x, r0, 1.0);
  return fma(r0, fma(e, e, e), r0);
}

// Reciprocal of a nonzero pivot: fast_rcp inside [1e-30, 1e30] (bounds compared on the bit
// patterns of |v|), Newton-Raphson from a rescaled seed outside.
__device__ __forceinline__ double pivot_rcp(double v) {
  const long long mag = __double_as_longlong(fabs(v));
  if (mag > 0x39b4484bfeebc2a0LL && mag < 0x46293e5939a08ceaLL)   // 1e-30 < |v| < 1e30
    return copysign(fast_rcp(fabs(v)), v);
  return nr_rcp(v);
}

// Total order of doubles as signed 64-bit integers (negative values have their magnitude bits
// flipped): comparisons on the integer pipe instead of ~64-cycle FP64 compares.
__device__ __forceinline__ long long order_key(double v) {
  const long long b = __double_as_longlong(v);
  return b < 0 ? b ^ 0x7fffffffffffffffLL : b;
}

// Pivot key of a diagonal entry at position i (< 256): the high word of a positive double
// (sign, exponent, 20 mantissa bits) with its low 8 bits replaced by 255 - i, so that an
// unsigned max picks the largest entry to ~2^-12 relative and the lowest index among near
// ties; 0 for entries <= 0.
__device__ __forceinline__ unsigned pivot_key(double v, int i) {
  const long long b = __double_as_longlong(v);
  return b > 0 ? (((unsigned)(b >> 32)) & ~255u) | (unsigned)(255 - i) : 0u;
}


// ------------------------------------------------------------------------------ GEMM
// GEMM micro-ops are thin (a rank-sized side of 10-60) or have a small output with a long
// reduction (Gram matrices). GB300 executes ~2 FP64 FMAs per clock per SM while shared memory
// delivers 16 doubles per clock, so the kernel needs no register blocking to keep the FP64 pipe
// busy, and register tiles of fixed shape would pad a 15 x 15 or 45 x 45 output to 16 x 16 or
// 64 x 64 (3.4x the useful FMAs on the H-LU plans). Instead the output is cut into exact tiles
// of at most GE elements (at most GTM rows and columns), each thread owns up to four output
// elements of a tile, and for tiles of fewer than 128 elements G = 2..8 threads split the
// reduction of one element (partial sums combined in shared memory). Slices of GKS reduction
// steps of both operands are staged in shared memory through two buffers: the next slice is
// fetched with cp.async while the current one is multiplied. A micro-op has a budget of CTAs
// along blockIdx.y (GemmOp::split), which the kernel divides between its C tiles and, for
// accumulating (atomic) micro-ops, reduction slices, from the actual sizes, so that a large
// micro-op does not sit on one SM.
constexpr int KMAX_ENTRIES = 256;   // largest number of pieces of one rounded addition (planner)
constexpr int GE = 1024;      // largest C tile (elements)
constexpr int GTM = 128;      // largest C tile side
constexpr int GKS = 16;       // staged reduction slice (two buffers: the next slice is fetched with
                              // cp.async while the current one is multiplied)
constexpr int GBUF = 2 * GKS * (GTM + 1);   // doubles of one buffer (A slice, then B slice)
constexpr int GEMM_SMEM = (2 * GBUF + 256) * (int)sizeof(double);
constexpr int GEMM32_SMEM = GEMM_SMEM + GBUF * (int)sizeof(float);

// 8-byte asynchronous copy global -> shared (zero-fill when !valid: no bytes are read)
__device__ __forceinline__ void cp_async8(double* dst, const double* src, bool valid) {
  const unsigned saddr = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(saddr), "l"(src), "r"(valid ? 8 : 0)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

__device__ __forceinline__ void gemm_tile_shape(int m, int n, int& mt, int& nt, int& nrt, int& nct) {
  nct = (n + GTM - 1) / GTM;
  nt = (n + nct - 1) / nct;
  const int capm = min(GTM, max(1, GE / nt));
  nrt = (m + capm - 1) / capm;
  mt = (m + nrt - 1) / nrt;
}

template <int W, typename T>
__device__ __forceinline__ void gemm_slice(const T* As, const T* Bs, int ks, const int (&ii)[4], const int (&jj)[4],
                                           T (&acc)[4]) {
  for (int l = 0; l < ks; ++l) {
    const T* a = As + l * (GTM + 1);
    const T* b = Bs + l * (GTM + 1);
#pragma unroll
    for (int j = 0; j < W; ++j) acc[j] = fma(a[ii[j]], b[jj[j]], acc[j]);
  }
}

// Entries (il, jl) of a tile at (i0, j0) with i0 + il <= j0 + jl, counted column by column:
// column jl holds clamp(jl + c0, 0, mi) of them (c0 = j0 - i0 + 1); sym_prefix(x) is the number
// in columns 0..x-1.
__device__ __forceinline__ int sym_tri(int v, int mi) {   // sum_{u=0}^{v-1} clamp(u, 0, mi)
  return v <= mi + 1 ? v * (v - 1) / 2 : mi * (mi + 1) / 2 + (v - mi - 1) * mi;
}
__device__ __forceinline__ int sym_prefix(int x, int c0, int mi) {
  return sym_tri(max(0, c0 + x), mi) - sym_tri(max(0, c0), mi);
}

// FP64 value to FP32 by integer moves of the exponent and the leading mantissa bits (mantissa
// truncated: relative error < 2^-23; magnitudes below the FP32 normal range become zero, above it
// infinity): conversions on the integer pipe instead of the narrow FP64 one.
__device__ __forceinline__ float f64_to_f32(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned hi = (unsigned)(b >> 32);
  const unsigned e = (hi >> 20) & 0x7ffu, sign = hi & 0x80000000u;
  unsigned f = sign | ((e - 896u) << 23) | ((unsigned)(b >> 29) & 0x7fffffu);
  f = e <= 896u ? sign : f;
  f = e >= 1151u ? (sign | 0x7f800000u) : f;
  return __uint_as_float(f);
}

// CT: arithmetic of the products. double: the FP64 GEMM. float (mixed precision): the staged FP64
// slices are converted to FP32 in shared memory and multiplied with FP32 FMAs and accumulators;
// the result is written in FP64.
template <typename CT>
__global__ void __launch_bounds__(256, 3) k_gemm_t(const GemmOp* __restrict__ ops, Bases B) {
  constexpr bool F32 = sizeof(CT) == 4;
  // CTAs beyond this micro-op's budget (the launch is sized for its largest) leave before any
  // other load
  const int split = ops[blockIdx.x].split;
  const int budget = max(1, split & 0xffff) * max(1, split >> 16);
  if ((int)blockIdx.y >= budget) return;
  const GemmOp op = ops[blockIdx.x];
  const int m = dimv(B, op.m, op.md), n = dimv(B, op.n, op.nd), k = max(dimv(B, op.k, op.kd), 0);
  const bool atomic = op.flags & GF_ATOMIC, overwrite = op.flags & GF_OVERWRITE;
  if (m <= 0 || n <= 0) return;
  if (k == 0 && !overwrite) return;
  const int nslices = (k + GKS - 1) / GKS;
  int mt, nt, nrt, nct;
  gemm_tile_shape(m, n, mt, nt, nrt, nct);
  // CTAs of this micro-op: the planner's budget (at most gridDim.y), lowered to the tuned work
  // per CTA for the actual sizes and factored here into C tiles (sy) times reduction slices (sz,
  // atomic micro-ops only), sy * sz <= budget. The factoring follows the actual sizes, so a Gram
  // product whose dynamic K x K output fits in a few tiles spreads its rows over the slices.
  const double work = (double)m * n * max(k, 1);
  const double per_cta = B.gemm_work > 0.f ? (double)B.gemm_work : 4096.0;
  const int want = min(budget, max(1, (int)ceil(work / per_cta)));
  const int sy = min(want, nrt * nct);
  const int sz = atomic ? max(1, min(want / sy, max(nslices, 1))) : 1;
  if ((int)blockIdx.y >= sy * sz) return;
  const int ty = (int)blockIdx.y % sy, z0 = (int)blockIdx.y / sy, zs = sz;
  extern __shared__ double gsm[];             // buffer b: A slice [GKS][GTM + 1], B slice [GKS][GTM + 1]
  double* red = gsm + 2 * GBUF;               // [256]
  float* fsl = (float*)(red + 256);           // FP32 copy of the current slice (F32 only)
  const double* A = dptr(B, op.A);
  const double* Bm = dptr(B, op.B);
  double* C = dptr(B, op.C);
  const int tid = threadIdx.x;
  const bool a_i_fast = op.a_rs <= op.a_cs;
  const bool b_j_fast = op.b_cs <= op.b_rs;
  const bool upper = op.flags & GF_A_UPPER, unitlower = op.flags & GF_A_UNITLOWER;
  const bool sym = op.flags & GF_SYM_UPPER;
  for (int tile = ty; tile < nrt * nct; tile += sy) {
    const int i0 = (tile % nrt) * mt, j0 = (tile / nrt) * nt;
    const int mi = min(mt, m - i0), nj = min(nt, n - j0);
    const int c0 = j0 - i0 + 1;
    if (sym && c0 + nj - 1 <= 0) continue;        // tile strictly below the diagonal
    const int ne = sym ? sym_prefix(nj, c0, mi) : mi * nj;
    int G = 1;
    while (G < 8 && ne * G * 2 <= 256) G *= 2;
    const int nslot = ne * G;
    // slots tid + 256 j (j < 4) of this thread; with G > 1 only slot 0 exists
    int ii[4], jj[4];
    int nmy = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int sl = tid + 256 * j;
      const int e = sl < nslot ? sl % ne : 0;
      if (sym) {
        int lo = 0, hi = nj - 1;                  // last column whose prefix is <= e
        while (lo < hi) {
          const int mid = (lo + hi + 1) >> 1;
          if (sym_prefix(mid, c0, mi) <= e) lo = mid;
          else hi = mid - 1;
        }
        jj[j] = lo;
        ii[j] = e - sym_prefix(lo, c0, mi);
      } else {
        ii[j] = e % mi;
        jj[j] = e / mi;
      }
      nmy += sl < nslot ? 1 : 0;
    }
    const int grp = tid < nslot ? tid / ne : 0;
    const int wmy = __reduce_max_sync(0xffffffffu, (unsigned)nmy);
    CT acc[4] = {0, 0, 0, 0};
    // stage slice `sl` of A (mi x ks) and B (ks x nj) into buffer `buf` with asynchronous copies
    auto stage = [&](int sl, int buf) {
      double* Asb = gsm + buf * GBUF;
      double* Bsb = Asb + GKS * (GTM + 1);
      const int L0 = sl * GKS, ks = min(GKS, k - L0);
      for (int e = tid; e < mi * ks; e += 256) {
        int i, l;
        if (a_i_fast) {
          i = e % mi;
          l = e / mi;
        } else {
          l = e % ks;
          i = e / ks;
        }
        const int gi = i0 + i, gl = L0 + l;
        const double* src = A + (int64_t)gi * op.a_rs + (int64_t)gl * op.a_cs;
        double* dst = Asb + l * (GTM + 1) + i;
        if (unitlower && gi == gl) *dst = 1.0;
        else cp_async8(dst, src, unitlower ? gi > gl : (upper ? gl >= gi : true));
      }
      for (int e = tid; e < ks * nj; e += 256) {
        int j, l;
        if (b_j_fast) {
          j = e % nj;
          l = e / nj;
        } else {
          l = e % ks;
          j = e / ks;
        }
        cp_async8(Bsb + l * (GTM + 1) + j, Bm + (int64_t)(L0 + l) * op.b_rs + (int64_t)(j0 + j) * op.b_cs, true);
      }
      cp_async_commit();
    };
    int buf = 0;
    if (z0 < nslices) stage(z0, 0);
    for (int sl = z0; sl < nslices; sl += zs) {
      const int ks = min(GKS, k - sl * GKS);
      if (sl + zs < nslices) {
        stage(sl + zs, buf ^ 1);
        cp_async_wait<1>();
      } else {
        cp_async_wait<0>();
      }
      __syncthreads();
      const CT* As;
      const CT* Bs;
      if constexpr (F32) {
        // convert the rows of the slice that are in use: A is mi x ks, B ks x nj (ld GTM + 1)
        const double* src = gsm + buf * GBUF;
        for (int e = tid; e < ks * (mi + nj); e += 256) {
          const int l = e / (mi + nj), c = e % (mi + nj);
          const int off = c < mi ? l * (GTM + 1) + c : GKS * (GTM + 1) + l * (GTM + 1) + (c - mi);
          fsl[off] = f64_to_f32(src[off]);
        }
        __syncthreads();
        As = (const CT*)fsl;
        Bs = (const CT*)(fsl + GKS * (GTM + 1));
      } else {
        As = (const CT*)(gsm + buf * GBUF);
        Bs = As + GKS * (GTM + 1);
      }
      if (G == 1) {
        // the slot count is made warp-uniform so that no DFMA is issued for an empty slot
        // (a predicated-off DFMA still takes its turn on the FP64 pipe); the extra lanes of
        // a warp compute on slot 0's indices into accumulators that are never written
        switch (wmy) {
          case 4: gemm_slice<4>(As, Bs, ks, ii, jj, acc); break;
          case 3: gemm_slice<3>(As, Bs, ks, ii, jj, acc); break;
          case 2: gemm_slice<2>(As, Bs, ks, ii, jj, acc); break;
          case 1: gemm_slice<1>(As, Bs, ks, ii, jj, acc); break;
          default: break;
        }
      } else if (nmy > 0) {
        const int lo = (grp * ks) / G, hi = ((grp + 1) * ks) / G;
        for (int l = lo; l < hi; ++l) acc[0] = fma(As[l * (GTM + 1) + ii[0]], Bs[l * (GTM + 1) + jj[0]], acc[0]);
      }
      __syncthreads();
      buf ^= 1;
    }
    if (G > 1) {
      __syncthreads();
      if (tid < nslot) red[tid] = (double)acc[0];
      __syncthreads();
      if (tid < ne) {
        double t = red[tid];
        for (int g = 1; g < G; ++g) t += red[tid + g * ne];
        acc[0] = (CT)t;
      }
      nmy = tid < ne ? 1 : 0;
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      if (j < nmy) {
        double* c = C + (int64_t)(i0 + ii[j]) * op.c_rs + (int64_t)(j0 + jj[j]) * op.c_cs;
        const double v = op.alpha * (double)acc[j];
        if (atomic) atomicAdd(c, v);
        else if (overwrite) *c = v;
        else *c += v;
      }
    }
  }
  if (threadIdx.x == 0 && blockIdx.y == 0) {
    // a symmetric product computes only the entries i <= j: sum_j min(j + 1, m) of them
    const double entries = sym ? (n <= m ? 0.5 * n * (n + 1.0) : 0.5 * m * (m + 1.0) + (double)(n - m) * m)
                               : (double)m * n;
    const unsigned long long f = (unsigned long long)(2.0 * entries * (double)k);
    if (op.fclass < FC_NONE) atomicAdd(&B.flops[op.fclass], f);
    atomicAdd(&B.flops[NFC + (F32 ? K_GEMM32 : K_GEMM)], f);
  }
}

// ------------------------------------------------------------------------------ TRSM
// Triangular solves / multiplies of a diagonal leaf's packed LU on many vectors. CTA (op, y)
// takes the chunks of 32 vectors y, y + Y, ... of the micro-op (CTAs past nv exit); for a chunk
// of nc vectors, thread t works on vector t % w and rows t / w, t / w + 256 / w, ... with w the
// next power of two >= nc (no index divisions in the sequential steps).
constexpr int TRSM_VC = 32;
__global__ void __launch_bounds__(256) k_trsm(const TrsmOp* __restrict__ ops, Bases B) {
  const TrsmOp op = ops[blockIdx.x];
  const int nv = dimv(B, op.nv, op.nvd), b = op.b;
  if (nv <= (int)blockIdx.y * TRSM_VC || b <= 0) return;
  extern __shared__ double trsm_smem[];   // T[64][65] then X[64][33]
  double(*T)[65] = reinterpret_cast<double(*)[65]>(trsm_smem);
  double(*X)[TRSM_VC + 1] = reinterpret_cast<double(*)[TRSM_VC + 1]>(trsm_smem + 64 * 65);
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
    for (int e = tid; e < b; e += 256) dinv[e] = nr_rcp(T[e][e]);
  const bool e_fast = op.x_es == 1;
  for (int v0 = blockIdx.y * TRSM_VC; v0 < nv; v0 += gridDim.y * TRSM_VC) {
  const int nc = min(TRSM_VC, nv - v0);
  // vector lanes: the next power of two >= nc, the remaining threads spread over the rows
  int vw = 1;
  while (vw < nc) vw *= 2;
  const int v = tid & (vw - 1), g = tid / vw, ng = blockDim.x / vw;
  for (int e = tid; e < b * nc; e += 256) {
    int ee, vv;
    if (e_fast) {
      ee = e % b;
      vv = e / b;
    } else {
      vv = e % nc;
      ee = e / nc;
    }
    X[ee][vv] = Xg[(int64_t)ee * op.x_es + (int64_t)(v0 + vv) * op.x_vs];
  }
  __syncthreads();
  const bool act = v < nc;
  if (op.mode == TM_L_PIV) {
    if (tid < nc)
      for (int i = 0; i < b; ++i) {
        const int p = piv[i];
        if (p != i) {
          const double t = X[i][tid];
          X[i][tid] = X[p][tid];
          X[p][tid] = t;
        }
      }
    __syncthreads();
    for (int j = 0; j < b - 1; ++j) {
      if (act) {
        const double xj = X[j][v];
        for (int i = j + 1 + g; i < b; i += ng) X[i][v] = fma(-T[i][j], xj, X[i][v]);
      }
      __syncthreads();
    }
  } else if (op.mode == TM_UT || op.mode == TM_U) {
    // every thread of vector v scales its own copy of x_j; thread group 0 stores it one step
    // later, after the barrier that ends the step's reads of the unscaled value
    __syncthreads();
    const bool up = op.mode == TM_UT;
    double xprev = 0.0;
    int jprev = -1;
    for (int s = 0; s < b; ++s) {
      const int j = up ? s : b - 1 - s;
      if (act) {
        if (g == 0 && jprev >= 0) X[jprev][v] = xprev;
        const double xj = X[j][v] * dinv[j];
        if (up)
          for (int i = j + 1 + g; i < b; i += ng) X[i][v] = fma(-T[j][i], xj, X[i][v]);
        else
          for (int i = g; i < j; i += ng) X[i][v] = fma(-T[i][j], xj, X[i][v]);
        xprev = xj;
        jprev = j;
      }
      __syncthreads();
    }
    if (act && g == 0 && jprev >= 0) X[jprev][v] = xprev;
  } else {
    // multiplies: each thread keeps its results in registers until all reads are done
    double y[8];   // rows g + q ng, q < 8 (ng >= 8 threads per vector cover b <= 64)
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int i = g + q * ng;
      double sacc = 0.0;
      if (act && i < b) {
        if (op.mode == TM_MUL_U) {
          for (int j = i; j < b; ++j) sacc = fma(T[i][j], X[j][v], sacc);
        } else {
          sacc = X[i][v];
          for (int j = 0; j < i; ++j) sacc = fma(T[i][j], X[j][v], sacc);
        }
      }
      y[q] = sacc;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int i = g + q * ng;
      if (act && i < b) X[i][v] = y[q];
    }
    __syncthreads();
    if (op.mode == TM_MUL_PL && tid < nc)
      for (int i = b - 1; i >= 0; --i) {
        const int p = piv[i];
        if (p != i) {
          const double t = X[i][tid];
          X[i][tid] = X[p][tid];
          X[p][tid] = t;
        }
      }
  }
  __syncthreads();
  for (int e = tid; e < b * nc; e += 256) {
    int ee, vv;
    if (e_fast) {
      ee = e % b;
      vv = e / b;
    } else {
      vv = e % nc;
      ee = e / nc;
    }
    Xg[(int64_t)ee * op.x_es + (int64_t)(v0 + vv) * op.x_vs] = X[ee][vv];
  }
  __syncthreads();
  if (tid == 0) {
    atomicAdd(&B.flops[FC_TRSM], (unsigned long long)nc * b * b);
    atomicAdd(&B.flops[NFC + K_TRSM], (unsigned long long)nc * b * b);
  }
  }
}

// ------------------------------------------------------------------------------ GETRF
// Partial-pivoting pivot of column c (rows r..b-1) of S by warp 0: the first row of largest
// |a| (64-bit compare of the magnitudes' bit patterns, then the lowest row among the maxima),
// and the reciprocal of the pivot (0 for a zero column). A pivot of magnitude <= sing_key (the
// bit pattern of b u max|A_leaf|) is numerically zero and counted as singular (status[0]); a
// row interchange is counted in status[3].
__device__ __forceinline__ void getrf_select(double (*S)[65], int c, int r, int b, int* piv, int* s_p,
                                             double* s_dinv, int slot, int* status, long long sing_key) {
  const int lane = threadIdx.x & 31;
  long long best = -1;
  int bi = b;
  for (int i = r + lane; i < b; i += 32) {
    const long long k = __double_as_longlong(fabs(S[i][c]));
    if (k > best) {
      best = k;
      bi = i;
    }
  }
  long long gmax = best;
  for (int o = 16; o > 0; o >>= 1) {
    const long long ob = __shfl_xor_sync(0xffffffffu, gmax, o);
    gmax = ob > gmax ? ob : gmax;
  }
  const int p = (int)__reduce_min_sync(0xffffffffu, (unsigned)(best == gmax ? bi : b));
  if (lane == 0) {
    const int pp = p < b ? p : r;
    const double v = S[pp][c];
    double dinv = 0.0;
    const long long mag = gmax;                      // bits of |pivot|
    if (mag <= sing_key) atomicAdd(&status[0], 1);
    if (pp != c) atomicAdd(&status[3], 1);
    if (mag > 0) dinv = pivot_rcp(v);
    s_p[slot] = pp;
    s_dinv[slot] = dinv;
    piv[c] = pp;
  }
}

// Dense LU with partial pivoting of a diagonal leaf (b <= 64) in shared memory. Step j: all
// threads interchange rows j and p_j (columns != j) and scale column j by 1 / pivot; then warp 0
// updates column j + 1, picks p_{j+1} and forms its reciprocal while warps 1.. apply the rank-one
// update to columns j + 2.. -- the pivot search of the next step overlaps this step's update.
__global__ void __launch_bounds__(256) k_getrf(const GetrfOp* __restrict__ ops, Bases B) {
  const GetrfOp op = ops[blockIdx.x];
  const int b = op.b;
  if (b <= 0) return;
  __shared__ double S[64][65];
  __shared__ int s_p[2];
  __shared__ double s_dinv[2];
  __shared__ double red[8];
  double* A = dptr(B, op.A);
  int* piv = iptr(B, op.piv);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  double amax = 0.0;
  for (int e = tid; e < b * b; e += 256) {
    const double v = A[e];
    S[e % b][e / b] = v;
    amax = fmax(amax, fabs(v));
  }
  // numerically zero pivot: |p| <= b u max|A_leaf| (u = 2^-53)
  const long long sing_key = __double_as_longlong(block_max(amax, red) * (double)b * 0x1p-53);
  if (warp == 0) getrf_select(S, 0, 0, b, piv, s_p, s_dinv, 0, B.status, sing_key);
  __syncthreads();
  for (int j = 0; j < b; ++j) {
    const int slot = j & 1;
    const int p = s_p[slot];
    const double dinv = s_dinv[slot];
    if (tid < b) {
      const int c = tid;
      if (c != j && p != j) {
        const double t = S[j][c];
        S[j][c] = S[p][c];
        S[p][c] = t;
      }
    } else if (tid >= 64 && tid < 64 + b) {
      const int i = tid - 64;
      if (i == j) {
        const double a = S[j][j], pv = S[p][j];
        S[j][j] = pv;
        if (p != j) S[p][j] = a * dinv;
      } else if (i > j && i != p) {
        S[i][j] *= dinv;
      }
    }
    __syncthreads();
    if (j + 1 < b) {
      if (warp == 0) {
        const double u = S[j][j + 1];
        for (int i = j + 1 + lane; i < b; i += 32) S[i][j + 1] = fma(-S[i][j], u, S[i][j + 1]);
        __syncwarp();
        getrf_select(S, j + 1, j + 1, b, piv, s_p, s_dinv, slot ^ 1, B.status, sing_key);
      } else {
        // dense enumeration of the trailing block (rows j+1.., columns j+2..): full FP64 warp
        // instructions
        const int m = b - 1 - j;
        for (int e = tid - 32; e < m * (m - 1); e += blockDim.x - 32) {
          const int i = j + 1 + e % m, c = j + 2 + e / m;
          S[i][c] = fma(-S[i][j], S[j][c], S[i][c]);
        }
      }
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
  auto put = [&](int i, int j) {
    double* d = dst + (int64_t)i * op.d_rs + (int64_t)j * op.d_cs;
    switch (op.mode) {
      case CM_ZERO: *d = 0.0; break;
      case CM_IDENTITY: *d = (i == j) ? 1.0 : 0.0; break;
      case CM_COPY: *d = op.alpha * src[(int64_t)i * op.s_rs + (int64_t)j * op.s_cs]; break;
      default: *d += op.alpha * src[(int64_t)i * op.s_rs + (int64_t)j * op.s_cs]; break;
    }
  };
  if (tot <= 0x7fffffff) {   // 32-bit index arithmetic (64-bit division is a long software sequence)
    const unsigned t = (unsigned)tot, fm = (unsigned)(i_fast ? m : n);
    for (unsigned e = threadIdx.x; e < t; e += blockDim.x) {
      const unsigned q = e / fm, r = e - q * fm;
      if (i_fast) put((int)r, (int)q);
      else put((int)q, (int)r);
    }
    return;
  }
  for (int64_t e = threadIdx.x; e < tot; e += blockDim.x) {
    int i, j;
    if (i_fast) { i = (int)(e % m); j = (int)(e / m); } else { j = (int)(e % n); i = (int)(e / n); }
    put(i, j);
  }
}

// ------------------------------------------------------------------------------ STACK
__global__ void __launch_bounds__(256) k_stack(const TruncOp* __restrict__ ops,
                                               const StackEntry* __restrict__ ent, Bases B) {
  // CTA (op, y) copies rows [y m / Y, (y + 1) m / Y) of the stacked left factor (Y: its share of
  // the launch's CTAs, from its size) and the same
  // share of the right factor's rows; every CTA derives the column layout itself, CTA y = 0 also
  // publishes the stacked rank and clears the Gram matrices.
  const TruncOp op = ops[blockIdx.x];
  const int m = op.m, n = op.n, Kc = op.Kcap, tid = threadIdx.x;
  // this rounded addition's share of the launch's CTAs along the rows: ~16k copied doubles each
  // (the launch is sized for its largest one; the others leave the surplus CTAs at once)
  const int ny = (int)min((int64_t)gridDim.y, max((int64_t)1, (int64_t)(m + n) * Kc / 16384));
  if ((int)blockIdx.y >= ny) return;
  const int kself = (op.flags & TF_NOSELF) ? 0 : *iptr(B, op.rank);
  const int ne = min(op.n_entries, KMAX_ENTRIES);
  __shared__ int s_ke[KMAX_ENTRIES], s_col[KMAX_ENTRIES], s_K;
  for (int e = tid; e < ne; e += blockDim.x) {
    const StackEntry& se = ent[op.first_entry + e];
    s_ke[e] = max(dimv(B, se.k, se.kd), 0);
  }
  __syncthreads();
  if (tid == 0) {
    int K = kself;
    for (int e = 0; e < ne; ++e) K += s_ke[e];
    if (K > Kc) K = Kc;   // the planner sizes Kcap from static maxima; never taken
    int col = min(kself, K);
    for (int e = 0; e < ne; ++e) {
      const int ke = max(0, min(s_ke[e], K - col));
      s_col[e] = col;
      s_ke[e] = ke;
      col += ke;
    }
    s_K = K;
    if (blockIdx.y == 0) *iptr(B, op.Kd) = K;
  }
  __syncthreads();
  const int K = s_K;
  double* Wst = dptr(B, op.Wst);
  double* Zst = dptr(B, op.Zst);
  if (blockIdx.y == 0) {
    double* Gw = dptr(B, op.Gw);
    double* Gz = dptr(B, op.Gz);
    for (int e = tid; e < K * K; e += blockDim.x) {
      const int i = e % K, j = e / K;
      Gw[i + (int64_t)j * Kc] = 0.0;
      Gz[i + (int64_t)j * Kc] = 0.0;
    }
  }
  const int y = blockIdx.y;
  const int w0 = (int)((int64_t)m * y / ny), wl = (int)((int64_t)m * (y + 1) / ny) - w0;
  const int z0 = (int)((int64_t)n * y / ny), zl = (int)((int64_t)n * (y + 1) / ny) - z0;
  const double* U = dptr(B, op.U);
  const double* V = dptr(B, op.V);
  const int cself = min(kself, K);
  if (wl > 0)
    for (int e = tid; e < wl * cself; e += blockDim.x) {
      const int i = w0 + e % wl, c = e / wl;
      Wst[(int64_t)c * m + i] = U[(int64_t)c * m + i];
    }
  if (zl > 0)
    for (int e = tid; e < zl * cself; e += blockDim.x) {
      const int j = z0 + e % zl, c = e / zl;
      Zst[(int64_t)c * n + j] = V[(int64_t)c * n + j];
    }
  for (int q = 0; q < ne; ++q) {
    const int ke = s_ke[q], col = s_col[q];
    if (ke <= 0) continue;
    const StackEntry se = ent[op.first_entry + q];
    const double* W = dptr(B, se.W);
    const double* Z = dptr(B, se.Z);
    if (wl > 0)
      for (int e = tid; e < wl * ke; e += blockDim.x) {
        const int i = w0 + e % wl, c = e / wl;
        double v = 0.0;
        if (i >= se.row_off && i < se.row_off + se.nrows)
          v = se.alpha * W[(int64_t)(i - se.row_off) * se.w_rs + (int64_t)c * se.w_cs];
        Wst[(int64_t)(col + c) * m + i] = v;
      }
    if (zl > 0)
      for (int e = tid; e < zl * ke; e += blockDim.x) {
        const int j = z0 + e % zl, c = e / zl;
        double v = 0.0;
        if (j >= se.col_off && j < se.col_off + se.ncols)
          v = Z[(int64_t)(j - se.col_off) * se.z_rs + (int64_t)c * se.z_cs];
        Zst[(int64_t)(col + c) * n + j] = v;
      }
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

#ifdef HM_CORE_TIMING
__device__ long long g_core_stamp[24];
__device__ int g_jac_maxcos[8];
__device__ float g_core_gf[64 * 64];
#define CORE_STAMP(i)                                  \
  do {                                                 \
    __syncthreads();                                   \
    if (threadIdx.x == 0) g_core_stamp[i] = clock64(); \
  } while (0)
#else
#define CORE_STAMP(i) \
  do {                \
  } while (0)
#endif

constexpr int KMAX = 256;       // largest stacked rank of one rounded addition
constexpr int JSM = 64;         // Jacobi problems up to this size run in shared memory

// Pivoted Cholesky (outer-product form, diagonal pivoting) of the symmetric positive
// semi-definite n x n matrix A (n <= 256, ld lda), with logical pivoting: A keeps its index
// order and every symmetric entry {i, k} lives at its lower position (max, min); nothing is
// interchanged. On return perm is the full pivot order (the rank pivots, then the remaining
// indices), rs[q] = 1/sqrt(pivot q) for q < rank, and the factor of P^T A P = L L^T is
// L(l, q) = a(perm[l], perm[q]) rs[q] for l >= q (chol_entry below). Stops when the largest
// remaining diagonal entry is <= tol (tol >= 0); returns the rank. The pivots must lie in
// [1e-30, 1e30] (callers scale A to unit diagonal or unit trace).
// Step j (pivot p, trailing index list of n - 1 - j entries): warps 1.. update the trailing
// pairs, a_ik -= a_ip (a_kp / a_pp), one list position per warp for k and lanes over i, while
// warp 0 updates its copy dg of the trailing diagonal with the same operations (bitwise the same
// values), picks the next pivot (warp max over 32-bit keys of the bit patterns), forms its
// reciprocal and writes the next list (this one without the new pivot) into the other buffer.
// One block barrier per step. dg, rs: n doubles; ul: 2 n ints; s_flag, s_pidx: 2 ints;
// s_val: 2 doubles (shared scratch; the 2-slot ones are double-buffered broadcast slots).
__device__ __forceinline__ int64_t chol_at(int i, int k, int lda) {
  return i >= k ? i + (int64_t)k * lda : k + (int64_t)i * lda;
}
__device__ __forceinline__ double chol_entry(const double* A, int lda, const int* perm, const double* rs, int l,
                                             int q) {
  return A[chol_at(perm[l], perm[q], lda)] * rs[q];
}

__device__ int pivoted_cholesky(double* A, int lda, int n, int* perm, double tol, double* dg, double* rs,
                                int* ul, int* s_flag, double* s_val, int* s_pidx) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  const long long tol_bits = __double_as_longlong(fmax(tol, 0.0));
  if (warp == 0) {
    for (int i = lane; i < n; i += 32) dg[i] = A[i + (int64_t)i * lda];
    __syncwarp();
    unsigned best = 0;
    for (int i = lane; i < n; i += 32) best = max(best, pivot_key(dg[i], i));
    best = __reduce_max_sync(0xffffffffu, best);
    const int p = best ? 255 - (int)(best & 255u) : -1;
    const bool go = p >= 0 && __double_as_longlong(dg[p]) > tol_bits;
    if (go)
      for (int r = lane; r < n - 1; r += 32) ul[r] = r < p ? r : r + 1;
    if (lane == 0) {
      s_flag[0] = go ? 1 : 0;
      s_pidx[0] = p;
      if (go) {
        s_val[0] = fast_rcp(dg[p]);
        perm[0] = p;
      }
    }
  }
  __syncthreads();
  int j = 0;
  for (; j < n; ++j) {
    const int slot = j & 1;
    if (!s_flag[slot]) break;
    const int p = s_pidx[slot];
    const double ipiv = s_val[slot];
    const int m = n - 1 - j;
    const int* cur = ul + slot * n;
    if (warp == 0) {
      for (int r = lane; r < m; r += 32) {
        const int i = cur[r];
        const double a = A[chol_at(i, p, lda)];
        dg[i] = fma(-a, a * ipiv, dg[i]);
      }
      __syncwarp();
      unsigned best = 0;
      for (int r = lane; r < m; r += 32) {
        const int i = cur[r];
        best = max(best, pivot_key(dg[i], i));
      }
      best = __reduce_max_sync(0xffffffffu, best);
      const int q = best ? 255 - (int)(best & 255u) : -1;
      const bool go = q >= 0 && __double_as_longlong(dg[q]) > tol_bits;
      if (go) {
        int pos = m;
        for (int r = lane; r < m; r += 32)
          if (cur[r] == q) pos = r;
        pos = (int)__reduce_min_sync(0xffffffffu, (unsigned)pos);
        int* nxt = ul + (slot ^ 1) * n;
        for (int r = lane; r < m - 1; r += 32) nxt[r] = cur[r < pos ? r : r + 1];
      }
      if (lane == 0) {
        s_flag[slot ^ 1] = go ? 1 : 0;
        s_pidx[slot ^ 1] = q;
        if (go) {
          s_val[slot ^ 1] = fast_rcp(dg[q]);
          perm[j + 1] = q;
        }
      }
    } else {
      for (int c = warp - 1; c < m; c += nw - 1) {
        const int kk = cur[c];
        const double t = A[chol_at(kk, p, lda)] * ipiv;
        for (int r = c + lane; r < m; r += 32) {
          const int ii = cur[r];
          double* x = A + chol_at(ii, kk, lda);
          *x = fma(-A[chol_at(ii, p, lda)], t, *x);
        }
      }
    }
    __syncthreads();
  }
  // the remaining indices complete the permutation; reciprocal square roots of the pivots
  if (j < n) {
    const int* rest = j >= 1 ? ul + ((j - 1) & 1) * n : nullptr;
    for (int r = tid; r < n - j; r += blockDim.x) perm[j + r] = rest ? rest[r] : r;
  }
  for (int q = tid; q < j; q += blockDim.x) {
    const int pq = perm[q];
    rs[q] = nr_rsqrt(A[pq + (int64_t)pq * lda]);
  }
  __syncthreads();
  return j;
}

// One-sided (Hestenes) Jacobi in FP32 on the columns of G (rows x cols, cols even, ld ldg):
// column pairs are rotated until orthogonal, and the rotations are accumulated into V (cols x
// cols, ld ldv) when V is given; "orthogonal" means |g_a . g_b| below the FP32 rounding level
// of the dot products. Applied to a Cholesky factor of a graded positive definite matrix it
// yields singular values with high relative accuracy (Demmel and Veselic, "Jacobi's method is
// more accurate than QR", 1992). Round-robin pairing; one half-warp (16 lanes) handles one pair
// of a round, so a block of 512 threads runs all pairs of a round concurrently for cols <= 64,
// and a round costs one block barrier.
// Rotation (c, s) of the one-sided Jacobi that orthogonalises two columns with squared norms al,
// be and dot product g: tan 2 theta = 2 g / (al - be), and t = tan theta is the smaller root,
// t = 2 g sgn(d) / (|d| + sqrt(d^2 + 4 g^2)) with d = be - al (the usual choice, written without
// the quotient zeta = d / (2 g)). d and g are first scaled by the power of two that brings
// max(al, be) into [1, 2) (exact), so d^2 + 4 g^2 stays in range; the chain has three dependent
// special-function operations (square root, reciprocal, reciprocal square root).
__device__ __forceinline__ void jacobi_cs(float al, float be, float g, float& c, float& s) {
  const float mx = fmaxf(al, be);
  const int ex = ((__float_as_int(mx) >> 23) & 0xff) - 127;
  const float sc = __int_as_float((127 - ex) << 23);
  const float d = (be - al) * sc, gg = g * sc;
  const float den = fabsf(d) + sqrtf(fmaf(d, d, 4.0f * gg * gg));
  float t = den > 0.f ? __fdividef(2.0f * gg, den) : 0.f;
  t = d < 0.f ? -t : t;
  c = rsqrtf(fmaf(t, t, 1.0f));
  s = t * c;
}

// NR: entries per lane of a column (rows <= 16 NR). A lane keeps its entries of the pair's two
// columns in registers from the dot products to the rotation: one load pass per round, and no
// store waits for a later load (the arithmetic is that of a load-compute-store pass).
template <int NR>
__device__ void onesided_jacobi_f32_t(float* G, int ldg, int rows, int cols, float* V, int ldv, int* flag,
                                      int max_sweeps) {
  const int hl = threadIdx.x & 15, hw = threadIdx.x >> 4, nh = blockDim.x >> 4;
  const unsigned hmask = 0xffffu << (threadIdx.x & 16);
  const int half = cols / 2;
  // orthogonality target at the FP32 rounding level of dot products of length `rows`
  const float tol = fmaxf(1e-6f, 6e-8f * (float)rows);
  // Jacobi converges quadratically here: a sweep whose largest |cos| stays below sqrt(tol)
  // leaves the next one below tol, so it ends the iteration (rotations still applied)
  const float tol_next = sqrtf(tol);
  int sweep = 0;
  for (; sweep < max_sweeps; ++sweep) {
    if (threadIdx.x == 0) *flag = 0;
    __syncthreads();
    for (int r = 0; r < cols - 1; ++r) {
      for (int q = hw; q < half; q += nh) {
        // round-robin pairing: position 0 fixed, positions 1..cols-1 rotate by r
        int x = q - 1 + r, y = cols - 2 - q + r;
        x = x >= cols - 1 ? x - (cols - 1) : x;
        y = y >= cols - 1 ? y - (cols - 1) : y;
        x = q == 0 ? 0 : 1 + x;
        y = 1 + y;
        const int a = min(x, y), b = max(x, y);
        float* ga = G + a * ldg;
        float* gb = G + b * ldg;
        float u[NR], v[NR];
#pragma unroll
        for (int k = 0; k < NR; ++k) {
          const int l = hl + 16 * k;
          u[k] = l < rows ? ga[l] : 0.f;
          v[k] = l < rows ? gb[l] : 0.f;
        }
        float al = 0.f, be = 0.f, ga_b = 0.f;
#pragma unroll
        for (int k = 0; k < NR; ++k) {
          al = fmaf(u[k], u[k], al);
          be = fmaf(v[k], v[k], be);
          ga_b = fmaf(u[k], v[k], ga_b);
        }
        for (int o = 8; o > 0; o >>= 1) {
          al += __shfl_xor_sync(hmask, al, o);
          be += __shfl_xor_sync(hmask, be, o);
          ga_b += __shfl_xor_sync(hmask, ga_b, o);
        }
        // gn = cos of the pair's angle (the convergence test; the rotation uses al, be, ga_b)
        const float rab = (al > 0.f && be > 0.f) ? rsqrtf(al) * rsqrtf(be) : 0.f;
        const float gn = ga_b * rab;
#ifdef HM_CORE_TIMING
        if (hl == 0 && sweep < 8) atomicMax(&g_jac_maxcos[sweep], __float_as_int(fabsf(gn)));
#endif
        if (fabsf(gn) > tol) {
          float c, s;
          jacobi_cs(al, be, ga_b, c, s);
          if (s != 0.f) {
#pragma unroll
            for (int k = 0; k < NR; ++k) {
              const int l = hl + 16 * k;
              if (l < rows) {
                ga[l] = c * u[k] - s * v[k];
                gb[l] = s * u[k] + c * v[k];
              }
            }
            if (V) {
              float* va = V + a * ldv;
              float* vb = V + b * ldv;
              for (int l = hl; l < cols; l += 16) {
                const float p0 = va[l], p1 = vb[l];
                va[l] = c * p0 - s * p1;
                vb[l] = s * p0 + c * p1;
              }
            }
            if (hl == 0 && fabsf(gn) > tol_next) *flag = 1;
          }
        }
      }
      __syncthreads();
    }
    if (*flag == 0) break;
    __syncthreads();
  }
#ifdef HM_CORE_TIMING
  if (threadIdx.x == 0) g_core_stamp[15] = sweep;
#endif
}

// NR = 0: columns of any length, loaded again for the rotation (no register copy)
template <>
__device__ void onesided_jacobi_f32_t<0>(float* G, int ldg, int rows, int cols, float* V, int ldv, int* flag,
                                         int max_sweeps) {
  const int hl = threadIdx.x & 15, hw = threadIdx.x >> 4, nh = blockDim.x >> 4;
  const unsigned hmask = 0xffffu << (threadIdx.x & 16);
  const int half = cols / 2;
  const float tol = fmaxf(1e-6f, 6e-8f * (float)rows);
  const float tol_next = sqrtf(tol);
  int sweep = 0;
  for (; sweep < max_sweeps; ++sweep) {
    if (threadIdx.x == 0) *flag = 0;
    __syncthreads();
    for (int r = 0; r < cols - 1; ++r) {
      for (int q = hw; q < half; q += nh) {
        int x = q - 1 + r, y = cols - 2 - q + r;
        x = x >= cols - 1 ? x - (cols - 1) : x;
        y = y >= cols - 1 ? y - (cols - 1) : y;
        x = q == 0 ? 0 : 1 + x;
        y = 1 + y;
        const int a = min(x, y), b = max(x, y);
        float* ga = G + a * ldg;
        float* gb = G + b * ldg;
        float al = 0.f, be = 0.f, ga_b = 0.f;
        for (int l = hl; l < rows; l += 16) {
          const float u = ga[l], v = gb[l];
          al = fmaf(u, u, al);
          be = fmaf(v, v, be);
          ga_b = fmaf(u, v, ga_b);
        }
        for (int o = 8; o > 0; o >>= 1) {
          al += __shfl_xor_sync(hmask, al, o);
          be += __shfl_xor_sync(hmask, be, o);
          ga_b += __shfl_xor_sync(hmask, ga_b, o);
        }
        const float rab = (al > 0.f && be > 0.f) ? rsqrtf(al) * rsqrtf(be) : 0.f;
        const float gn = ga_b * rab;
        if (fabsf(gn) > tol) {
          float c, s;
          jacobi_cs(al, be, ga_b, c, s);
          if (s != 0.f) {
            for (int l = hl; l < rows; l += 16) {
              const float u = ga[l], v = gb[l];
              ga[l] = c * u - s * v;
              gb[l] = s * u + c * v;
            }
            if (V) {
              float* va = V + a * ldv;
              float* vb = V + b * ldv;
              for (int l = hl; l < cols; l += 16) {
                const float p0 = va[l], p1 = vb[l];
                va[l] = c * p0 - s * p1;
                vb[l] = s * p0 + c * p1;
              }
            }
            if (hl == 0 && fabsf(gn) > tol_next) *flag = 1;
          }
        }
      }
      __syncthreads();
    }
    if (*flag == 0) break;
    __syncthreads();
  }
#ifdef HM_CORE_TIMING
  if (threadIdx.x == 0) g_core_stamp[15] = sweep;
#endif
}

__device__ void onesided_jacobi_f32(float* G, int ldg, int rows, int cols, float* V, int ldv, int* flag,
                                    int max_sweeps) {
  if (rows <= 64) onesided_jacobi_f32_t<4>(G, ldg, rows, cols, V, ldv, flag, max_sweeps);
  else onesided_jacobi_f32_t<0>(G, ldg, rows, cols, V, ldv, flag, max_sweeps);
}

// Back substitution Rf11 x = y for the NQ columns y_c (c = warp + nw q) of Y owned by one warp,
// in lockstep (see k_core step 7); Rf11(p, l) = R[l + p * Kc], rdinv[l] = 1 / Rf11(l, l).
template <int NQ>
__device__ __forceinline__ void backsub_warp(double* Y, int ldy, const double* R, int Kc, const double* rdinv, int r,
                                             int warp, int nw) {
  const int lane = threadIdx.x & 31;
  for (int l = r - 1; l >= 0; --l) {
    const double rd = rdinv[l];
    double x[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) x[q] = Y[l + (int64_t)(warp + nw * q) * ldy] * rd;
    for (int p = lane; p < l; p += 32) {
      const double rr = R[l + (int64_t)p * Kc];
#pragma unroll
      for (int q = 0; q < NQ; ++q) {
        double* y = Y + p + (int64_t)(warp + nw * q) * ldy;
        *y = fma(-rr, x[q], *y);
      }
    }
    __syncwarp();
    if (lane == 0)
#pragma unroll
      for (int q = 0; q < NQ; ++q) Y[l + (int64_t)(warp + nw * q) * ldy] = x[q];
    __syncwarp();
  }
}

// Rounded truncation core, one rounded addition per CTA (§2.3: the sum of low-rank updates of a
// leaf truncated to precision eps, at most the rank cap). From the Gram matrices G_W = W^T W and
// G_Z = Z^T Z of the stacked factors W = [U, a_1 W_1, ...], Z = [V, Z_1, ...] (upper triangles,
// formed by k_gemm) it computes the coefficient matrices of the truncated U = W T_W, V = Z T_Z
// (rebuilt by k_gemm):
//   1. equilibrate G_W; pivoted Cholesky G' = Pi Rf^T Rf Pi^T (tolerance 4 K u);
//   2-4. Bm = D Pi Rf^T and M = Bm^T G_Z Bm (triangular products);
//   5. eigen-decomposition of M: pivoted Cholesky of M / tr(M) and FP32 one-sided Jacobi on the
//      factor's transpose (rank <= 128), else FP64 two-sided Jacobi on M;
//   6. keep sigma_i = sqrt(lam_i) > eps sigma_1 (at most the cap); FP64 orthogonalisation of the
//      kept vectors in order of decreasing eigenvalue;
//   7. T_Z = Bm X_k S^{-1/2}, T_W = D^-1 Pi Rf11^-1 X_k S^{1/2} (back substitution).
// V = Z T_Z has orthonormal columns; U = W T_W carries the singular values.
__global__ void __launch_bounds__(512) k_core(const TruncOp* __restrict__ ops, const StackEntry* __restrict__ ent,
                                              Bases B) {
  const TruncOp op = ops[blockIdx.x];
  extern __shared__ double smem[];            // 2 * JSM * (JSM + 1) doubles
  __shared__ double d[KMAX], dinv[KMAX], rdinv[KMAX], lam[KMAX], cs[KMAX / 2], sn[KMAX / 2], red[32];
  __shared__ int perm[KMAX], perm2[KMAX], pa[KMAX / 2], pb[KMAX / 2], order[KMAX], s_int[4], ul[2 * KMAX];
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
  // the Gram GEMMs wrote the upper triangles only
  for (int e = tid; e < K * K; e += nt) {
    const int i = e % K, j = e / K;
    if (i > j) {
      Gw[i + (int64_t)j * Kc] = Gw[j + (int64_t)i * Kc];
      Gz[i + (int64_t)j * Kc] = Gz[j + (int64_t)i * Kc];
    }
  }
  __syncthreads();
  double* R = Gw;                              // K x K (ld Kc): the Cholesky factor of the equilibrated G_W
  double* Bm = work;                           // K x r
  double* T1 = work + (int64_t)Kc * Kc;        // K x r, later a temporary
  CORE_STAMP(0);
  // 1. equilibrate the Gram matrix of the stacked left factor: G' = D^-1 G_W D^-1
  for (int i = tid; i < K; i += nt) {
    const double g = Gw[i + (int64_t)i * Kc];
    const double gi = g > 0.0 ? nr_rsqrt(g) : 1.0;
    d[i] = g > 0.0 ? g * gi : 1.0;
    dinv[i] = gi;
    perm[i] = i;
  }
  __syncthreads();
  double* Rc = R;                              // factorise in shared memory when K fits
  int ldr = Kc;
  if (K <= JSM) {
    Rc = smem;
    ldr = JSM + 1;
  }
  for (int e = tid; e < K * K; e += nt) {
    int i = e % K, j = e / K;
    Rc[i + (int64_t)j * ldr] = R[i + (int64_t)j * Kc] * (dinv[i] * dinv[j]);
  }
  __syncthreads();
  CORE_STAMP(1);
  // 2. pivoted Cholesky G' = Pi Rf^T Rf Pi^T; the tolerance is the noise level of a Gram
  //    matrix. Rf is stored transposed in pivoted order: Rf(q, l) = R[l + q * Kc] for l >= q.
  const int r = pivoted_cholesky(Rc, ldr, K, perm, 4.0 * K * 2.2e-16, lam, rdinv, ul, &s_int[2], &red[2], pa);
  // the factor in pivoted layout, R[l + q * Kc] = Rf(q, l) for l >= q (q < r), zero elsewhere;
  // when Rc is R itself (K > JSM) it is gathered into T1 and copied back
  {
    double* Lp = Rc != R ? R : T1;
    for (int e = tid; e < K * K; e += nt) {
      const int l = e % K, q = e / K;
      Lp[l + (int64_t)q * Kc] = (q < r && l >= q) ? chol_entry(Rc, ldr, perm, rdinv, l, q) : 0.0;
    }
    __syncthreads();
    if (Lp == T1) {
      for (int e = tid; e < K * K; e += nt) {
        const int l = e % K, q = e / K;
        R[l + (int64_t)q * Kc] = T1[l + (int64_t)q * Kc];
      }
      __syncthreads();
    }
  }
  if (r == 0) {
    if (tid == 0) *rk = 0;
    return;
  }
  CORE_STAMP(2);
  // 3. Bm = D Pi Rf^T (K x r), kept with its rows in pivoted order: Bm(l, q) = d[perm[l]] Rf(q, l)
  //    for l >= q and zero above, so that the products below skip the zero triangle
  for (int e = tid; e < K * r; e += nt) {
    const int l = e % K, q = e / K;
    Bm[l + (int64_t)q * Kc] = l >= q ? d[perm[l]] * R[l + (int64_t)q * Kc] : 0.0;
  }
  __syncthreads();
  // 4. M = Bm^T G_Z Bm (r x r): the Gram matrix of Z D Pi Rf^T, whose eigen-decomposition gives
  //    the singular values (squared) and right factors of W Z^T. T1 = G_Z Pi Bm with rows in
  //    the original order: T1(i, q) = sum_{l >= q} G_Z(i, perm[l]) Bm(l, q).
  for (int e = tid; e < K * r; e += nt) {
    const int i = e % K, q = e / K;
    double sm4 = 0.0;
    for (int l = q; l < K; ++l) sm4 = fma(Gz[i + (int64_t)perm[l] * Kc], Bm[l + (int64_t)q * Kc], sm4);
    T1[i + (int64_t)q * Kc] = sm4;
  }
  __syncthreads();
  const int rp = r + (r & 1);                  // even size (Jacobi pairs), zero padding
  double* Mj;
  double* Yj;
  int ldj;
  if (rp <= JSM) {
    Mj = smem;
    Yj = smem + JSM * (JSM + 1);
    ldj = JSM + 1;
  } else {
    Mj = Gz;       // Gz is dead once T1 = G_Z Bm is formed
    Yj = T1;       // reused after M is formed (the global path keeps M in Gz)
    ldj = Kc;
  }
  // M(p, q) = sum_{l >= p} Bm(l, p) T1(perm[l], q) for p <= q, mirrored (zero padding at rp > r)
  for (int e = tid; e < rp * rp; e += nt) {
    const int p = e % rp, q = e / rp;
    if (p > q) continue;
    double sm4 = 0.0;
    if (q < r)
      for (int l = p; l < K; ++l) sm4 = fma(Bm[l + (int64_t)p * Kc], T1[perm[l] + (int64_t)q * Kc], sm4);
    Mj[p + (int64_t)q * ldj] = sm4;
    Mj[q + (int64_t)p * ldj] = sm4;
  }
  __syncthreads();
  if (tid < 32) {
    double tr = 0.0;
    for (int q = tid; q < r; q += 32) tr += fabs(Mj[q + (int64_t)q * ldj]);
    for (int o = 16; o > 0; o >>= 1) tr += __shfl_xor_sync(0xffffffffu, tr, o);
    if (tid == 0) red[1] = tr;
  }
  __syncthreads();
  const double tr = red[1];
  CORE_STAMP(3);
  // 5. eigen-decomposition M = X diag(lam) X^T
  // Drmac-Veselic path (FP32 vectors) up to rp = 2 JSM: M and X in shared memory for rp <= JSM,
  // in global scratch (Gz, T1) above, where the FP32 matrix takes all of the dynamic smem
  const bool dv = rp <= 2 * JSM && tr > 0.0;
  if (dv) {
    // (a) FP64 pivoted Cholesky M / tr = P R2^T R2 P^T (in place in Mj);
    // (b) FP32 one-sided Jacobi on the columns of R2^T (below), whose column norms squared give
    //     the eigenvalues lam_i / tr with high relative accuracy, so FP32 resolves the graded
    //     spectrum down to the rank threshold, and whose normalised columns give X;
    // (c) after the rank is chosen, the kept columns are made orthonormal in FP64 (step 6b).
    const double itr = nr_rcp(tr);
    for (int e = tid; e < rp * rp; e += nt) {
      const int p = e % rp, q = e / rp;
      Mj[p + q * ldj] *= itr;                          // unit trace for the factorisation
    }
    for (int i = tid; i < rp; i += nt) perm2[i] = i;
    __syncthreads();
    // the tolerance is one rounding unit of the trace: the Schur complement left behind perturbs
    // the eigenvalues by at most rp u tr, the rounding level of M itself
    const int rc = pivoted_cholesky(Mj, ldj, rp, perm2, 2.2e-16, lam, rdinv, ul, &s_int[2], &red[2], pa);
    // Drmac-Veselic preconditioning: one-sided Jacobi on the columns of C = R2^T (the rows of the
    // pivoted Cholesky factor are graded and nearly orthogonal, so it converges in a few
    // sweeps): C Q = [s_1 u_1, ...] with C C^T = R2^T R2 = P^T M P, i.e. the columns of C Q are
    // the eigenvectors of P^T M P scaled by sqrt(eigenvalue); Q itself is not needed.
    const int rcp = rc + (rc & 1);
    // rp x rcp floats: in the X region for rp <= JSM, else the whole dynamic smem (ld 2 JSM + 1)
    float* Gf = rp <= JSM ? reinterpret_cast<float*>(Yj) : reinterpret_cast<float*>(smem);
    const int ldf = rp <= JSM ? JSM + 1 : 2 * JSM + 1;
    for (int e = tid; e < rp * rcp; e += nt) {
      const int l = e % rp, q = e / rp;    // row l = pivoted position, column q = row q of R2
      float v = 0.0f;
      if (q < rc && l >= q) v = (float)chol_entry(Mj, ldj, perm2, rdinv, l, q);
      Gf[l + q * ldf] = v;
    }
    __syncthreads();
    CORE_STAMP(8);
#ifdef HM_CORE_TIMING
    if (blockIdx.x == 0 && rp * rcp <= 64 * 64) {
      for (int e = tid; e < rp * rcp; e += nt) g_core_gf[e] = Gf[(e % rp) + (e / rp) * ldf];
      if (tid == 0) { g_core_stamp[13] = rp; g_core_stamp[14] = rcp; }
    }
    __syncthreads();
    CORE_STAMP(8);
#endif
    onesided_jacobi_f32(Gf, ldf, rp, rcp, nullptr, 0, &s_int[1], 15);
    CORE_STAMP(9);
    for (int q = tid; q < rp; q += nt) {
      float s2 = 0.0f;
      if (q < rc)
        for (int l = 0; l < rp; ++l) s2 = fmaf(Gf[l + q * ldf], Gf[l + q * ldf], s2);
      lam[q] = (double)s2 * tr;
      rdinv[q] = s2 > 0.0f ? (double)rsqrtf(s2) : 0.0;   // 1 / |column| (FP32 accuracy suffices:
                                                         // step 6b fixes the norms)
    }
    __syncthreads();
    // X[perm2[l]][q] = C Q[l][q] / |column q|, staged through T1 (global) when X overwrites Gf
    for (int e = tid; e < rp * rp; e += nt) {
      const int l = e % rp, q = e / rp;
      T1[perm2[l] + (int64_t)q * Kc] = q < rc ? (double)Gf[l + q * ldf] * rdinv[q] : 0.0;
    }
    __syncthreads();
    if (Yj != T1) {
      for (int e = tid; e < rp * rp; e += nt) {
        const int p = e % rp, q = e / rp;
        Yj[p + q * ldj] = T1[p + (int64_t)q * Kc];
      }
      __syncthreads();
    }
  } else {
    for (int e = tid; e < rp * rp; e += nt) {
      int p = e % rp, q = e / rp;
      Yj[p + (int64_t)q * ldj] = (p == q) ? 1.0 : 0.0;
    }
    __syncthreads();
    jacobi_eigen<double>(Mj, ldj, Yj, ldj, rp, cs, sn, pa, pb, &s_int[1], K * 2.2e-16 * tr, 40);
    __syncthreads();
    for (int q = tid; q < rp; q += nt) lam[q] = Mj[q + (int64_t)q * ldj];
  }
  __syncthreads();
  CORE_STAMP(5);
  // 6. order the eigenvalues (descending, ties by index) and choose the rank; the order
  //    array is first the identity so that it stays a valid index list even with NaNs
  for (int q = tid; q < rp; q += nt) order[q] = q;
  __syncthreads();
  for (int q = tid; q < rp; q += nt) {
    int pos = 0;
    const long long v = order_key(lam[q]);
    for (int p = 0; p < rp; ++p) {
      const long long w = order_key(lam[p]);
      if (w > v || (w == v && p < q)) ++pos;
    }
    order[pos] = q;
  }
  __syncthreads();
  const double smax = lam[order[0]];
  const long long thr = order_key(op.eps * op.eps * smax);
  int kk = __syncthreads_count(smax > 0.0 && tid < r && order_key(lam[order[tid]]) > thr);
  if (kk > op.cap) {
    if (tid == 0) atomicAdd(&B.status[1], 1);
    kk = op.cap;
  }
  if (dv && kk > 0) {
    // 6b. ordered orthogonalisation of the kept FP32 vectors X_k = X[:, order[0..kk)] in FP64:
    //     with F = X_k^T X_k - I, X_k <- X_k (I - U1), U1 = strict upper part of F + diag(F)/2,
    //     the first-order term of Cholesky QR, so that column c mixes only with columns of
    //     larger eigenvalue and never takes in a discarded direction (a symmetric
    //     orthogonalisation would leak the FP32 non-orthogonality of the small vectors into the
    //     large ones, ~1e-6 sigma_1). The remaining non-orthogonality is O(F^2) ~ 1e-11, below
    //     the Gram approach's own error. F goes to shared memory (the Cholesky factor of M or
    //     the FP32 matrix are dead here), X_k U1 to T1 or, when X itself lives in T1, to Gz.
    double* Fm = rp <= JSM ? Mj : smem;
    const int ldm = JSM + 1;
    double* Tp = Yj != T1 ? T1 : Gz;
    for (int e = tid; e < kk * kk; e += nt) {
      const int a = e % kk, b = e / kk;
      double sf = 0.0;
      if (a <= b) {
        const double* xa = Yj + (int64_t)order[a] * ldj;
        const double* xb = Yj + (int64_t)order[b] * ldj;
        for (int l = 0; l < rp; ++l) sf = fma(xa[l], xb[l], sf);
        if (a == b) sf = 0.5 * (sf - 1.0);
      }
      Fm[a + b * ldm] = sf;
    }
    __syncthreads();
    for (int e = tid; e < rp * kk; e += nt) {
      const int l = e % rp, c = e / rp;
      double sf = 0.0;
      for (int a = 0; a <= c; ++a) sf = fma(Yj[l + (int64_t)order[a] * ldj], Fm[a + c * ldm], sf);
      Tp[l + (int64_t)c * Kc] = sf;
    }
    __syncthreads();
    for (int e = tid; e < rp * kk; e += nt) {
      const int l = e % rp, c = e / rp;
      Yj[l + (int64_t)order[c] * ldj] -= Tp[l + (int64_t)c * Kc];
    }
    __syncthreads();
  }
  CORE_STAMP(6);
  // 7. coefficient matrices: Tz = Bm X_k S_k^{-1/2}, Tw = D^{-1} Pi_r Rf11^{-1} X_k S_k^{1/2}
  double* Tw = dptr(B, op.Tw);
  double* Tz = dptr(B, op.Tz);
  // r x kk scratch for the back substitution: shared memory when X lives there (the first half
  // of the dynamic smem is dead by now), else Gz
  const bool ysm = dv && rp <= JSM;
  double* Y = ysm ? smem : Gz;
  const int ldy = ysm ? JSM + 1 : Kc;
  if (tid < kk) {
    const double l = lam[order[tid]];
    const double is = nr_rsqrt(l);
    cs[tid] = l * is;      // sigma of the c-th kept direction
    sn[tid] = is;          // 1 / sigma
  }
  for (int l = tid; l < r; l += nt) rdinv[l] = nr_rcp(R[l + (int64_t)l * Kc]);
  __syncthreads();
  CORE_STAMP(16);
  for (int e = tid; e < K * kk; e += nt) {
    const int l = e % K, c = e / K;     // l: pivoted row of Bm
    const int q = order[c];
    double sz = 0.0;
    const int pe = min(l, r - 1);
    for (int p = 0; p <= pe; ++p) sz = fma(Bm[l + (int64_t)p * Kc], Yj[p + (int64_t)q * ldj], sz);
    Tz[perm[l] + (int64_t)c * Kc] = sz * sn[c];
    if (l < r) Y[l + (int64_t)c * ldy] = Yj[l + (int64_t)q * ldj] * cs[c];
  }
  __syncthreads();
  CORE_STAMP(17);
  // back substitution Rf11 x = X_k S^{1/2} (Rf11 upper r x r, Rf11(p, l) = R[l + p * Kc]),
  // column oriented: one warp owns columns c = warp + nw q (q < nq <= 4; kk <= 64 = 4 x 16 warps)
  // and walks l = r-1 .. 0 with all of them in lockstep: x_l = y_l / Rf11(l, l), then lanes
  // p < l subtract Rf11(p, l) x_l from y_p. The step is specialised to the warp's exact column
  // count: predicated-off DFMAs would still take turns on the shared FP64 pipe.
  {
    const int warp = tid >> 5, nw = nt >> 5;
    const int nq = kk > warp ? (kk - warp + nw - 1) / nw : 0;
    switch (nq) {
      case 4: backsub_warp<4>(Y, ldy, R, Kc, rdinv, r, warp, nw); break;
      case 3: backsub_warp<3>(Y, ldy, R, Kc, rdinv, r, warp, nw); break;
      case 2: backsub_warp<2>(Y, ldy, R, Kc, rdinv, r, warp, nw); break;
      case 1: backsub_warp<1>(Y, ldy, R, Kc, rdinv, r, warp, nw); break;
      default: break;
    }
  }
  __syncthreads();
  CORE_STAMP(18);
  // scatter to the rows perm[0..r) and undo the equilibration (rows of Tw scale by 1/d_i)
  for (int e = tid; e < K * kk; e += nt) {
    const int l = e % K, c = e / K;
    const int i = perm[l];
    Tw[i + (int64_t)c * Kc] = l < r ? Y[l + (int64_t)c * ldy] * dinv[i] : 0.0;
  }
  CORE_STAMP(7);
  if (tid == 0) {
    *rk = kk;
    double Kd = K;
    auto qr = [](double mm, double kq) {
      return mm >= kq ? 2.0 * mm * kq * kq - 2.0 * kq * kq * kq / 3.0
                      : 2.0 * kq * mm * mm - 2.0 * mm * mm * mm / 3.0;
    };
    // model flops of a fixed schedule, independent of how many pieces the plan merges into one
    // rounded addition: the pieces are added one at a time (§2.3's truncation after every
    // update), each to the target's current rank r: K_i = r + k_i, QR(m, K_i) + QR(n, K_i) +
    // 2 K_i^3 + 21 K_i^3 + 2 (m + n) K_i r', with r' = min(K_i, final rank) carried on
    const int ne = ent ? min(op.n_entries, KMAX_ENTRIES) : 0;
    int ksum = 0;
    for (int e = 0; e < ne; ++e) ksum += max(dimv(B, ent[op.first_entry + e].k, ent[op.first_entry + e].kd), 0);
    int r = max(0, K - ksum);
    double f = 0.0;
    for (int e = 0; e < ne; ++e) {
      const int ke = max(dimv(B, ent[op.first_entry + e].k, ent[op.first_entry + e].kd), 0);
      const double Ki = (double)(r + ke);
      if (Ki <= 0.0) continue;
      const int rn = min(r + ke, kk);
      f += qr(m, Ki) + qr(n, Ki) + 23.0 * Ki * Ki * Ki + 2.0 * (m + n) * Ki * rn;
      r = rn;
    }
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
// Exact kernel matrix times vectors, y = A x with a_ij = 1/(4 pi (|p_i - p_j| + h)), by tiles of
// 128 x 128 point pairs. A is symmetric, so a CTA takes one pair of point tiles (I, J), I <= J,
// evaluates each a_ij once and adds it to both y_i (a_ij x_j, summed in registers) and, for
// I < J, y_j (a_ij x_i, summed in shared memory); the partial sums go to y with atomic adds, so
// y must be zero on entry. Warp w works on the 32-column slice (w + s) mod 4 of tile J in
// super-step s, lane l on column (l + q) mod 32 of it in step q: every column has one writer at
// a time. The entry is formed with one rounding chain of FP64 FMAs instead of IEEE square
// root and division: y = 1/sqrt(r^2) from an FP32 seed (operand and seed moved between FP64
// and FP32 by integer bit moves, r^2 inside the FP32 normal range for any two distinct points
// of coordinates O(1)) corrected by the series of (1 - e)^(-1/2) to second order,
// y (1 + e/2 + 3 e^2 / 8) with e = 1 - r^2 y^2; r = r^2 y; 1/(r + h) by fast_rcp; 1/(4 pi) is
// folded into the staged x. Relative error of each entry ~ 1e-15.
constexpr int XT = 128;       // points per tile
constexpr int XNC = 4;        // right-hand sides per pass

__device__ __forceinline__ double rsqrt_fp64(double x) {
  constexpr long long kBias = (long long)(1023 - 127) << 23;
  const long long xb = __double_as_longlong(x);
  const float xf = __int_as_float((int)((xb >> 29) - kBias));
  float yf;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(yf) : "f"(xf));
  const double y0 = __longlong_as_double(((long long)__float_as_int(yf) + kBias) << 29);
  const double e = fma(-x * y0, y0, 1.0);
  return fma(y0, e * fma(0.375, e, 0.5), y0);
}

__device__ __forceinline__ double kernel_rcp_entry(double dx, double dy, double dz, double h) {
  const double r2 = fma(dx, dx, fma(dy, dy, dz * dz));
  const double r = r2 > 0.0 ? r2 * rsqrt_fp64(r2) : 0.0;
  return fast_rcp(r + h);
}

__global__ void __launch_bounds__(XT) k_exact_mv_sym(const double* __restrict__ P, int n, int nt, double h,
                                                     const double* __restrict__ x, int64_t ldx, double* y,
                                                     int64_t ldy, int c0, int nc) {
  // tile pair (I, J), I <= J, from the linear index b = S(I) + (J - I), S(I) = I nt - I (I - 1) / 2
  const long long b = blockIdx.x;
  int I = (int)(nt + 0.5 - sqrt((nt + 0.5) * (nt + 0.5) - 2.0 * (double)b));
  auto S = [nt](long long i) { return i * nt - i * (i - 1) / 2; };
  while (I > 0 && S(I) > b) --I;
  while (S(I + 1) <= b) ++I;
  const int J = I + (int)(b - S(I));
  __shared__ double pj[3][XT];
  __shared__ double xj[XNC][XT];
  __shared__ double yj[XNC][XT];
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const double scale = 1.0 / (4.0 * M_PI);
  {
    const int j = J * XT + t;
    const bool ok = j < n;
    // padding points sit far away with x = 0: finite entries that add nothing
    pj[0][t] = ok ? P[3 * j] : 1e3 + t;
    pj[1][t] = ok ? P[3 * j + 1] : 1e3;
    pj[2][t] = ok ? P[3 * j + 2] : 1e3;
    for (int c = 0; c < XNC; ++c) {
      xj[c][t] = (ok && c < nc) ? x[j + (int64_t)(c0 + c) * ldx] * scale : 0.0;
      yj[c][t] = 0.0;
    }
  }
  const int i = I * XT + t;
  const bool iok = i < n;
  const double px = iok ? P[3 * i] : -1e3 - t, py = iok ? P[3 * i + 1] : -1e3, pz = iok ? P[3 * i + 2] : -1e3;
  double xi[XNC], acc[XNC];
#pragma unroll
  for (int c = 0; c < XNC; ++c) {
    xi[c] = (iok && c < nc) ? x[i + (int64_t)(c0 + c) * ldx] * scale : 0.0;
    acc[c] = 0.0;
  }
  __syncthreads();
  const bool sym = I < J;
  for (int st = 0; st < 4; ++st) {
    const int base = ((warp + st) & 3) * 32;
    for (int q = 0; q < 32; ++q) {
      const int j = base + ((lane + q) & 31);
      const double a = kernel_rcp_entry(px - pj[0][j], py - pj[1][j], pz - pj[2][j], h);
#pragma unroll
      for (int c = 0; c < XNC; ++c) {
        if (c < nc) {
          acc[c] = fma(a, xj[c][j], acc[c]);
          if (sym) yj[c][j] = fma(a, xi[c], yj[c][j]);
        }
      }
      __syncwarp();
    }
    __syncthreads();
  }
  if (iok)
    for (int c = 0; c < nc; ++c) atomicAdd(&y[i + (int64_t)(c0 + c) * ldy], acc[c]);
  if (sym) {
    const int j = J * XT + t;
    if (j < n)
      for (int c = 0; c < nc; ++c) atomicAdd(&y[j + (int64_t)(c0 + c) * ldy], yj[c][t]);
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
constexpr int TRSM_SMEM = (64 * 65 + 64 * (TRSM_VC + 1)) * (int)sizeof(double);
constexpr int CORE_SMEM = 2 * JSM * (JSM + 1) * (int)sizeof(double);

static void set_attributes() {
  if (g_attr_set) return;
  cudaFuncSetAttribute(k_trsm, cudaFuncAttributeMaxDynamicSharedMemorySize, TRSM_SMEM);
  cudaFuncSetAttribute(k_gemm_t<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, GEMM_SMEM);
  cudaFuncSetAttribute(k_gemm_t<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, GEMM32_SMEM);
  cudaFuncSetAttribute(k_core, cudaFuncAttributeMaxDynamicSharedMemorySize, CORE_SMEM);
  g_attr_set = true;
}

void prepare_kernels() { set_attributes(); }

cudaError_t launch_kind(int kind, const void* ops, int count, const StackEntry* entries, const Bases& B,
                        double h, cudaStream_t s, int gy, int gz) {
  if (count <= 0) return cudaSuccess;
  set_attributes();
  switch (kind) {
    case K_GETRF: k_getrf<<<count, 256, 0, s>>>((const GetrfOp*)ops, B); break;
    case K_TRSM: k_trsm<<<dim3(count, gy), 256, TRSM_SMEM, s>>>((const TrsmOp*)ops, B); break;
    case K_GEMM: k_gemm_t<double><<<dim3(count, gy, gz), 256, GEMM_SMEM, s>>>((const GemmOp*)ops, B); break;
    case K_GEMM32: k_gemm_t<float><<<dim3(count, gy, gz), 256, GEMM32_SMEM, s>>>((const GemmOp*)ops, B); break;
    case K_COPY: k_copy<<<count, 256, 0, s>>>((const CopyOp*)ops, B); break;
    case K_STACK: k_stack<<<dim3(count, gy), 256, 0, s>>>((const TruncOp*)ops, entries, B); break;
    case K_CORE: k_core<<<count, 512, CORE_SMEM, s>>>((const TruncOp*)ops, entries, B); break;
    case K_EVAL: k_eval<<<count, 256, 0, s>>>((const EvalOp*)ops, B, h); break;
    case K_ACA: k_aca<<<count, 256, 0, s>>>((const AcaOp*)ops, B, h); break;
    case K_GEMM_TC: return launch_gemm_tc((const GemmOp*)ops, count, B, s, gy, gz);
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
  if (n <= 0 || nrhs <= 0) return cudaSuccess;
  // y is accumulated with atomic adds: clear it (column by column when ldy > n)
  cudaError_t e = ldy == n ? cudaMemsetAsync(y, 0, (size_t)n * nrhs * sizeof(double), s)
                           : cudaMemset2DAsync(y, (size_t)ldy * sizeof(double), 0, (size_t)n * sizeof(double),
                                               (size_t)nrhs, s);
  if (e) return e;
  const long long nt = (n + XT - 1) / XT;
  const long long pairs = nt * (nt + 1) / 2;
  if (pairs > 0x7fffffffLL) return cudaErrorInvalidValue;
  for (int c0 = 0; c0 < nrhs; c0 += XNC)
    k_exact_mv_sym<<<(unsigned)pairs, XT, 0, s>>>(P, n, (int)nt, h, x, ldx, y, ldy, c0, min(XNC, nrhs - c0));
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

// y[i] = f(x[i]) for one of the reciprocal helpers of the serial sections (which: 0 nr_rcp,
// 1 nr_rsqrt, 2 fast_rcp, 3 pivot_rcp), to check them against IEEE division and square root
__global__ void k_selftest_rcp(const double* __restrict__ x, double* y, int64_t n, int which) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double v = x[i];
  double r;
  switch (which) {
    case 0: r = nr_rcp(v); break;
    case 1: r = nr_rsqrt(v); break;
    case 2: r = fast_rcp(v); break;
    default: r = pivot_rcp(v); break;
  }
  y[i] = r;
}

cudaError_t launch_selftest_rcp(const double* x, double* y, int64_t n, int which, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_selftest_rcp<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(x, y, n, which);
  return cudaGetLastError();
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
