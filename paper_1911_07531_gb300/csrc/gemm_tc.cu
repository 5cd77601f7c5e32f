// Batched GEMM micro-ops on the 5th-generation tensor cores (tcgen05, kind::tf32) for the mixed-
// precision H-LU: the factor products of Alg 1 (low-rank and dense leaf products, their
// application to dense leaves) and the rebuild products of the rounded truncation, with FP32
// accumulation. Operands stay FP64 in memory; each is split on load into two TF32 parts,
// a = a_hi + a_lo (a_hi = tf32(a), a_lo = tf32(a - a_hi) in FP32), and the product is formed as
// a_hi b_hi + a_hi b_lo + a_lo b_hi (three MMAs; the dropped a_lo b_lo term is ~2^-22 |a| |b|),
// which keeps about FP32 accuracy (~1e-6 relative to |A| |B| over the reductions of an H-LU).
//
// A persistent grid (at most two CTAs of 256 threads per SM) walks the micro-ops; a CTA computes
// all 128 x 64 C tiles of its micro-op in turn:
//   - the CTA's 64 TMEM columns hold the 128 x 64 FP32 accumulator of the current tile
//     (lane = row);
//   - for every slice of 64 reduction steps all threads read the FP64 operands from global
//     memory (any strides; groups of eight independent loads), split them and store them in
//     shared memory in the K-major, unswizzled core-matrix layout the MMA reads (8 rows x 16
//     bytes per core matrix; core matrices along K 128 bytes apart, groups of 8 rows 1024 bytes
//     apart), in one stage buffer;
//   - one thread issues the 8 x 3 MMAs of the slice and commits them to the stage's mbarrier;
//     the stage is refilled only after that commit completed (bounded wait);
//   - the 8 warps read the accumulator back (warp w: lanes 32 (w % 4).., columns 32 (w / 4)..)
//     and apply alpha and the micro-op's write mode (atomic add, overwrite, or add).
// A wait that does not end within its bound sets status[4] (the host reports HM_ETIMEOUT), the
// CTA stops issuing, waits (bounded) for what it issued, frees its TMEM and exits.
#include <cuda_runtime.h>

#include <cstdint>

#include "kernels.h"

namespace hm {

namespace {

constexpr int TM = 128;          // rows of a C tile (MMA M)
constexpr int TN = 64;           // columns of a C tile (MMA N)
constexpr int TK = 64;           // reduction steps per staged slice (8 MMAs of K = 8)
constexpr int TMEM_COLS = 64;    // FP32 accumulator columns
constexpr int A_BYTES = TM * TK * 4;    // one TF32 part of the A slice
constexpr int B_BYTES = TN * TK * 4;
constexpr long long WAIT_LIMIT = 1ll << 26;   // polls of an mbarrier before giving up

__device__ __forceinline__ double* tc_dptr(const Bases& B, uint64_t r) {
  return r ? B.d[(r >> 60) - 1] + (r & REF_MASK) : nullptr;
}
__device__ __forceinline__ int tc_dimv(const Bases& B, int s, uint64_t d) {
  return s + (d ? *(B.i[(d >> 60) - 1] + (d & REF_MASK)) : 0);
}

__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ unsigned to_tf32(float x) {
  unsigned r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

// float offset of element (row, kk) of a K-major core-matrix tile with TK K per row group
__device__ __forceinline__ int kmajor_off(int row, int kk) {
  return (row >> 3) * (8 * TK) + (kk >> 2) * 32 + (row & 7) * 4 + (kk & 3);
}
constexpr unsigned SBO = 8 * TK * 4;   // bytes between groups of 8 rows
constexpr unsigned LBO = 128;          // bytes between core matrices along K

// shared-memory matrix descriptor: start, leading (K) and stride (8-row) byte offsets, no swizzle
__device__ __forceinline__ uint64_t smem_desc(unsigned addr, unsigned lbo, unsigned sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((addr & 0x3FFFF) >> 4);
  d |= (uint64_t)((lbo & 0x3FFFF) >> 4) << 16;
  d |= (uint64_t)((sbo & 0x3FFFF) >> 4) << 32;
  d |= (uint64_t)1 << 46;          // fixed 0b001 in bits 46-48
  return d;                        // base offset 0, relative LBO, SWIZZLE_NONE
}

// instruction descriptor of kind::tf32: D FP32, A and B TF32, both K-major, M = 128, N = 64
__host__ __device__ constexpr unsigned tf32_idesc() {
  return (1u << 4)                 // D format: F32
         | (2u << 7)               // A format: TF32
         | (2u << 10)              // B format: TF32
         | ((unsigned)(TN >> 3) << 17) | ((unsigned)(TM >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(unsigned tmem, uint64_t a, uint64_t b, unsigned idesc, int accum) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(accum)
      : "memory");
}

__device__ __forceinline__ void mma_commit(unsigned mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(mbar)
               : "memory");
}

// bounded wait for the mbarrier phase `parity` to complete; false if the bound was reached
__device__ __forceinline__ bool mbar_wait(unsigned mbar, unsigned parity) {
  for (long long it = 0; it < WAIT_LIMIT; ++it) {
    unsigned done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(done)
        : "r"(mbar), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

__device__ __forceinline__ void tmem_ld16(unsigned taddr, float (&v)[16]) {
  unsigned r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
      "%14, %15}, [%16];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
  for (int q = 0; q < 16; ++q) v[q] = __uint_as_float(r[q]);
}

}  // namespace

constexpr int STAGE_BYTES = 2 * A_BYTES + 2 * B_BYTES;   // hi and lo parts of one A and one B slice
constexpr int TC_SMEM = STAGE_BYTES + 64;                   // one stage + mbarrier + TMEM slot

// Stage slice [l0, l0 + TK) of rows [r0, r0 + rmax) of X (X(r, l) = X[r rs + l cs]) into the
// hi / lo TF32 tiles: only the rmax valid rows are written (rows past them feed only outputs that
// are never stored), reduction steps past k as zeros. A thread's loads of a group are issued
// before any of them is converted, so that they are in flight together.
__device__ __forceinline__ void stage_operand(const double* __restrict__ X, int64_t rs, int64_t cs, int r0, int rmax,
                                              int l0, int k, bool r_fast, float* hi, float* lo) {
  constexpr int GROUP = 8;
  const int total = rmax * TK;
  for (int g0 = threadIdx.x; g0 < total; g0 += 256 * GROUP) {
    double v[GROUP];
#pragma unroll
    for (int q = 0; q < GROUP; ++q) {
      const int e = g0 + 256 * q;
      const int r = r_fast ? e % rmax : e / TK, l = r_fast ? e / rmax : e % TK;
      v[q] = (e < total && l0 + l < k) ? X[(int64_t)(r0 + r) * rs + (int64_t)(l0 + l) * cs] : 0.0;
    }
#pragma unroll
    for (int q = 0; q < GROUP; ++q) {
      const int e = g0 + 256 * q;
      if (e >= total) break;
      const int r = r_fast ? e % rmax : e / TK, l = r_fast ? e / rmax : e % TK;
      const int o = kmajor_off(r, l);
      const float f = (float)v[q];
      const unsigned h = to_tf32(f);
      hi[o] = __uint_as_float(h);
      lo[o] = __uint_as_float(to_tf32(f - __uint_as_float(h)));
    }
  }
}

// Persistent: a CTA takes micro-ops blockIdx.x, blockIdx.x + gridDim.x, ... and computes every
// 128 x 64 tile of each, keeping its TMEM and mbarrier.
__global__ void __launch_bounds__(256, 2) k_gemm_tc(const GemmOp* __restrict__ ops, int count, Bases B) {
  extern __shared__ __align__(1024) unsigned char tsm[];
  float* Ahi = (float*)tsm;
  float* Alo = (float*)(tsm + A_BYTES);
  float* Bhi = (float*)(tsm + 2 * A_BYTES);
  float* Blo = (float*)(tsm + 2 * A_BYTES + B_BYTES);
  uint64_t* mbar = (uint64_t*)(tsm + STAGE_BYTES);
  unsigned* tslot = (unsigned*)(mbar + 1);
  const int tid = threadIdx.x, warp = tid >> 5;
  const unsigned mbar_a = smem_u32(mbar);
  const unsigned ah = smem_u32(Ahi), al = smem_u32(Alo), bh = smem_u32(Bhi), bl = smem_u32(Blo);

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(tslot)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(mbar_a) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const unsigned tmem = *tslot;
  const unsigned idesc = tf32_idesc();
  unsigned phase = 0;
  bool ok = true;
  for (int opi = blockIdx.x; opi < count && ok; opi += gridDim.x) {
    const GemmOp& op = ops[opi];
    const int m = tc_dimv(B, op.m, op.md), n = tc_dimv(B, op.n, op.nd), k = max(tc_dimv(B, op.k, op.kd), 0);
    const bool atomic = op.flags & GF_ATOMIC, overwrite = op.flags & GF_OVERWRITE;
    if (m <= 0 || n <= 0 || (k == 0 && !overwrite)) continue;
    if (tid == 0) {
      const unsigned long long f = (unsigned long long)(2.0 * m * n * (double)k);
      if (op.fclass < FC_NONE) atomicAdd(&B.flops[op.fclass], f);
      atomicAdd(&B.flops[NFC + K_GEMM_TC], f);
    }
    const int mt = (m + TM - 1) / TM, ntl = (n + TN - 1) / TN;
    const int nslices = (k + TK - 1) / TK;
    const double* A = tc_dptr(B, op.A);
    const double* Bm = tc_dptr(B, op.B);
    double* C = tc_dptr(B, op.C);
    const bool a_i_fast = op.a_rs <= op.a_cs;
    const bool b_j_fast = op.b_cs <= op.b_rs;
    for (int tile = 0; tile < mt * ntl && ok; ++tile) {
      const int i0 = (tile % mt) * TM, j0 = (tile / mt) * TN;
      const int mrows = min(TM, m - i0), ncols = min(TN, n - j0);
      for (int sl = 0; sl < nslices; ++sl) {
        const int l0 = sl * TK;
        stage_operand(A, op.a_rs, op.a_cs, i0, mrows, l0, k, a_i_fast, Ahi, Alo);
        stage_operand(Bm, op.b_cs, op.b_rs, j0, ncols, l0, k, b_j_fast, Bhi, Blo);
        // make the generic-proxy stores visible to the tensor core (async proxy)
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        __syncthreads();
        if (tid == 0) {
          asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
          const int ksteps = (min(TK, k - l0) + 7) / 8;
#pragma unroll 1
          for (int q = 0; q < ksteps; ++q) {
            const unsigned off = q * 256;   // two core matrices of 128 bytes per K = 8 step
            const uint64_t dah = smem_desc(ah + off, LBO, SBO), dal = smem_desc(al + off, LBO, SBO);
            const uint64_t dbh = smem_desc(bh + off, LBO, SBO), dbl = smem_desc(bl + off, LBO, SBO);
            mma_tf32(tmem, dah, dbh, idesc, (sl > 0 || q > 0) ? 1 : 0);
            mma_tf32(tmem, dah, dbl, idesc, 1);
            mma_tf32(tmem, dal, dbh, idesc, 1);
          }
          mma_commit(mbar_a);
        }
        // the slice buffer is refilled, and the accumulator read, only after the MMAs completed
        ok = __syncthreads_and(mbar_wait(mbar_a, phase)) != 0;
        phase ^= 1u;
        if (!ok) break;
      }
      if (!ok) break;
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
      // epilogue: warp w reads lanes 32 (w % 4) .. of columns 32 (w / 4) ..; row = lane of TMEM
      const int quarter = warp & 3, half = warp >> 2;
      const int gi = i0 + 32 * quarter + (tid & 31);
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int c0 = 32 * half + 16 * h;
        if (c0 >= ncols) continue;                       // warp-uniform
        float v[16];
        const unsigned taddr = tmem + ((unsigned)(32 * quarter) << 16) + (unsigned)c0;
        if (nslices > 0) {
          tmem_ld16(taddr, v);
        } else {
#pragma unroll
          for (int q = 0; q < 16; ++q) v[q] = 0.0f;
        }
        if (gi < m) {
#pragma unroll
          for (int q = 0; q < 16; ++q) {
            const int gj = j0 + c0 + q;
            if (gj < n) {
              double* c = C + (int64_t)gi * op.c_rs + (int64_t)gj * op.c_cs;
              const double val = op.alpha * (double)v[q];
              if (atomic) atomicAdd(c, val);
              else if (overwrite) *c = val;
              else *c += val;
            }
          }
        }
      }
      // the next tile's first MMA overwrites the accumulator: every read of it must be done
      asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
      __syncthreads();
    }
  }
  if (!ok && tid == 0) atomicAdd(&B.status[4], 1);
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
  }
}

cudaError_t launch_gemm_tc(const GemmOp* ops, int count, const Bases& B, cudaStream_t s, int gy, int gz) {
  (void)gy;
  (void)gz;
  if (count <= 0) return cudaSuccess;
  static int grid_cap = 0;
  if (!grid_cap) {
    cudaError_t e = cudaFuncSetAttribute(k_gemm_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM);
    if (e) return e;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) sms = 152;
    grid_cap = 2 * sms;   // two resident CTAs per SM (registers and shared memory)
  }
  const int grid = count < grid_cap ? count : grid_cap;
  k_gemm_tc<<<grid, 256, TC_SMEM, s>>>(ops, count, B);
  return cudaGetLastError();
}

}  // namespace hm
