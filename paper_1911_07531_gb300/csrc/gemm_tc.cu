// Batched GEMM micro-ops on the 5th-generation tensor cores (tcgen05, kind::tf32) for the mixed-
// precision H-LU: the factor products of Alg 1 (low-rank and dense leaf products, their
// application to dense leaves) and the rebuild products of the rounded truncation, with FP32
// accumulation. Operands stay FP64 in memory; each is split on load into two TF32 parts,
// a = a_hi + a_lo (a_hi = tf32(a), a_lo = tf32(a - a_hi) in FP32), and the product is formed as
// a_hi b_hi + a_hi b_lo + a_lo b_hi (three MMAs; the dropped a_lo b_lo term is ~2^-22 |a| |b|),
// which keeps about FP32 accuracy (~1e-6 relative to |A| |B| over the reductions of an H-LU).
//
// One CTA (256 threads) computes one 128 x 64 tile of C for one micro-op:
//   - the CTA's 64 TMEM columns hold the 128 x 64 FP32 accumulator (lane = row);
//   - for every slice of 32 reduction steps all threads read the FP64 operands from global
//     memory (any strides), split them and store them in shared memory in the K-major,
//     unswizzled core-matrix layout the MMA reads (8 rows x 16 bytes per core matrix; core
//     matrices along K 128 bytes apart, groups of 8 rows 1024 bytes apart);
//   - one thread issues the 4 x 3 MMAs of the slice and commits them to an mbarrier; every
//     thread waits on it (bounded) before the slice buffer is refilled;
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
constexpr int TK = 32;           // reduction steps per staged slice (4 MMAs of K = 8)
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

// float offset of element (row, kk) of a K-major core-matrix tile with 32 K per row group
__device__ __forceinline__ int kmajor_off(int row, int kk) {
  return (row >> 3) * (8 * 32) + (kk >> 2) * 32 + (row & 7) * 4 + (kk & 3);
}

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

constexpr int TC_SMEM = 2 * A_BYTES + 2 * B_BYTES + 64;

__global__ void __launch_bounds__(256) k_gemm_tc(const GemmOp* __restrict__ ops, Bases B) {
  const GemmOp op = ops[blockIdx.x];
  const int m = tc_dimv(B, op.m, op.md), n = tc_dimv(B, op.n, op.nd), k = max(tc_dimv(B, op.k, op.kd), 0);
  const bool atomic = op.flags & GF_ATOMIC, overwrite = op.flags & GF_OVERWRITE;
  if (m <= 0 || n <= 0) return;
  if (k == 0 && !overwrite) return;
  const int mt = (m + TM - 1) / TM, ntl = (n + TN - 1) / TN;
  const int tile = blockIdx.y;
  if (tile == 0 && threadIdx.x == 0 && mt * ntl > (int)gridDim.y) atomicAdd(&B.status[5], 1);   // planner bound
  if (tile >= mt * ntl) return;
  const int i0 = (tile % mt) * TM, j0 = (tile / mt) * TN;

  extern __shared__ __align__(1024) unsigned char tsm[];
  float* Ahi = (float*)tsm;
  float* Alo = (float*)(tsm + A_BYTES);
  float* Bhi = (float*)(tsm + 2 * A_BYTES);
  float* Blo = (float*)(tsm + 2 * A_BYTES + B_BYTES);
  uint64_t* mbar = (uint64_t*)(tsm + 2 * A_BYTES + 2 * B_BYTES);
  unsigned* tslot = (unsigned*)(mbar + 1);
  const int tid = threadIdx.x, warp = tid >> 5;
  const unsigned mbar_a = smem_u32(mbar);

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

  const double* A = tc_dptr(B, op.A);
  const double* Bm = tc_dptr(B, op.B);
  const bool a_i_fast = op.a_rs <= op.a_cs;
  const bool b_j_fast = op.b_cs <= op.b_rs;
  const unsigned idesc = tf32_idesc();
  const int nslices = (k + TK - 1) / TK;
  unsigned phase = 0;
  bool ok = true;
  int issued = 0;   // commits issued and not yet waited for
  for (int sl = 0; sl < nslices && ok; ++sl) {
    const int l0 = sl * TK;
    // stage the slice: A (TM x TK) and B (TK x TN, stored N x K), split into TF32 hi / lo parts
    for (int e = tid; e < TM * TK; e += 256) {
      int i, l;
      if (a_i_fast) {
        i = e % TM;
        l = e / TM;
      } else {
        l = e % TK;
        i = e / TK;
      }
      const int gi = i0 + i, gl = l0 + l;
      float v = 0.0f;
      if (gi < m && gl < k) v = (float)A[(int64_t)gi * op.a_rs + (int64_t)gl * op.a_cs];
      const unsigned hi = to_tf32(v);
      const unsigned lo = to_tf32(v - __uint_as_float(hi));
      const int o = kmajor_off(i, l);
      Ahi[o] = __uint_as_float(hi);
      Alo[o] = __uint_as_float(lo);
    }
    for (int e = tid; e < TN * TK; e += 256) {
      int j, l;
      if (b_j_fast) {
        j = e % TN;
        l = e / TN;
      } else {
        l = e % TK;
        j = e / TK;
      }
      const int gj = j0 + j, gl = l0 + l;
      float v = 0.0f;
      if (gj < n && gl < k) v = (float)Bm[(int64_t)gl * op.b_rs + (int64_t)gj * op.b_cs];
      const unsigned hi = to_tf32(v);
      const unsigned lo = to_tf32(v - __uint_as_float(hi));
      const int o = kmajor_off(j, l);
      Bhi[o] = __uint_as_float(hi);
      Blo[o] = __uint_as_float(lo);
    }
    // make the generic-proxy stores visible to the tensor core (async proxy)
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
      const unsigned ah = smem_u32(Ahi), al = smem_u32(Alo), bh = smem_u32(Bhi), bl = smem_u32(Blo);
      const int ksteps = (min(TK, k - l0) + 7) / 8;
#pragma unroll 1
      for (int q = 0; q < ksteps; ++q) {
        const unsigned off = q * 256;   // two core matrices of 128 bytes per K = 8 step
        const uint64_t dah = smem_desc(ah + off, 128, 1024), dal = smem_desc(al + off, 128, 1024);
        const uint64_t dbh = smem_desc(bh + off, 128, 1024), dbl = smem_desc(bl + off, 128, 1024);
        mma_tf32(tmem, dah, dbh, idesc, (sl > 0 || q > 0) ? 1 : 0);
        mma_tf32(tmem, dah, dbl, idesc, 1);
        mma_tf32(tmem, dal, dbh, idesc, 1);
      }
      mma_commit(mbar_a);
    }
    issued = 1;
    // the slice buffer is refilled only after the MMAs that read it have completed; the
    // outcome is made uniform over the CTA
    ok = __syncthreads_and(mbar_wait(mbar_a, phase)) != 0;
    issued = ok ? 0 : 1;
    phase ^= 1;
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  }
  if (!ok) {
    if (tid == 0) atomicAdd(&B.status[4], 1);
    if (issued) mbar_wait(mbar_a, phase ^ 1);   // once more, bounded, for the MMAs in flight
  } else {
    // epilogue: warp w reads lanes 32 (w % 4) .. of columns 32 (w / 4) ..; row = lane of TMEM
    const int quarter = warp & 3, half = warp >> 2;
    const int row = 32 * quarter + (tid & 31);
    const int gi = i0 + row;
    double* C = tc_dptr(B, op.C);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int c0 = 32 * half + 16 * h;
      float v[16];
      const unsigned taddr = tmem + ((unsigned)(32 * quarter) << 16) + (unsigned)c0;
      if (k > 0) {
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
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
  }
  if (tid == 0 && blockIdx.y == 0) {
    const unsigned long long f = (unsigned long long)(2.0 * m * n * (double)k);
    if (op.fclass < FC_NONE) atomicAdd(&B.flops[op.fclass], f);
    atomicAdd(&B.flops[NFC + K_GEMM_TC], f);
  }
}

cudaError_t launch_gemm_tc(const GemmOp* ops, int count, const Bases& B, cudaStream_t s, int gy) {
  if (count <= 0) return cudaSuccess;
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_gemm_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM);
    if (e) return e;
    attr = true;
  }
  k_gemm_tc<<<dim3(count, gy), 256, TC_SMEM, s>>>(ops, B);
  return cudaGetLastError();
}

}  // namespace hm
