// Host-callable launchers of the batched kernels (kernels.cu).
#pragma once

#include <cuda_runtime.h>

#include "ops.h"

namespace hm {

// sets the kernels' shared-memory attributes (call before capturing launches into a graph)
void prepare_kernels();
// gy, gz: extra grid dimensions of a GEMM launch (C tiles and reduction slices of one
// micro-op spread over several CTAs); ignored by the other kinds
cudaError_t launch_kind(int kind, const void* ops, int count, const StackEntry* entries, const Bases& B,
                        double h, cudaStream_t s, int gy = 1, int gz = 1);
// K_GEMM_TC launch: a persistent grid of at most two CTAs per SM walks the micro-ops (gy, gz
// unused: every CTA computes whole micro-ops)
cudaError_t launch_gemm_tc(const GemmOp* ops, int count, const Bases& B, cudaStream_t s, int gy, int gz);
cudaError_t launch_nn2(const double* P, int n, double* out, cudaStream_t s);
cudaError_t launch_exact_mv(const double* P, int n, double h, const double* x, int64_t ldx, double* y,
                            int64_t ldy, int nrhs, cudaStream_t s);
cudaError_t launch_permute(const double* src, int64_t lds, double* dst, int64_t ldd, const int64_t* perm,
                           int n, int nrhs, int scatter, double alpha, double beta, int accumulate,
                           cudaStream_t s);
cudaError_t launch_set_int(int* p, int v, cudaStream_t s);
cudaError_t launch_permute_points(const double* P, const int64_t* perm, int n, double* out, cudaStream_t s);

}  // namespace hm

namespace hm {
cudaError_t launch_colnorm2(const double* x, int64_t ld, int n, int nrhs, double* out, cudaStream_t s);
cudaError_t launch_selftest_rcp(const double* x, double* y, int64_t n, int which, cudaStream_t s);
cudaError_t launch_axpby(const double* x, int64_t ldx, double* y, int64_t ldy, int n, int nrhs, double alpha,
                         double beta, cudaStream_t s);
}  // namespace hm
