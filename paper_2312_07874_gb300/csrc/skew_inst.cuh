// Skew-symmetric residual kernels instantiated per (dimension, nodes per line N, model):
// included by skew_d2.cu, skew_d3.cu and skew_d3_hi.cu so that the instantiations
// compile in parallel.  Model: NC = dim + 2 (Euler) or NC = 1 (linear advection).
#pragma once

#include "skew.cuh"

namespace esd {

template <int D, int N, int NC>
cudaError_t launch_skew_residual_n(const DevRef& R, const DevMesh& M, const SkewModel& P, const double* sdir,
                                   int epc, int threads, size_t smem, const double* u, double* dudt,
                                   cudaStream_t s) {
  const unsigned grid = (unsigned)((M.E + epc - 1) / epc);
  skew_residual_kernel<D, N, NC><<<grid, threads, smem, s>>>(R, M, P, sdir, epc, u, dudt);
  return cudaGetLastError();
}

// Sets the kernel's dynamic shared-memory limit and reports its registers per thread and
// the largest block the runtime accepts for it (registers included).
template <int D, int N, int NC>
cudaError_t skew_residual_attrs_n(int smem_limit, int* regs, int* max_threads) {
  cudaError_t e = cudaFuncSetAttribute(skew_residual_kernel<D, N, NC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       smem_limit);
  if (e) return e;
  cudaFuncAttributes a;
  e = cudaFuncGetAttributes(&a, skew_residual_kernel<D, N, NC>);
  if (!e) {
    *regs = a.numRegs;
    *max_threads = a.maxThreadsPerBlock;
  }
  return e;
}

}  // namespace esd

