// Skew-symmetric residual and trace kernels for triangles, every degree (N = p + 1 = 2..11),
// Euler (NC = 4) and linear advection (NC = 1).
#include "skew_inst.cuh"

namespace esd {

#define ESD_SKEW_CASES(X) X(2) X(3) X(4) X(5) X(6) X(7) X(8) X(9) X(10) X(11)

cudaError_t launch_skew_residual_d2(int n, int nc, const DevRef& R, const DevMesh& M, const SkewModel& P,
                                    const double* sdir, int epc, int threads, size_t smem, const double* u,
                                    double* dudt, cudaStream_t s) {
#define X(N)                                                                                        \
  case N:                                                                                           \
    return nc == 1 ? launch_skew_residual_n<2, N, 1>(R, M, P, sdir, epc, threads, smem, u, dudt, s) \
                   : launch_skew_residual_n<2, N, 4>(R, M, P, sdir, epc, threads, smem, u, dudt, s);
  switch (n) { ESD_SKEW_CASES(X) default: return cudaErrorInvalidValue; }
#undef X
}

cudaError_t skew_residual_attrs_d2(int n, int nc, int smem_limit, int* regs, int* max_threads) {
#define X(N) \
  case N: return nc == 1 ? skew_residual_attrs_n<2, N, 1>(smem_limit, regs, max_threads) : skew_residual_attrs_n<2, N, 4>(smem_limit, regs, max_threads);
  switch (n) { ESD_SKEW_CASES(X) default: return cudaErrorInvalidValue; }
#undef X
}

cudaError_t launch_skew_trace_d2(int nc, const DevRef& R, const DevMesh& M, const SkewModel& P, int epc,
                                 int threads, size_t smem, const double* u, cudaStream_t s) {
  const unsigned grid = (unsigned)((M.E + epc - 1) / epc);
  if (nc == 1)
    skew_trace_kernel<2, 1><<<grid, threads, smem, s>>>(R, M, P, epc, u);
  else
    skew_trace_kernel<2, 4><<<grid, threads, smem, s>>>(R, M, P, epc, u);
  return cudaGetLastError();
}

cudaError_t skew_trace_attrs_d2(int smem_limit) {
  cudaError_t e = cudaFuncSetAttribute(skew_trace_kernel<2, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_limit);
  if (e) return e;
  return cudaFuncSetAttribute(skew_trace_kernel<2, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_limit);
}

}  // namespace esd
