// Skew-symmetric residual and trace kernels for tetrahedra, N = p + 1 = 2..7 (larger N in
// skew_d3_hi.cu), Euler (NC = 5) and linear advection (NC = 1).
#include "skew_inst.cuh"

namespace esd {

cudaError_t launch_skew_residual_d3_hi(int n, int nc, const DevRef& R, const DevMesh& M, const SkewModel& P,
                                       const double* sdir, int epc, int threads, size_t smem, const double* u,
                                       double* dudt, cudaStream_t s);
cudaError_t skew_residual_attrs_d3_hi(int n, int nc, int smem_limit, int* regs, int* max_threads);

#define ESD_SKEW_CASES(X) X(2) X(3) X(4) X(5) X(6) X(7)

cudaError_t launch_skew_residual_d3(int n, int nc, const DevRef& R, const DevMesh& M, const SkewModel& P,
                                    const double* sdir, int epc, int threads, size_t smem, const double* u,
                                    double* dudt, cudaStream_t s) {
#define X(N)                                                                                        \
  case N:                                                                                           \
    return nc == 1 ? launch_skew_residual_n<3, N, 1>(R, M, P, sdir, epc, threads, smem, u, dudt, s) \
                   : launch_skew_residual_n<3, N, 5>(R, M, P, sdir, epc, threads, smem, u, dudt, s);
  switch (n) {
    ESD_SKEW_CASES(X)
    default: return launch_skew_residual_d3_hi(n, nc, R, M, P, sdir, epc, threads, smem, u, dudt, s);
  }
#undef X
}

cudaError_t skew_residual_attrs_d3(int n, int nc, int smem_limit, int* regs, int* max_threads) {
#define X(N) \
  case N: return nc == 1 ? skew_residual_attrs_n<3, N, 1>(smem_limit, regs, max_threads) : skew_residual_attrs_n<3, N, 5>(smem_limit, regs, max_threads);
  switch (n) { ESD_SKEW_CASES(X) default: return skew_residual_attrs_d3_hi(n, nc, smem_limit, regs, max_threads); }
#undef X
}

cudaError_t launch_skew_trace_d3(int nc, const DevRef& R, const DevMesh& M, const SkewModel& P, int epc,
                                 int threads, size_t smem, const double* u, cudaStream_t s) {
  const unsigned grid = (unsigned)((M.E + epc - 1) / epc);
  if (nc == 1)
    skew_trace_kernel<3, 1><<<grid, threads, smem, s>>>(R, M, P, epc, u);
  else
    skew_trace_kernel<3, 5><<<grid, threads, smem, s>>>(R, M, P, epc, u);
  return cudaGetLastError();
}

cudaError_t skew_trace_attrs_d3(int smem_limit) {
  cudaError_t e = cudaFuncSetAttribute(skew_trace_kernel<3, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_limit);
  if (e) return e;
  return cudaFuncSetAttribute(skew_trace_kernel<3, 5>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_limit);
}

}  // namespace esd
