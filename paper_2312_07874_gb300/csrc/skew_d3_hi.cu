// Skew-symmetric residual kernels for tetrahedra of degree 7..10 (N = 8..11).
#include "skew_inst.cuh"

namespace esd {

#define ESD_SKEW_CASES(X) X(8) X(9) X(10) X(11)

cudaError_t launch_skew_residual_d3_hi(int n, int nc, const DevRef& R, const DevMesh& M, const SkewModel& P,
                                       const double* sdir, int epc, int threads, size_t smem, const double* u,
                                       double* dudt, cudaStream_t s) {
#define X(N)                                                                                        \
  case N:                                                                                           \
    return nc == 1 ? launch_skew_residual_n<3, N, 1>(R, M, P, sdir, epc, threads, smem, u, dudt, s) \
                   : launch_skew_residual_n<3, N, 5>(R, M, P, sdir, epc, threads, smem, u, dudt, s);
  switch (n) { ESD_SKEW_CASES(X) default: return cudaErrorInvalidValue; }
#undef X
}

cudaError_t skew_residual_attrs_d3_hi(int n, int nc, int smem_limit, int* regs, int* max_threads) {
#define X(N) \
  case N: return nc == 1 ? skew_residual_attrs_n<3, N, 1>(smem_limit, regs, max_threads) : skew_residual_attrs_n<3, N, 5>(smem_limit, regs, max_threads);
  switch (n) { ESD_SKEW_CASES(X) default: return cudaErrorInvalidValue; }
#undef X
}

}  // namespace esd
