// Residual kernels for tetrahedra, one instantiation per nodes-per-line N = p + 1
// (N <= 7 here, larger N in residual_d3_hi.cu).
#include "residual_inst.cuh"

namespace esd {

#define ESD_CASES(X) X(2) X(3) X(4) X(5) X(6) X(7)

cudaError_t launch_residual_d3(const DevRef& R, const DevMesh& M, const LaunchCfg& L, const Epilogue& ep,
                               cudaStream_t s) {
#define X(N) case N: return launch_residual_n<3, N>(R, M, L, ep, s);
  switch (R.n) { ESD_CASES(X) default: return launch_residual_d3_hi(R, M, L, ep, s); }
#undef X
}

cudaError_t launch_residual_batch_d3(int n, const BatchMesh* meshes, const BatchItem* items, int nitems, int grid,
                                     int threads, size_t smem, cudaStream_t s) {
#define X(N) case N: return launch_residual_batch_n<3, N>(meshes, items, nitems, grid, threads, smem, s);
  switch (n) { ESD_CASES(X) default: return launch_residual_batch_d3_hi(n, meshes, items, nitems, grid, threads, smem, s); }
#undef X
}

cudaError_t set_residual_smem_d3(int lim) {
  cudaError_t e = cudaSuccess;
#define X(N) if (!e) e = set_residual_smem_n<3, N>(lim);
  ESD_CASES(X)
#undef X
  if (!e) e = set_residual_smem_d3_hi(lim);
  return e;
}

}  // namespace esd
