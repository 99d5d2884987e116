// Residual kernels for tetrahedra of degree 7 to 10 (nodes per line N = p + 1 = 8..11),
// in their own translation unit so that they compile in parallel with the lower degrees.
#include "residual_inst.cuh"

namespace esd {

#define ESD_CASES(X) X(8) X(9) X(10) X(11)

cudaError_t launch_residual_d3_hi(const DevRef& R, const DevMesh& M, const LaunchCfg& L, const Epilogue& ep,
                                  cudaStream_t s) {
#define X(N) case N: return launch_residual_n<3, N>(R, M, L, ep, s);
  switch (R.n) { ESD_CASES(X) default: return cudaErrorInvalidValue; }
#undef X
}

cudaError_t launch_residual_batch_d3_hi(int n, const BatchMesh* meshes, const BatchItem* items, int nitems,
                                        int grid, int threads, size_t smem, cudaStream_t s) {
#define X(N) case N: return launch_residual_batch_n<3, N>(meshes, items, nitems, grid, threads, smem, s);
  switch (n) { ESD_CASES(X) default: return cudaErrorInvalidValue; }
#undef X
}

cudaError_t set_residual_smem_d3_hi(int lim) {
  cudaError_t e = cudaSuccess;
#define X(N) if (!e) e = set_residual_smem_n<3, N>(lim);
  ESD_CASES(X)
#undef X
  return e;
}

}  // namespace esd
