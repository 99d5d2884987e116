// Residual kernels for tetrahedra with pair directions formed on the fly from per-node
// metric terms (meshes created with ESD_MESH_METRICS_ON_THE_FLY), N = p + 1 = 2..11.
#include "residual_inst.cuh"

namespace esd {

#define ESD_CASES(X) X(2) X(3) X(4) X(5) X(6) X(7) X(8) X(9) X(10) X(11)

cudaError_t launch_residual_otf_d3(const DevRef& R, const DevMesh& M, const LaunchCfg& L, const Epilogue& ep,
                                   cudaStream_t s) {
#define X(N) case N: return launch_residual_otf_n<3, N>(R, M, L, ep, s);
  switch (R.n) { ESD_CASES(X) default: return cudaErrorInvalidValue; }
#undef X
}

cudaError_t set_residual_otf_smem_d3(int lim) {
  cudaError_t e = cudaSuccess;
#define X(N) if (!e) e = set_residual_otf_smem_n<3, N>(lim);
  ESD_CASES(X)
#undef X
  return e;
}

}  // namespace esd
