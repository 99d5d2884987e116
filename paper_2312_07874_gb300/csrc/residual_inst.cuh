// Residual kernels instantiated per (dimension, nodes per line); included by
// residual_d2.cu and residual_d3.cu so that each instantiation gets its own
// register allocation and the two dimensions compile in parallel.
#pragma once

#include "device.cuh"

namespace esd {

template <int D, int N, bool OTF = false>
__global__ void residual_kernel(DevRef R, DevMesh M, int epc, Epilogue ep) {
  const int64_t e0 = (int64_t)blockIdx.x * epc;
  const int E = (int)((M.E - e0) < (int64_t)epc ? (M.E - e0) : (int64_t)epc);
  residual_tile<D, N, OTF>(R, M, e0, E, ep);
}

// Batched execution of many meshes with the same (dimension, degree): a persistent grid
// walks a list of (mesh, element tile) items; each item runs the same tile code with that
// mesh's tables, layout and epilogue.
template <int D, int N>
__global__ void residual_batch_kernel(const BatchMesh* __restrict__ meshes, const BatchItem* __restrict__ items,
                                      int nitems) {
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const BatchItem w = items[it];
    const BatchMesh& bm = meshes[w.mesh];
    residual_tile<D, N>(bm.R, bm.M, w.e0, w.E, bm.ep);
    __syncthreads();
  }
}

template <int D, int N>
cudaError_t launch_residual_n(const DevRef& R, const DevMesh& M, const LaunchCfg& L, const Epilogue& ep,
                              cudaStream_t s) {
  const unsigned grid = (unsigned)((M.E + L.eb - 1) / L.eb);
  residual_kernel<D, N><<<grid, L.tb, L.sb, s>>>(R, M, L.eb, ep);
  return cudaGetLastError();
}

template <int D, int N>
cudaError_t launch_residual_batch_n(const BatchMesh* meshes, const BatchItem* items, int nitems, int grid,
                                    int threads, size_t smem, cudaStream_t s) {
  residual_batch_kernel<D, N><<<grid, threads, smem, s>>>(meshes, items, nitems);
  return cudaGetLastError();
}

template <int D, int N>
cudaError_t set_residual_smem_n(int lim) {
  cudaError_t e = cudaFuncSetAttribute(residual_kernel<D, N>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  if (e) return e;
  return cudaFuncSetAttribute(residual_batch_kernel<D, N>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
}

}  // namespace esd

namespace esd {

// The residual kernel with pair directions formed on the fly (residual_otf_*.cu).
template <int D, int N>
cudaError_t launch_residual_otf_n(const DevRef& R, const DevMesh& M, const LaunchCfg& L, const Epilogue& ep,
                                  cudaStream_t s) {
  const unsigned grid = (unsigned)((M.E + L.eb - 1) / L.eb);
  residual_kernel<D, N, true><<<grid, L.tb, L.sb, s>>>(R, M, L.eb, ep);
  return cudaGetLastError();
}

template <int D, int N>
cudaError_t set_residual_otf_smem_n(int lim) {
  return cudaFuncSetAttribute(residual_kernel<D, N, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
}

}  // namespace esd
