// Internal declarations shared by the host setup (setup.cpp), the kernels
// (kernels.cu, residual_d*.cu and the device headers) and the C ABI (api.cu).  Not part of
// the public interface.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "esd_test.h"   // the product ABI (esd.h) and the test hooks

namespace esd {

constexpr int kMaxPTri = 10;
constexpr int kMaxPTet = 10;

// Number of per-node fields kept for the two-point flux: rho, v_1..v_d, p,
// beta = rho/p, ln rho, ln beta.
constexpr int nfields(int dim) { return dim + 5; }

// Reference-element tables for one (dim, p), built on the host (setup.cpp).
// Index conventions (internal to the library):
//   volume node   v = c1 + n*(c2 + n*c3)          (c_k = index along eta_k)
//   facet node    f = zeta*Nqf + j, j = a + n*b    (a along the first facet
//                 coordinate, b along the second; triangles j = a)
//   modes         the ABI order (alpha_1 slowest)
struct RefTables {
  int dim = 0, p = 0, n = 0, Nq = 0, Np = 0, Nf = 0, Nqf = 0, Nfn = 0, Ntot = 0;
  int T = 0;      // line tasks per phase, n^(dim-1)
  int Lv = 0;     // pairs per line, q(q+1)/2
  int S12 = 0;    // number of (alpha1, alpha2) pairs (tetrahedra)
  int nvp = 0, nfp = 0;          // volume / facet pairs per element
  int fph_off[4] = {0, 0, 0, 0}; // offsets (in doubles) of the facet pair phases in fdir
  int fph_len[4] = {0, 0, 0, 0}; // facet pairs per task in each phase
  std::vector<double> eta[3], w1[3];
  std::vector<double> dl[3];          // dl[k][a*n+b] = d ell_{k,b}/d eta (eta_{k,a})
  std::vector<double> l1m, l1p, l2m, l3m, L2J;
  std::vector<double> psi1, psi2, psi3;
  std::vector<int> ints;              // off1[p+1] | s12_a1[S12] | moff[S12] | mode_s12[Np] (tri: mode_a1[Np])
                                      // | s12 by decreasing alpha3 length [S12] (tets)
  int i_off1 = 0, i_s12a1 = 0, i_moff = 0, i_mode = 0, i_s12len = 0;
  std::vector<double> wvol;           // [Nq]
  std::vector<double> wfac;           // [Nfn]
  std::vector<double> xi_vol, xi_fac; // [Nq*dim], [Nfn*dim]
  std::vector<double> deta;           // [Nq][3][3]: d eta_k / d xi_l at volume nodes (k-major)
  double nhat[4][3] = {};
  std::vector<double> Vd;             // [Nq][Np] dense generalized Vandermonde (library node order)
  int dense_minv = 0;                 // apply V^T (W/J) V as a stored per-element Np x Np matrix
};

// Per-mesh host geometry (setup.cpp) ready to upload.
struct HostMesh {
  RefTables ref;
  int64_t E = 0;
  std::vector<double> vdir, fdir;     // [E][nvp*dim], [E][nfp*dim] (phase-major)
  std::vector<double> wj, wdj;        // [E][Nq] W J and W / J (interpolated J)
  std::vector<double> bj, nrm;        // [E][Nfn], [E][dim][Nfn]
  std::vector<int32_t> nbr_e, nbr_f;  // [E][Nfn]
  std::vector<double> xvol;           // [E][Nq][dim]
  std::vector<double> minv;           // [E][Np][Np] V^T (W/J) V (when ref.dense_minv)
  std::vector<double> sdir;           // [E][dim][n(n-1)][dim][T] skew-form line-pair coefficients
  std::vector<double> gvol;           // [E][dim*dim][Nq] metric terms G_lm (component l*dim+m)
  std::vector<double> jnf;            // [E][dim][Nfn] G^T nhat at the facet nodes (J^zeta n)
};

// which mesh-static pair tables build_host_mesh computes
constexpr int kTablesEntropyStable = 1;   // vdir, fdir (the entropy-stable residual)
constexpr int kTablesSkew = 2;            // sdir (the skew-symmetric form, skew.cuh)
constexpr int kTablesMetrics = 4;         // gvol, jnf (pair directions formed on the fly)

esd_status build_ref(int dim, int p, RefTables* out, std::string* err);
// n_ghost > 0: a partition mesh whose last n_ghost elements are ghosts (esd_part_create):
// geometry for all, facet matching and the returned tables for the local elements only
esd_status build_host_mesh(const esd_mesh_desc& d, HostMesh* out, std::string* err,
                           int tables = kTablesEntropyStable, int64_t n_ghost = 0);

// Device views passed to kernels by value.
// Tables of the table-driven logarithm and exponential (device.cuh: log_tab, exp_tab),
// laid out in one array of doubles:
//   [0,129) 1/F_j, [129,258) ln F_j (high part), [258,387) ln F_j (low part), F_j = 1 + j/128;
//   [387,419) 2^(j/32) (high), [419,451) 2^(j/32) (low);
//   [451] ln2 high, [452] ln2 low, [453] (ln2/32) high, [454] (ln2/32) low, [455] 32/ln2.
constexpr int kMathTabSize = 456;
void build_math_table(double* out);   // setup.cpp, host long double

struct DevRef {
  int dim, p, n, Nq, Np, Nf, Nqf, Nfn, Ntot, T, Lv, S12, nvp, nfp;
  int fph_off[4], fph_len[4];
  const double *psi1, *psi2, *psi3;
  const int *off1, *s12a1, *moff, *mode, *s12len;
  const double *l1m, *l1p, *l2m, *l3m, *L2J;
  const double* wvol;
  int dense_minv;
  const double* mtab;   // kMathTabSize doubles
  // pair directions formed on the fly (meshes created with ESD_MESH_METRICS_ON_THE_FLY)
  const double* aw;     // [dim (family k)][dim (l)][Nq]: w_v (d eta_k / d xi_l)(xi_v)
  const double* dk4;    // [dim][n*n]: dl[k][a*n+b] / 4
  const double* wfac;   // [Nfn] facet quadrature weights
  double nhat[4][3];    // reference facet normals
};

// bits of DevMesh::flag (read and cleared by esd_mesh_check)
constexpr int kFlagState = 1;     // a non-admissible state (rho <= 0, p <= 0, non-finite)
constexpr int kFlagTimeout = 2;   // a shared-memory staging copy did not complete in time
constexpr int kFlagIndex = 4;     // a trace export named an element outside the partition

struct DevMesh {
  int64_t E;
  const double *vdir, *fdir, *wj, *wdj, *bj, *nrm;
  const double* minv;   // [E][Np][Np] weight-adjusted inverse (symmetric), or null
  const int32_t *nbr_e, *nbr_f;
  double* states;   // [E][nfields][Ntot]
  double* cfac;     // [E][Nfn] sound speed at facet nodes
  int* flag;        // admissibility flag
  double gamma;
  int lf;
  const double* gvol;   // [E][dim*dim][Nq] metric terms, when directions are formed on the fly
  const double* jnf;    // [E][dim][Nfn] J^zeta n at the facet nodes (same)
};

struct LaunchCfg {
  int ea = 1, ta = 128;  size_t sa = 0;   // projection kernel: elements/CTA, threads, smem bytes
  int eb = 1, tb = 128;  size_t sb = 0;   // residual kernel
  int ev = 1, tv = 128;  size_t sv = 0;   // residual adjoint kernel
  int eq = 1, tq = 128;  size_t sq = 0;   // projection adjoint kernel (projection-sized tiles)
};

// RK epilogue of the residual kernel: acc_out = acc_in + cb*k, stage_out = u0 + ca*k.
struct Epilogue {
  int mode;                 // 0: store dudt; 1: RK stage update; 2: diagnostics partials
  double* dudt;
  const double* u0;
  const double* acc_in;
  double* acc_out;
  double* stage_out;
  double ca, cb;
  double* diag;             // [E][nc+2] partial sums (mode 2)
};

// batched execution: one entry per mesh, one per (mesh, element tile)
struct BatchMesh {
  DevRef R;
  DevMesh M;
  const double* u;   // stage input for the projection
  Epilogue ep;       // residual epilogue (RK update)
};
struct BatchItem {
  int mesh;
  int E;
  int64_t e0;
};

LaunchCfg choose_launch(const RefTables& r);
bool audit_layouts(std::string* err);   // kernels.cu, host only
size_t smem_project(const RefTables& r, int e);
size_t smem_residual(const RefTables& r, int e);
size_t smem_residual_adj(const RefTables& r, int e);
int adj_threads_host(const RefTables& r, int e);   // threads of a residual-adjoint CTA of e elements

// Kernel launchers (kernels.cu).  All return cudaGetLastError().
cudaError_t launch_project(const DevRef& R, const DevMesh& M, const LaunchCfg& L, const double* u,
                           double* w_modal, cudaStream_t s);
cudaError_t launch_residual(const DevRef& R, const DevMesh& M, const LaunchCfg& L, const Epilogue& ep,
                            cudaStream_t s);
cudaError_t launch_l2_project(const DevRef& R, const DevMesh& M, const double* un, double* um,
                              cudaStream_t s);
// project_first = false: M.states / M.cfac already hold the entropy projection of u
// (a tape saved by the forward call), so the projection kernel is not launched again
cudaError_t launch_vjp(const DevRef& R, const DevMesh& M, const LaunchCfg& L, const double* u, const double* cot,
                       double* grad, double* qbar, double* qext, cudaStream_t s, bool project_first = true);
// threads per line task of the residual kernel: 2 for tetrahedra with N = p + 1 >= 8
// (device.cuh: kLineLanes, line_task_split), else 1; a residual block needs
// residual_threads(dim, n, T, e) threads for e elements of T line tasks each
inline int residual_line_lanes(int dim, int n) { return dim == 3 && n >= 8 ? 2 : 1; }
inline int residual_threads(int dim, int n, int T, int e) {
  const int w = (residual_line_lanes(dim, n) * e * T + 31) / 32 * 32;
  return w > 64 ? w : 64;
}
cudaError_t launch_residual_adjoint(const DevRef& R, const DevMesh& M, const LaunchCfg& L, const double* cot,
                                    double* qbar, double* qext, cudaStream_t s);
cudaError_t launch_project_adjoint(const DevRef& R, const DevMesh& M, const LaunchCfg& L, const double* u,
                                   const double* qbar, const double* qext, double* grad, cudaStream_t s);
// partition trace messages (kind 0: states and sound speeds; kind 1: interface cotangents)
cudaError_t launch_trace_export(const DevRef& R, const DevMesh& M, const double* qext, int kind,
                                const int64_t* elems, int64_t n, double* buf, cudaStream_t s);
cudaError_t launch_trace_import(const DevRef& R, const DevMesh& M, double* qext, int kind, const double* buf,
                                int64_t first, int64_t n, cudaStream_t s);
cudaError_t launch_axpby(double* out, double a, const double* x, double b, const double* y, int64_t n,
                         cudaStream_t s);
cudaError_t launch_batch(int dim, int n, int stage, const BatchMesh* meshes, const BatchItem* items, int nitems,
                         int grid, int threads, size_t smem, cudaStream_t s);
// per-dimension residual instantiations (residual_d2.cu, residual_d3.cu)
cudaError_t launch_residual_d2(const DevRef& R, const DevMesh& M, const LaunchCfg& L, const Epilogue& ep,
                               cudaStream_t s);
cudaError_t launch_residual_d3(const DevRef& R, const DevMesh& M, const LaunchCfg& L, const Epilogue& ep,
                               cudaStream_t s);
cudaError_t launch_residual_batch_d2(int n, const BatchMesh* meshes, const BatchItem* items, int nitems, int grid,
                                     int threads, size_t smem, cudaStream_t s);
cudaError_t launch_residual_batch_d3(int n, const BatchMesh* meshes, const BatchItem* items, int nitems, int grid,
                                     int threads, size_t smem, cudaStream_t s);
cudaError_t set_residual_smem_d2(int lim);
cudaError_t set_residual_smem_d3(int lim);
// tetrahedra of degree 7..10 (residual_d3_hi.cu); reached through the *_d3 entry points
cudaError_t launch_residual_d3_hi(const DevRef& R, const DevMesh& M, const LaunchCfg& L, const Epilogue& ep,
                                  cudaStream_t s);
cudaError_t launch_residual_batch_d3_hi(int n, const BatchMesh* meshes, const BatchItem* items, int nitems,
                                        int grid, int threads, size_t smem, cudaStream_t s);
cudaError_t set_residual_smem_d3_hi(int lim);
// pair directions formed on the fly (residual_otf_d2.cu, residual_otf_d3.cu)
cudaError_t launch_residual_otf_d2(const DevRef& R, const DevMesh& M, const LaunchCfg& L, const Epilogue& ep,
                                   cudaStream_t s);
cudaError_t launch_residual_otf_d3(const DevRef& R, const DevMesh& M, const LaunchCfg& L, const Epilogue& ep,
                                   cudaStream_t s);
cudaError_t set_residual_otf_smem_d2(int lim);
cudaError_t set_residual_otf_smem_d3(int lim);
cudaError_t launch_reduce_diag(const double* part, int64_t E, int ncol, double* out, cudaStream_t s);
cudaError_t launch_integrals(const DevRef& R, const DevMesh& M, const LaunchCfg& L, const double* u, double* part,
                             cudaStream_t s);
cudaError_t launch_copy(const double* src, double* dst, int64_t n, cudaStream_t s);
cudaError_t measure_fp64(double* flops, cudaStream_t s);
cudaError_t launch_staging_timeout_probe(int* flag, double seconds, cudaStream_t s);
cudaError_t launch_math_probe(int which, const double* mtab, const double* x, double* y, int64_t n, cudaStream_t s);
cudaError_t set_smem_limits(const LaunchCfg& L, int dim);

// skew-symmetric form (skew.cuh; skew_d2.cu, skew_d3.cu, skew_d3_hi.cu)
struct SkewModel;
cudaError_t launch_skew_residual_d2(int n, int nc, const DevRef& R, const DevMesh& M, const SkewModel& P,
                                    const double* sdir, int epc, int threads, size_t smem, const double* u,
                                    double* dudt, cudaStream_t s);
cudaError_t launch_skew_residual_d3(int n, int nc, const DevRef& R, const DevMesh& M, const SkewModel& P,
                                    const double* sdir, int epc, int threads, size_t smem, const double* u,
                                    double* dudt, cudaStream_t s);
cudaError_t skew_residual_attrs_d2(int n, int nc, int smem_limit, int* regs, int* max_threads);
cudaError_t skew_residual_attrs_d3(int n, int nc, int smem_limit, int* regs, int* max_threads);
cudaError_t launch_skew_trace_d2(int nc, const DevRef& R, const DevMesh& M, const SkewModel& P, int epc,
                                 int threads, size_t smem, const double* u, cudaStream_t s);
cudaError_t launch_skew_trace_d3(int nc, const DevRef& R, const DevMesh& M, const SkewModel& P, int epc,
                                 int threads, size_t smem, const double* u, cudaStream_t s);
cudaError_t skew_trace_attrs_d2(int smem_limit);
cudaError_t skew_trace_attrs_d3(int smem_limit);

}  // namespace esd
