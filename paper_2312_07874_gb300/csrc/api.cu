// C ABI of the library (declared in include/esd.h): argument checking, device
// allocation at mesh creation, launch sequencing, and CUDA-graph replay of RK4.
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <functional>
#include <mutex>
#include <string>
#include <vector>

#include "esd_internal.h"
#include "skew.cuh"

// NVTX ranges name each entry point's host-side span (enqueue, capture or graph launch) for
// profilers (e.g. ncu --nvtx --nvtx-include "esd_rhs/").  Header-only NVTX 3: without an
// attached tool the calls return at once.  Built without it if the header is absent.
#if __has_include(<nvtx3/nvToolsExt.h>)
#include <nvtx3/nvToolsExt.h>
namespace {
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};
}  // namespace
#define ESD_RANGE(name) NvtxRange esd_nvtx_range_(name)
#else
#define ESD_RANGE(name) ((void)0)
#endif

using namespace esd;

namespace {
thread_local std::string g_err;

esd_status fail(esd_status s, const std::string& msg) {
  g_err = msg;
  return s;
}

esd_status cuda_fail(cudaError_t e, const char* where) {
  return fail(ESD_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

esd_status check_dev(const void* p, const char* name) {
  if (!is_device_ptr(p)) return fail(ESD_ERR_ARG, std::string(name) + " is not a device pointer");
  if (reinterpret_cast<uintptr_t>(p) % 8 != 0) return fail(ESD_ERR_ARG, std::string(name) + " is not 8-byte aligned");
  return ESD_OK;
}

// Every device-side call on a mesh must run with the mesh's own device current: its
// tables and workspace live there, and a launch on another device would read them
// through peer mappings (or fault).  Checked before anything is enqueued.
esd_status check_device(int mesh_device) {
  int cur = -1;
  cudaError_t e = cudaGetDevice(&cur);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (cur != mesh_device)
    return fail(ESD_ERR_ARG, "the mesh was created on device " + std::to_string(mesh_device) + " but device " +
                                 std::to_string(cur) + " is current");
  return ESD_OK;
}
}  // namespace

// Captured RK4 (and batch) graphs kept per handle; the oldest is dropped beyond this.
constexpr size_t kMaxCachedGraphs = 16;

struct GraphEntry {
  double* u;
  double dt;
  double* ckpt;
  double* tapes;   // esd_rk_step_save: the four stages' forward tapes (else null)
  cudaStream_t s;
  cudaGraphExec_t exec;
};

struct esd_mesh_s {
  int dim = 0, p = 0, nc = 0;
  int device = -1;             // the device current at esd_mesh_create; it owns every allocation
  int64_t E = 0;
  int64_t n_ghost = 0;         // partition meshes (esd_part_create): ghost elements after the E local ones
  RefTables ref;
  std::vector<double> xvol;
  DevRef R{};
  DevMesh M{};
  LaunchCfg L{};
  std::vector<void*> allocs;
  size_t bytes = 0;
  double* ws_acc = nullptr;
  double* ws_stage = nullptr;
  double* ws_diag = nullptr;
  double* ws_qbar = nullptr;   // VJP: per-node cotangents [E][nq][Ntot]
  double* ws_qext = nullptr;   // VJP: interface cotangents for the neighbour [E][nq][Nfn]
  double* ws_adj[4] = {nullptr, nullptr, nullptr, nullptr};  // RK adjoint: cot copy, k_b, y_b, acc
  double* sdir = nullptr;      // skew-symmetric form: line-pair coefficients (esd_skew_create)
  std::vector<GraphEntry> graphs;

  template <class T>
  esd_status alloc(T** p, size_t count) {
    void* q = nullptr;
    if (count == 0) count = 1;
    cudaError_t e = cudaMalloc(&q, count * sizeof(T));
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail(ESD_ERR_NOMEM, "cudaMalloc failed at mesh creation");
    }
    allocs.push_back(q);
    bytes += count * sizeof(T);
    *p = static_cast<T*>(q);
    return ESD_OK;
  }
  template <class T>
  esd_status upload(T** p, const std::vector<T>& h) {
    esd_status s = alloc(p, h.size());
    if (s != ESD_OK) return s;
    if (!h.empty()) {
      cudaError_t e = cudaMemcpy(*p, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice);
      if (e != cudaSuccess) return cuda_fail(e, "upload");
    }
    return ESD_OK;
  }
  ~esd_mesh_s() {
    for (auto& g : graphs) cudaGraphExecDestroy(g.exec);
    for (void* q : allocs) cudaFree(q);
  }
};

extern "C" {

const char* esd_status_string(esd_status s) {
  switch (s) {
    case ESD_OK: return "ESD_OK";
    case ESD_ERR_ARG: return "ESD_ERR_ARG: invalid argument";
    case ESD_ERR_MESH: return "ESD_ERR_MESH: invalid mesh";
    case ESD_ERR_CUDA: return "ESD_ERR_CUDA: CUDA runtime error";
    case ESD_ERR_STATE: return "ESD_ERR_STATE: non-admissible state";
    case ESD_ERR_TIMEOUT: return "ESD_ERR_TIMEOUT: bounded device wait gave up";
    case ESD_ERR_NOMEM: return "ESD_ERR_NOMEM: device allocation failed";
    case ESD_ERR_UNSUPPORTED: return "ESD_ERR_UNSUPPORTED: unsupported configuration";
  }
  return "unknown status";
}

const char* esd_last_error(void) { return g_err.c_str(); }

static esd_status mesh_create(const esd_mesh_desc* d, int tables, esd_mesh* out, int64_t n_ghost = 0);

esd_status esd_mesh_create(const esd_mesh_desc* d, esd_mesh* out) {
  ESD_RANGE("esd_mesh_create");
  return mesh_create(d, kTablesEntropyStable, out);
}

esd_status esd_mesh_create_ex(const esd_mesh_desc* d, int options, esd_mesh* out) {
  ESD_RANGE("esd_mesh_create_ex");
  if (options == ESD_MESH_PAIR_TABLES) return mesh_create(d, kTablesEntropyStable, out);
  if (options == ESD_MESH_METRICS_ON_THE_FLY) return mesh_create(d, kTablesMetrics, out);
  if (out) *out = nullptr;
  return fail(ESD_ERR_ARG, "options must be ESD_MESH_PAIR_TABLES or ESD_MESH_METRICS_ON_THE_FLY");
}

// Calls that evaluate a whole right-hand side in one go need every neighbour's trace; on a
// partition mesh the ghosts' traces arrive between the phases (esd_rhs_begin ... esd_rhs_end).
static esd_status reject_partition(const esd_mesh_s* m, const char* call) {
  if (m->n_ghost == 0) return ESD_OK;
  return fail(ESD_ERR_UNSUPPORTED, std::string(call) + " on a partition mesh: use esd_rhs_begin, esd_part_export / "
                                   "esd_part_import and esd_rhs_end (esd_rhs_vjp_mid / esd_rhs_vjp_end for the VJP)");
}

// Mesh creation with the chosen pair tables (entropy-stable pair directions, or the
// skew-symmetric form's line-pair coefficients for esd_skew_create).
static esd_status mesh_create(const esd_mesh_desc* d, int tables, esd_mesh* out, int64_t n_ghost) {
  if (!d || !out) return fail(ESD_ERR_ARG, "null descriptor or output");
  *out = nullptr;
  if (d->dim != 2 && d->dim != 3) return fail(ESD_ERR_ARG, "dim must be 2 or 3");
  if (d->n_elem <= 0 || d->n_elem > (int64_t)1 << 28) return fail(ESD_ERR_ARG, "n_elem out of range");
  if (!d->map_nodes || !d->nbr_elem || !d->nbr_face) return fail(ESD_ERR_ARG, "null mesh arrays");
  if (!(d->gamma > 1.0) || d->gamma > 10.0) return fail(ESD_ERR_ARG, "gamma must be in (1, 10]");
  if (d->flux != ESD_FLUX_EC && d->flux != ESD_FLUX_LF) return fail(ESD_ERR_ARG, "flux must be ESD_FLUX_EC or ESD_FLUX_LF");
  HostMesh H;
  std::string err;
  esd_status st = build_host_mesh(*d, &H, &err, tables, n_ghost);
  if (st != ESD_OK) return fail(st, err);
  int device = -1;
  cudaError_t de = cudaGetDevice(&device);
  if (de != cudaSuccess) return cuda_fail(de, "cudaGetDevice");
  esd_mesh m = new esd_mesh_s();
  m->device = device;
  m->dim = d->dim;
  m->p = d->p;
  m->nc = d->dim + 2;
  m->E = d->n_elem - n_ghost;
  m->n_ghost = n_ghost;
  m->ref = H.ref;
  m->xvol = std::move(H.xvol);
  const RefTables& r = m->ref;
  // reference tables
  std::vector<double> dt;
  auto push = [&](const std::vector<double>& v) {
    size_t o = dt.size();
    dt.insert(dt.end(), v.begin(), v.end());
    return o;
  };
  size_t o_psi1 = push(r.psi1), o_psi2 = push(r.psi2), o_psi3 = push(r.psi3), o_l1m = push(r.l1m),
         o_l1p = push(r.l1p), o_l2m = push(r.l2m), o_l3m = push(r.l3m), o_L2J = push(r.L2J), o_w = push(r.wvol);
  std::vector<double> mt(kMathTabSize);
  build_math_table(mt.data());
  size_t o_mt = push(mt);
  // on-the-fly pair directions: w_v d eta_k/d xi_l per family, D_k / 4, facet weights
  std::vector<double> aw((size_t)r.dim * r.dim * r.Nq), dk4((size_t)r.dim * r.n * r.n);
  for (int k = 0; k < r.dim; ++k) {
    for (int l = 0; l < r.dim; ++l)
      for (int v = 0; v < r.Nq; ++v) aw[((size_t)k * r.dim + l) * r.Nq + v] = r.wvol[v] * r.deta[v * 9 + k * 3 + l];
    for (int ab = 0; ab < r.n * r.n; ++ab) dk4[(size_t)k * r.n * r.n + ab] = 0.25 * r.dl[k][ab];
  }
  size_t o_aw = push(aw), o_dk4 = push(dk4), o_wfac = push(r.wfac);
  double* dtab = nullptr;
  int* itab = nullptr;
  if ((st = m->upload(&dtab, dt)) != ESD_OK || (st = m->upload(&itab, r.ints)) != ESD_OK) {
    delete m;
    return st;
  }
  DevRef& R = m->R;
  R.dim = r.dim; R.p = r.p; R.n = r.n; R.Nq = r.Nq; R.Np = r.Np; R.Nf = r.Nf; R.Nqf = r.Nqf; R.Nfn = r.Nfn;
  R.Ntot = r.Ntot; R.T = r.T; R.Lv = r.Lv; R.S12 = r.S12; R.nvp = r.nvp; R.nfp = r.nfp;
  for (int i = 0; i < 4; ++i) { R.fph_off[i] = r.fph_off[i]; R.fph_len[i] = r.fph_len[i]; }
  R.psi1 = dtab + o_psi1; R.psi2 = dtab + o_psi2; R.psi3 = dtab + o_psi3;
  R.l1m = dtab + o_l1m; R.l1p = dtab + o_l1p; R.l2m = dtab + o_l2m; R.l3m = dtab + o_l3m; R.L2J = dtab + o_L2J;
  R.wvol = dtab + o_w;
  R.dense_minv = r.dense_minv;
  R.mtab = dtab + o_mt;
  R.aw = dtab + o_aw;
  R.dk4 = dtab + o_dk4;
  R.wfac = dtab + o_wfac;
  for (int z = 0; z < 4; ++z)
    for (int l = 0; l < 3; ++l) R.nhat[z][l] = r.nhat[z][l];
  R.off1 = itab + r.i_off1; R.s12a1 = itab + r.i_s12a1; R.moff = itab + r.i_moff; R.mode = itab + r.i_mode;
  R.s12len = itab + r.i_s12len;
  // per-element data
  DevMesh& M = m->M;
  M.E = m->E;
  M.gamma = d->gamma;
  M.lf = d->flux == ESD_FLUX_LF;
  double *vdir, *fdir, *wj, *wdj, *bj, *nrm;
  int32_t *ne, *nf;
  if ((st = m->upload(&vdir, H.vdir)) || (st = m->upload(&fdir, H.fdir)) || (st = m->upload(&wj, H.wj)) ||
      (st = m->upload(&wdj, H.wdj)) || (st = m->upload(&bj, H.bj)) || (st = m->upload(&nrm, H.nrm)) ||
      (st = m->upload(&ne, H.nbr_e)) || (st = m->upload(&nf, H.nbr_f))) {
    delete m;
    return st;
  }
  M.vdir = vdir; M.fdir = fdir; M.wj = wj; M.wdj = wdj; M.bj = bj; M.nrm = nrm; M.nbr_e = ne; M.nbr_f = nf;
  if ((tables & kTablesSkew) && (st = m->upload(&m->sdir, H.sdir))) {
    delete m;
    return st;
  }
  M.gvol = M.jnf = nullptr;
  if (tables & kTablesMetrics) {
    double *gv = nullptr, *jn = nullptr;
    if ((st = m->upload(&gv, H.gvol)) || (st = m->upload(&jn, H.jnf))) {
      delete m;
      return st;
    }
    M.gvol = gv;
    M.jnf = jn;
  }
  M.minv = nullptr;
  if (r.dense_minv) {
    double* mi = nullptr;
    if ((st = m->upload(&mi, H.minv))) {
      delete m;
      return st;
    }
    M.minv = mi;
  }
  // per-node states and facet sound speeds: rows for the local elements, then (partition
  // meshes) the ghosts' rows, written by esd_part_import
  const int64_t Erow = m->E + n_ghost;
  const size_t nstate = (size_t)Erow * nfields(r.dim) * r.Ntot;
  const size_t nmodal = (size_t)m->E * m->nc * r.Np;
  if ((st = m->alloc(&M.states, nstate)) || (st = m->alloc(&M.cfac, (size_t)Erow * r.Nfn)) ||
      (st = m->alloc(&M.flag, 1)) || (st = m->alloc(&m->ws_acc, nmodal)) || (st = m->alloc(&m->ws_stage, nmodal)) ||
      (st = m->alloc(&m->ws_diag, (size_t)m->E * (m->nc + 2)))) {
    delete m;
    return st;
  }
  // the VJP's workspaces, only where the VJP can run (meshes with the stored pair tables)
  if ((tables & kTablesEntropyStable) &&
      ((st = m->alloc(&m->ws_qbar, (size_t)m->E * m->nc * r.Ntot)) ||
       (st = m->alloc(&m->ws_qext, (size_t)Erow * m->nc * r.Nfn)) || (st = m->alloc(&m->ws_adj[0], nmodal)) ||
       (st = m->alloc(&m->ws_adj[1], nmodal)) || (st = m->alloc(&m->ws_adj[2], nmodal)) ||
       (st = m->alloc(&m->ws_adj[3], nmodal)))) {
    delete m;
    return st;
  }
  cudaMemset(M.flag, 0, sizeof(int));
  if (n_ghost > 0) {   // defined values in the ghost rows until the first import
    cudaMemset(M.states, 0, nstate * sizeof(double));
    cudaMemset(M.cfac, 0, (size_t)Erow * r.Nfn * sizeof(double));
    if (m->ws_qext) cudaMemset(m->ws_qext, 0, (size_t)Erow * m->nc * r.Nfn * sizeof(double));
  }
  m->L = choose_launch(r);
  cudaError_t e = set_smem_limits(m->L, r.dim);
  if (e != cudaSuccess) {
    delete m;
    return cuda_fail(e, "cudaFuncSetAttribute");
  }
  e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    delete m;
    return cuda_fail(e, "mesh upload");
  }
  *out = m;
  return ESD_OK;
}

esd_status esd_mesh_destroy(esd_mesh m) {
  if (!m) return fail(ESD_ERR_ARG, "null mesh");
  cudaDeviceSynchronize();
  delete m;
  return ESD_OK;
}

esd_status esd_mesh_info(esd_mesh m, esd_info* o) {
  if (!m || !o) return fail(ESD_ERR_ARG, "null argument");
  const RefTables& r = m->ref;
  o->dim = r.dim; o->p = r.p; o->n_c = m->nc; o->n_modes = r.Np; o->n_vol_nodes = r.Nq;
  o->n_facets = r.Nf; o->n_facet_nodes = r.Nqf; o->n_elem = m->E;
  o->vol_pairs_per_elem = r.nvp;
  o->facet_pairs_per_elem = r.nfp;
  const int64_t q = r.p, n = q + 1;
  o->paper_flux_count_per_elem = r.dim == 2 ? (q * n * n) / 2 + q * n * n + 3 * n * n
                                            : 3 * q * n * n * n + 3 * n * n * n + n * n * n * n;
  o->device_bytes = m->bytes;
  o->elems_per_cta_project = m->L.ea;
  o->elems_per_cta_residual = m->L.eb;
  return ESD_OK;
}

esd_status esd_mesh_check(esd_mesh m, void* stream) {
  if (!m) return fail(ESD_ERR_ARG, "null mesh");
  if (esd_status ds = check_device(m->device)) return ds;
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "stream synchronize");
  int flag = 0;
  e = cudaMemcpy(&flag, m->M.flag, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "flag read");
  if (flag) {
    cudaMemset(m->M.flag, 0, sizeof(int));
    if (flag & kFlagTimeout)
      return fail(ESD_ERR_TIMEOUT, "a shared-memory staging copy did not complete within its time limit");
    if (flag & kFlagIndex)
      return fail(ESD_ERR_ARG, "esd_part_export: an element index is outside [0, n_elem) (zeros were sent)");
    return fail(ESD_ERR_STATE, "non-admissible state (rho <= 0, p <= 0 or non-finite) at a quadrature node");
  }
  return ESD_OK;
}

esd_status esd_debug_staging_timeout(esd_mesh m, double seconds, void* stream) {
  if (!m) return fail(ESD_ERR_ARG, "null mesh");
  if (esd_status ds = check_device(m->device)) return ds;
  if (!(seconds > 0.0) || seconds > 10.0) return fail(ESD_ERR_ARG, "seconds must be in (0, 10]");
  cudaError_t e = launch_staging_timeout_probe(m->M.flag, seconds, (cudaStream_t)stream);
  return e ? cuda_fail(e, "timeout probe launch") : ESD_OK;
}

esd_status esd_debug_set_mesh_device(esd_mesh m, int device) {
  if (!m) return fail(ESD_ERR_ARG, "null mesh");
  m->device = device;
  return ESD_OK;
}

esd_status esd_mesh_volume_nodes(esd_mesh m, double* x) {
  if (!m || !x) return fail(ESD_ERR_ARG, "null argument");
  std::memcpy(x, m->xvol.data(), m->xvol.size() * sizeof(double));
  return ESD_OK;
}

esd_status esd_l2_project(esd_mesh m, const double* un, double* um, void* stream) {
  ESD_RANGE("esd_l2_project");
  if (!m) return fail(ESD_ERR_ARG, "null mesh");
  if (esd_status ds = check_device(m->device)) return ds;
  esd_status st;
  if ((st = check_dev(un, "u_nodal")) || (st = check_dev(um, "u_modal"))) return st;
  cudaError_t e = launch_l2_project(m->R, m->M, un, um, (cudaStream_t)stream);
  return e ? cuda_fail(e, "l2_project launch") : ESD_OK;
}

esd_status esd_project_entropy(esd_mesh m, const double* u, double* w, void* stream) {
  ESD_RANGE("esd_project_entropy");
  if (!m) return fail(ESD_ERR_ARG, "null mesh");
  if (esd_status ds = check_device(m->device)) return ds;
  esd_status st;
  if ((st = check_dev(u, "u")) || (st = check_dev(w, "w_modal"))) return st;
  cudaError_t e = launch_project(m->R, m->M, m->L, u, w, (cudaStream_t)stream);
  return e ? cuda_fail(e, "project launch") : ESD_OK;
}

esd_status esd_rhs(esd_mesh m, const double* u, double* dudt, void* stream) {
  ESD_RANGE("esd_rhs");
  if (!m) return fail(ESD_ERR_ARG, "null mesh");
  if (esd_status ds = check_device(m->device)) return ds;
  if (esd_status ps = reject_partition(m, "esd_rhs")) return ps;
  esd_status st;
  if ((st = check_dev(u, "u")) || (st = check_dev(dudt, "dudt"))) return st;
  if (u == dudt) return fail(ESD_ERR_ARG, "u and dudt must not alias");
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = launch_project(m->R, m->M, m->L, u, nullptr, s);
  if (e) return cuda_fail(e, "project launch");
  Epilogue ep{};
  ep.mode = 0;
  ep.dudt = dudt;
  e = launch_residual(m->R, m->M, m->L, ep, s);
  return e ? cuda_fail(e, "residual launch") : ESD_OK;
}

// Forward tape (esd_rhs_save, esd_rk_step_save): the entropy-projected states with their
// derived fields, [E][nfields][Ntot], padded to a multiple of 32 doubles (256 bytes), then
// the facet sound speeds [E][Nfn], padded the same way: what the projection kernel writes and the residual kernel
// and the VJP kernels read.
static size_t tape_states_doubles(const esd_mesh_s* m) {
  return ((size_t)m->E * nfields(m->dim) * m->ref.Ntot + 31) / 32 * 32;
}
static size_t tape_doubles(const esd_mesh_s* m) {   // a multiple of 32: stage tapes stay aligned
  return tape_states_doubles(m) + ((size_t)m->E * m->ref.Nfn + 31) / 32 * 32;
}
static DevMesh on_tape(const esd_mesh_s* m, const double* tape) {
  DevMesh M = m->M;
  M.states = const_cast<double*>(tape);   // read-only for the VJP kernels
  M.cfac = const_cast<double*>(tape) + tape_states_doubles(m);
  return M;
}
// the residual kernel stages each element's states with a bulk copy: 16-byte alignment
static esd_status check_tape(const void* t, const char* name) {
  if (esd_status st = check_dev(t, name)) return st;
  if (reinterpret_cast<uintptr_t>(t) % 16 != 0) return fail(ESD_ERR_ARG, std::string(name) + " is not 16-byte aligned");
  return ESD_OK;
}

esd_status esd_tape_doubles(esd_mesh m, int64_t* n_doubles) {
  if (!m || !n_doubles) return fail(ESD_ERR_ARG, "null argument");
  *n_doubles = (int64_t)tape_doubles(m);
  return ESD_OK;
}

esd_status esd_rhs_save(esd_mesh m, const double* u, double* dudt, double* tape, void* stream) {
  ESD_RANGE("esd_rhs_save");
  if (!m) return fail(ESD_ERR_ARG, "null mesh");
  if (esd_status ds = check_device(m->device)) return ds;
  if (esd_status ps = reject_partition(m, "esd_rhs_save")) return ps;
  if (m->M.gvol) return fail(ESD_ERR_UNSUPPORTED, "the VJP needs the stored pair tables (esd_mesh_create)");
  esd_status st;
  if ((st = check_dev(u, "u")) || (st = check_dev(dudt, "dudt")) || (st = check_tape(tape, "tape"))) return st;
  if (u == dudt) return fail(ESD_ERR_ARG, "u and dudt must not alias");
  cudaStream_t s = (cudaStream_t)stream;
  const DevMesh M = on_tape(m, tape);
  cudaError_t e = launch_project(m->R, M, m->L, u, nullptr, s);
  if (e) return cuda_fail(e, "project launch");
  Epilogue ep{};
  ep.mode = 0;
  ep.dudt = dudt;
  e = launch_residual(m->R, M, m->L, ep, s);
  return e ? cuda_fail(e, "residual launch") : ESD_OK;
}

static cudaError_t rk_sequence(esd_mesh m, double* u, double dt, double* ck, double* tapes, cudaStream_t s) {
  const size_t nmodal = (size_t)m->E * m->nc * m->ref.Np;
  cudaError_t e;
  if (ck && (e = launch_copy(u, ck, (int64_t)nmodal, s))) return e;
  const double a[4] = {0.5, 0.5, 1.0, 0.0};
  const double b[4] = {1.0 / 6.0, 1.0 / 3.0, 1.0 / 3.0, 1.0 / 6.0};
  const double* in = u;
  for (int st = 0; st < 4; ++st) {
    const DevMesh M = tapes ? on_tape(m, tapes + st * tape_doubles(m)) : m->M;
    if ((e = launch_project(m->R, M, m->L, in, nullptr, s))) return e;
    Epilogue ep{};
    ep.mode = 1;
    ep.u0 = u;
    ep.acc_in = st == 0 ? u : m->ws_acc;
    ep.acc_out = st == 3 ? u : m->ws_acc;
    ep.stage_out = st == 3 ? nullptr : (ck ? ck + (size_t)(st + 1) * nmodal : m->ws_stage);
    ep.ca = a[st] * dt;
    ep.cb = b[st] * dt;
    if ((e = launch_residual(m->R, M, m->L, ep, s))) return e;
    in = ep.stage_out;
  }
  return cudaSuccess;
}

static esd_status rk_step(esd_mesh m, double* u, double dt, double* ck, double* tapes, void* stream) {
  if (!m) return fail(ESD_ERR_ARG, "null mesh");
  if (esd_status ds = check_device(m->device)) return ds;
  if (esd_status ps = reject_partition(m, "esd_rk_step")) return ps;
  esd_status st;
  if ((st = check_dev(u, "u"))) return st;
  if (ck && (st = check_dev(ck, "stage_ckpt"))) return st;
  if (tapes && (st = check_tape(tapes, "tapes"))) return st;
  if (!(dt == dt) || dt <= 0.0) return fail(ESD_ERR_ARG, "dt must be positive");
  cudaStream_t s = (cudaStream_t)stream;
  if (s == nullptr) {  // the legacy stream cannot be captured: launch directly
    cudaError_t e = rk_sequence(m, u, dt, ck, tapes, s);
    return e ? cuda_fail(e, "rk launch") : ESD_OK;
  }
  for (auto& g : m->graphs)
    if (g.u == u && g.dt == dt && g.ckpt == ck && g.tapes == tapes && g.s == s) {
      cudaError_t e = cudaGraphLaunch(g.exec, s);
      return e ? cuda_fail(e, "graph launch") : ESD_OK;
    }
  cudaGraph_t graph;
  cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
  if (e) return cuda_fail(e, "begin capture");
  cudaError_t e1 = rk_sequence(m, u, dt, ck, tapes, s);
  e = cudaStreamEndCapture(s, &graph);
  if (e1 || e) {
    if (!e) cudaGraphDestroy(graph);
    return e1 ? cuda_fail(e1, "rk capture") : cuda_fail(e, "end capture");
  }
  cudaGraphExec_t exec;
  e = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e) return cuda_fail(e, "graph instantiate");
  if (m->graphs.size() >= kMaxCachedGraphs) {
    cudaGraphExecDestroy(m->graphs.front().exec);   // an in-flight launch completes first
    m->graphs.erase(m->graphs.begin());
  }
  m->graphs.push_back({u, dt, ck, tapes, s, exec});
  e = cudaGraphLaunch(exec, s);
  return e ? cuda_fail(e, "graph launch") : ESD_OK;
}

esd_status esd_rk_step(esd_mesh m, double* u, double dt, double* ck, void* stream) {
  ESD_RANGE("esd_rk_step");
  return rk_step(m, u, dt, ck, nullptr, stream);
}

esd_status esd_rk_step_save(esd_mesh m, double* u, double dt, double* ck, double* tapes, void* stream) {
  ESD_RANGE("esd_rk_step_save");
  if (!m) return fail(ESD_ERR_ARG, "null mesh");
  if (!ck || !tapes) return fail(ESD_ERR_ARG, "esd_rk_step_save needs stage_ckpt and tapes");
  if (m->M.gvol) return fail(ESD_ERR_UNSUPPORTED, "the VJP needs the stored pair tables (esd_mesh_create)");
  return rk_step(m, u, dt, ck, tapes, stream);
}

esd_status esd_diagnostics(esd_mesh m, const double* u, double* out, void* stream) {
  ESD_RANGE("esd_diagnostics");
  if (!m) return fail(ESD_ERR_ARG, "null mesh");
  if (esd_status ds = check_device(m->device)) return ds;
  if (esd_status ps = reject_partition(m, "esd_diagnostics")) return ps;
  esd_status st;
  if ((st = check_dev(u, "u")) || (st = check_dev(out, "out"))) return st;
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = launch_project(m->R, m->M, m->L, u, nullptr, s);
  if (e) return cuda_fail(e, "project launch");
  Epilogue ep{};
  ep.mode = 2;
  ep.diag = m->ws_diag;
  if ((e = launch_residual(m->R, m->M, m->L, ep, s))) return cuda_fail(e, "residual launch");
  e = launch_reduce_diag(m->ws_diag, m->E, m->nc + 2, out, s);
  return e ? cuda_fail(e, "reduce launch") : ESD_OK;
}

esd_status esd_integrals(esd_mesh m, const double* u, double* out, void* stream) {
  ESD_RANGE("esd_integrals");
  if (!m) return fail(ESD_ERR_ARG, "null mesh");
  if (esd_status ds = check_device(m->device)) return ds;
  esd_status st;
  if ((st = check_dev(u, "u")) || (st = check_dev(out, "out"))) return st;
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = launch_integrals(m->R, m->M, m->L, u, m->ws_diag, s);
  if (e) return cuda_fail(e, "integrals launch");
  e = launch_reduce_diag(m->ws_diag, m->E, m->nc + 1, out, s);
  return e ? cuda_fail(e, "reduce launch") : ESD_OK;
}

// tape: null (the projection of u is recomputed first) or the forward's saved tape of u
static esd_status rhs_vjp(esd_mesh m, const double* u, const double* tape, const double* cot, double* grad,
                          void* stream) {
  if (!m) return fail(ESD_ERR_ARG, "null mesh");
  if (esd_status ds = check_device(m->device)) return ds;
  if (esd_status ps = reject_partition(m, "esd_rhs_vjp")) return ps;
  if (m->M.gvol) return fail(ESD_ERR_UNSUPPORTED, "the VJP needs the stored pair tables (esd_mesh_create)");
  esd_status st;
  if ((st = check_dev(u, "u")) || (st = check_dev(cot, "cot")) || (st = check_dev(grad, "grad"))) return st;
  if (grad == u || grad == cot) return fail(ESD_ERR_ARG, "grad must not alias u or cot");
  if (tape && (st = check_tape(tape, "tape"))) return st;
  const DevMesh M = tape ? on_tape(m, tape) : m->M;
  cudaError_t e = launch_vjp(m->R, M, m->L, u, cot, grad, m->ws_qbar, m->ws_qext, (cudaStream_t)stream, !tape);
  return e ? cuda_fail(e, "vjp launch") : ESD_OK;
}

// Discrete adjoint of the RK4 step.  With stage inputs Y1..Y4 and k_s = F(Y_s):
//   u+ = u + dt/6 (k1 + 2k2 + 2k3 + k4),  Y2 = u + dt/2 k1,  Y3 = u + dt/2 k2,  Y4 = u + dt k3.
// Reverse: k4_b = dt/6 c;  Y4_b = J(Y4)^T k4_b;  k3_b = dt/3 c + dt Y4_b;  Y3_b = J(Y3)^T k3_b;
//          k2_b = dt/3 c + dt/2 Y3_b;  Y2_b = J(Y2)^T k2_b;  k1_b = dt/6 c + dt/2 Y2_b;
//          Y1_b = J(Y1)^T k1_b;  u_b = c + Y1_b + Y2_b + Y3_b + Y4_b.
// tapes: null (each stage's projection is recomputed) or the four stages' saved tapes
static esd_status rk_step_vjp(esd_mesh m, const double* ck, const double* tapes, double dt, const double* co,
                              double* ci, void* stream) {
  if (!m) return fail(ESD_ERR_ARG, "null mesh");
  if (esd_status ds = check_device(m->device)) return ds;
  if (esd_status ps = reject_partition(m, "esd_rk_step_vjp")) return ps;
  if (m->M.gvol) return fail(ESD_ERR_UNSUPPORTED, "the VJP needs the stored pair tables (esd_mesh_create)");
  esd_status st;
  if ((st = check_dev(ck, "stage_ckpt")) || (st = check_dev(co, "cot_out")) || (st = check_dev(ci, "cot_in")))
    return st;
  if (tapes && (st = check_tape(tapes, "tapes"))) return st;
  if (!(dt == dt) || dt <= 0.0) return fail(ESD_ERR_ARG, "dt must be positive");
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t nmodal = m->E * m->nc * m->ref.Np;
  double *c = m->ws_adj[0], *kb = m->ws_adj[1], *yb = m->ws_adj[2], *acc = m->ws_adj[3];
  const double ck_a[4] = {dt / 6.0, dt / 3.0, dt / 3.0, dt / 6.0};   // weight of c in k_s_b
  const double ck_b[4] = {0.0, dt, 0.5 * dt, 0.5 * dt};              // weight of the previous Y_b
  cudaError_t e;
  if ((e = launch_copy(co, c, nmodal, s)) || (e = launch_copy(co, acc, nmodal, s))) return cuda_fail(e, "rk vjp");
  for (int j = 0; j < 4; ++j) {
    const int stage = 3 - j;  // Y4, Y3, Y2, Y1
    if ((e = launch_axpby(kb, ck_a[j], c, ck_b[j], j ? yb : nullptr, nmodal, s))) return cuda_fail(e, "rk vjp");
    const DevMesh M = tapes ? on_tape(m, tapes + stage * tape_doubles(m)) : m->M;
    if ((e = launch_vjp(m->R, M, m->L, ck + (size_t)stage * nmodal, kb, yb, m->ws_qbar, m->ws_qext, s, !tapes)))
      return cuda_fail(e, "rk vjp");
    if ((e = launch_axpby(j == 3 ? ci : acc, 1.0, acc, 1.0, yb, nmodal, s))) return cuda_fail(e, "rk vjp");
  }
  return ESD_OK;
}

esd_status esd_rhs_vjp(esd_mesh m, const double* u, const double* cot, double* grad, void* stream) {
  ESD_RANGE("esd_rhs_vjp");
  return rhs_vjp(m, u, nullptr, cot, grad, stream);
}

esd_status esd_rhs_vjp_saved(esd_mesh m, const double* u, const double* tape, const double* cot, double* grad,
                             void* stream) {
  ESD_RANGE("esd_rhs_vjp_saved");
  if (!tape) return fail(ESD_ERR_ARG, "null tape");
  return rhs_vjp(m, u, tape, cot, grad, stream);
}

esd_status esd_rk_step_vjp(esd_mesh m, const double* ck, double dt, const double* co, double* ci, void* stream) {
  ESD_RANGE("esd_rk_step_vjp");
  return rk_step_vjp(m, ck, nullptr, dt, co, ci, stream);
}

esd_status esd_rk_step_vjp_saved(esd_mesh m, const double* ck, const double* tapes, double dt, const double* co,
                                 double* ci, void* stream) {
  ESD_RANGE("esd_rk_step_vjp_saved");
  if (!tapes) return fail(ESD_ERR_ARG, "null tapes");
  return rk_step_vjp(m, ck, tapes, dt, co, ci, stream);
}

// ---------------------------------------------------------------------------
// Element partitions: one facet-trace exchange per right-hand side (and one cotangent
// exchange per VJP) between the phases of the evaluation.
// ---------------------------------------------------------------------------
esd_status esd_part_create(const esd_mesh_desc* d, int64_t n_ghost, esd_mesh* out) {
  if (!d || !out) return fail(ESD_ERR_ARG, "null descriptor or output");
  if (n_ghost < 0 || n_ghost >= d->n_elem) return fail(ESD_ERR_ARG, "n_ghost must be in [0, n_elem)");
  return mesh_create(d, kTablesEntropyStable, out, n_ghost);
}

esd_status esd_part_info(esd_mesh m, int64_t* n_ghost, int64_t* trace_doubles, int64_t* cotangent_doubles) {
  if (!m) return fail(ESD_ERR_ARG, "null mesh");
  const int64_t Nfn = m->ref.Nfn;
  if (n_ghost) *n_ghost = m->n_ghost;
  if (trace_doubles) *trace_doubles = (nfields(m->dim) + 1) * Nfn;
  if (cotangent_doubles) *cotangent_doubles = m->nc * Nfn;
  return ESD_OK;
}

esd_status esd_rhs_begin(esd_mesh m, const double* u, void* stream) {
  ESD_RANGE("esd_rhs_begin");
  if (!m) return fail(ESD_ERR_ARG, "null mesh");
  if (esd_status ds = check_device(m->device)) return ds;
  if (esd_status st = check_dev(u, "u")) return st;
  cudaError_t e = launch_project(m->R, m->M, m->L, u, nullptr, (cudaStream_t)stream);
  return e ? cuda_fail(e, "project launch") : ESD_OK;
}

esd_status esd_rhs_end(esd_mesh m, double* dudt, void* stream) {
  ESD_RANGE("esd_rhs_end");
  if (!m) return fail(ESD_ERR_ARG, "null mesh");
  if (esd_status ds = check_device(m->device)) return ds;
  if (esd_status st = check_dev(dudt, "dudt")) return st;
  Epilogue ep{};
  ep.mode = 0;
  ep.dudt = dudt;
  cudaError_t e = launch_residual(m->R, m->M, m->L, ep, (cudaStream_t)stream);
  return e ? cuda_fail(e, "residual launch") : ESD_OK;
}

esd_status esd_rhs_vjp_mid(esd_mesh m, const double* cot, void* stream) {
  ESD_RANGE("esd_rhs_vjp_mid");
  if (!m) return fail(ESD_ERR_ARG, "null mesh");
  if (esd_status ds = check_device(m->device)) return ds;
  if (m->M.gvol || !m->ws_qbar) return fail(ESD_ERR_UNSUPPORTED, "the VJP needs the stored pair tables (esd_mesh_create)");
  if (esd_status st = check_dev(cot, "cot")) return st;
  cudaError_t e = launch_residual_adjoint(m->R, m->M, m->L, cot, m->ws_qbar, m->ws_qext, (cudaStream_t)stream);
  return e ? cuda_fail(e, "residual adjoint launch") : ESD_OK;
}

esd_status esd_rhs_vjp_end(esd_mesh m, const double* u, double* grad, void* stream) {
  ESD_RANGE("esd_rhs_vjp_end");
  if (!m) return fail(ESD_ERR_ARG, "null mesh");
  if (esd_status ds = check_device(m->device)) return ds;
  if (m->M.gvol || !m->ws_qbar) return fail(ESD_ERR_UNSUPPORTED, "the VJP needs the stored pair tables (esd_mesh_create)");
  esd_status st;
  if ((st = check_dev(u, "u")) || (st = check_dev(grad, "grad"))) return st;
  if (grad == u) return fail(ESD_ERR_ARG, "grad must not alias u");
  cudaError_t e = launch_project_adjoint(m->R, m->M, m->L, u, m->ws_qbar, m->ws_qext, grad, (cudaStream_t)stream);
  return e ? cuda_fail(e, "projection adjoint launch") : ESD_OK;
}

esd_status esd_part_export(esd_mesh m, int kind, const int64_t* elems, int64_t n, double* buf, void* stream) {
  ESD_RANGE("esd_part_export");
  if (!m) return fail(ESD_ERR_ARG, "null mesh");
  if (esd_status ds = check_device(m->device)) return ds;
  if (kind != ESD_TRACE_STATES && kind != ESD_TRACE_COTANGENTS) return fail(ESD_ERR_ARG, "unknown trace kind");
  if (kind == ESD_TRACE_COTANGENTS && !m->ws_qext) return fail(ESD_ERR_UNSUPPORTED, "this mesh has no VJP");
  if (n < 0) return fail(ESD_ERR_ARG, "n must be >= 0");
  if (n == 0) return ESD_OK;
  esd_status st;
  if ((st = check_dev(elems, "elems")) || (st = check_dev(buf, "buf"))) return st;
  cudaError_t e = launch_trace_export(m->R, m->M, m->ws_qext, kind, elems, n, buf, (cudaStream_t)stream);
  return e ? cuda_fail(e, "trace export launch") : ESD_OK;
}

esd_status esd_part_import(esd_mesh m, int kind, const double* buf, int64_t first, int64_t n, void* stream) {
  ESD_RANGE("esd_part_import");
  if (!m) return fail(ESD_ERR_ARG, "null mesh");
  if (esd_status ds = check_device(m->device)) return ds;
  if (kind != ESD_TRACE_STATES && kind != ESD_TRACE_COTANGENTS) return fail(ESD_ERR_ARG, "unknown trace kind");
  if (kind == ESD_TRACE_COTANGENTS && !m->ws_qext) return fail(ESD_ERR_UNSUPPORTED, "this mesh has no VJP");
  if (first < 0 || n < 0 || first + n > m->n_ghost) return fail(ESD_ERR_ARG, "ghost range outside [0, n_ghost)");
  if (n == 0) return ESD_OK;
  if (esd_status st = check_dev(buf, "buf")) return st;
  cudaError_t e = launch_trace_import(m->R, m->M, m->ws_qext, kind, buf, first, n, (cudaStream_t)stream);
  return e ? cuda_fail(e, "trace import launch") : ESD_OK;
}

// A mesh whose residual launch fills the GPU for at least this many waves on its own runs
// with its own launches inside the batch graph (see esd_batch_create); tests change it
// through esd_debug_batch_solo_waves.
static int g_batch_solo_waves = 1;

esd_status esd_debug_batch_solo_waves(int waves) {
  if (waves < 0) return fail(ESD_ERR_ARG, "waves must be >= 0");
  g_batch_solo_waves = waves;
  return ESD_OK;
}

struct BatchGroup {
  int dim = 0, p = 0;
  std::vector<int> members;          // indices into the batch's mesh list (persistent launches)
  std::vector<int> solo;             // large meshes of the group, launched on their own
  std::vector<BatchItem> pitems, ritems;
  BatchItem* d_pitems = nullptr;
  BatchItem* d_ritems = nullptr;
  int pthreads = 256, rthreads = 64;
  size_t psmem = 0, rsmem = 0;
  int pgrid = 1, rgrid = 1;
};

struct BatchGraph {
  std::vector<const double*> u;
  std::vector<double> dt;
  cudaStream_t s;
  int kind;   // 0: rhs, 1: rk step
  std::vector<BatchMesh*> d_tables;   // device BatchMesh arrays used by the graph (one per launch)
  cudaGraphExec_t exec = nullptr;
  // callers make sure no launch of the graph is still in flight
  void release() {
    if (exec) cudaGraphExecDestroy(exec);
    exec = nullptr;
    for (auto* p : d_tables) cudaFree(p);
    d_tables.clear();
  }
};

struct esd_batch_s {
  std::vector<esd_mesh> meshes;
  std::vector<BatchGroup> groups;
  std::vector<BatchGraph> graphs;
  std::vector<void*> allocs;
  ~esd_batch_s() {
    for (auto& g : graphs) g.release();
    for (void* p : allocs) cudaFree(p);
  }
};

static int sm_count() {
  int dev = 0, n = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
  return n > 0 ? n : 1;
}

esd_status esd_batch_create(const esd_mesh* meshes, int n, esd_batch* out) {
  if (!meshes || n <= 0 || !out) return fail(ESD_ERR_ARG, "invalid batch arguments");
  for (int i = 0; i < n; ++i)
    if (!meshes[i]) return fail(ESD_ERR_ARG, "null mesh in batch");
  for (int i = 0; i < n; ++i)
    if (esd_status ds = check_device(meshes[i]->device)) return ds;
  for (int i = 0; i < n; ++i)
    if (meshes[i]->M.gvol) return fail(ESD_ERR_UNSUPPORTED, "batches need meshes with stored pair tables");
  for (int i = 0; i < n; ++i)
    if (esd_status ps = reject_partition(meshes[i], "esd_batch_create")) return ps;
  esd_batch b = new esd_batch_s();
  b->meshes.assign(meshes, meshes + n);
  const int sms = sm_count();
  for (int key = 0; key < 2 * 16; ++key) {   // one group per (dimension, degree)
    const int dim = 2 + key / 16, deg = key % 16;
    BatchGroup g;
    g.dim = dim;
    g.p = deg;
    for (int i = 0; i < n; ++i) {
      if (meshes[i]->dim != dim || meshes[i]->p != deg) continue;
      esd_mesh m = meshes[i];
      // A mesh that fills the GPU for several waves gains nothing from the persistent
      // launch (its tail is a small part of its time) and loses to it: the persistent kernel
      // reads each mesh's tables through global memory, where a mesh's own launch has them
      // as kernel parameters.  Such meshes run their own launches in the group's branch.
      const int64_t ctas = (m->E + m->L.eb - 1) / m->L.eb;
      const int64_t per_sm = std::max<int64_t>(1, (int64_t)(227 * 1024) / (int64_t)std::max<size_t>(m->L.sb, 1));
      if (ctas >= (int64_t)g_batch_solo_waves * sms * per_sm) {
        g.solo.push_back(i);
        continue;
      }
      const int mi = (int)g.members.size();
      g.members.push_back(i);
      for (int64_t e0 = 0; e0 < m->E; e0 += m->L.ea)
        g.pitems.push_back({mi, (int)std::min<int64_t>(m->L.ea, m->E - e0), e0});
      for (int64_t e0 = 0; e0 < m->E; e0 += m->L.eb)
        g.ritems.push_back({mi, (int)std::min<int64_t>(m->L.eb, m->E - e0), e0});
      g.psmem = std::max(g.psmem, m->L.sa);
      g.rsmem = std::max(g.rsmem, m->L.sb);
      g.pthreads = std::max(g.pthreads, m->L.ta);
      g.rthreads = std::max(g.rthreads, m->L.tb);
    }
    if (g.members.empty() && g.solo.empty()) continue;
    if (g.members.empty()) {   // only large meshes: no persistent launch
      b->groups.push_back(g);
      continue;
    }
    // largest items first so that the persistent grid finishes evenly
    auto by_cost = [&](const BatchItem& x, const BatchItem& y) {
      const esd_mesh mx = meshes[g.members[x.mesh]], my = meshes[g.members[y.mesh]];
      return (double)x.E * mx->ref.Nq * mx->ref.n > (double)y.E * my->ref.Nq * my->ref.n;
    };
    std::stable_sort(g.pitems.begin(), g.pitems.end(), by_cost);
    std::stable_sort(g.ritems.begin(), g.ritems.end(), by_cost);
    const int per_sm_p = std::max(1, (int)(227 * 1024 / std::max<size_t>(g.psmem, 1)));
    const int per_sm_r = std::max(1, (int)(227 * 1024 / std::max<size_t>(g.rsmem, 1)));
    g.pgrid = std::min<int>((int)g.pitems.size(), sms * std::min(per_sm_p, 2048 / g.pthreads));
    g.rgrid = std::min<int>((int)g.ritems.size(), sms * std::min(per_sm_r, 2048 / g.rthreads));
    for (auto* items : {&g.pitems, &g.ritems}) {
      void* p = nullptr;
      if (cudaMalloc(&p, items->size() * sizeof(BatchItem)) != cudaSuccess) {
        delete b;
        return fail(ESD_ERR_NOMEM, "batch item list");
      }
      b->allocs.push_back(p);
      cudaMemcpy(p, items->data(), items->size() * sizeof(BatchItem), cudaMemcpyHostToDevice);
      (items == &g.pitems ? g.d_pitems : g.d_ritems) = static_cast<BatchItem*>(p);
    }
    b->groups.push_back(g);
  }
  cudaError_t e = cudaDeviceSynchronize();
  if (e) {
    delete b;
    return cuda_fail(e, "batch create");
  }
  *out = b;
  return ESD_OK;
}

esd_status esd_batch_destroy(esd_batch b) {
  if (!b) return fail(ESD_ERR_ARG, "null batch");
  cudaDeviceSynchronize();
  delete b;
  return ESD_OK;
}

// Enqueue (or capture) the batched launches.  kind 0: one d u~/dt per mesh; kind 1: one RK4 step.
static cudaError_t batch_sequence(esd_batch b, BatchGraph& G, cudaStream_t s) {
  const int nst = G.kind == 0 ? 1 : 4;
  const double ra[4] = {0.5, 0.5, 1.0, 0.0};
  const double rb[4] = {1.0 / 6.0, 1.0 / 3.0, 1.0 / 3.0, 1.0 / 6.0};
  cudaError_t e;
  for (int st = 0; st < nst; ++st) {
    for (auto& g : b->groups) {
      if (g.members.empty()) {   // no persistent launch in this group
        G.d_tables.push_back(nullptr);
        continue;
      }
      std::vector<BatchMesh> tab(g.members.size());
      for (size_t k = 0; k < g.members.size(); ++k) {
        const int i = g.members[k];
        esd_mesh m = b->meshes[i];
        BatchMesh& t = tab[k];
        t.R = m->R;
        t.M = m->M;
        double* u = const_cast<double*>(G.u[i]);
        if (G.kind == 0) {
          t.u = u;
          t.ep = Epilogue{};
          t.ep.mode = 0;
          t.ep.dudt = const_cast<double*>(G.u[b->meshes.size() + i]);
        } else {
          const double dt = G.dt[i];
          t.u = st == 0 ? u : m->ws_stage;
          t.ep = Epilogue{};
          t.ep.mode = 1;
          t.ep.u0 = u;
          t.ep.acc_in = st == 0 ? u : m->ws_acc;
          t.ep.acc_out = st == 3 ? u : m->ws_acc;
          t.ep.stage_out = st == 3 ? nullptr : m->ws_stage;
          t.ep.ca = ra[st] * dt;
          t.ep.cb = rb[st] * dt;
        }
      }
      void* p = nullptr;
      if ((e = cudaMalloc(&p, tab.size() * sizeof(BatchMesh)))) return e;
      G.d_tables.push_back(static_cast<BatchMesh*>(p));
      if ((e = cudaMemcpy(p, tab.data(), tab.size() * sizeof(BatchMesh), cudaMemcpyHostToDevice))) return e;
    }
  }
  return cudaSuccess;
}

static esd_status batch_run(esd_batch b, int kind, const std::vector<const double*>& ptrs, const std::vector<double>& dts,
                            cudaStream_t s) {
  for (auto& G : b->graphs)
    if (G.kind == kind && G.u == ptrs && G.dt == dts && G.s == s) {
      cudaError_t e = cudaGraphLaunch(G.exec, s);
      return e ? cuda_fail(e, "batch graph launch") : ESD_OK;
    }
  BatchGraph G;
  G.u = ptrs;
  G.dt = dts;
  G.s = s;
  G.kind = kind;
  cudaError_t e = batch_sequence(b, G, s);  // per-launch device tables (allocated outside capture)
  if (e) {
    G.release();
    return cuda_fail(e, "batch tables");
  }
  cudaStream_t cs = s;
  cudaStream_t own = nullptr;
  if (cs == nullptr) {  // the legacy stream cannot be captured: capture on a private stream
    cudaStreamCreateWithFlags(&own, cudaStreamNonBlocking);
    cs = own;
  }
  // The groups (one per dimension and degree) share no data: each group's stages form
  // one chain on its own forked stream, so the graph runs the groups concurrently and the
  // tail of one group's launch overlaps the work of the others.
  const size_t ng = b->groups.size();
  std::vector<cudaStream_t> gs(ng, nullptr);
  std::vector<cudaEvent_t> ev(ng + 1, nullptr);
  cudaError_t e1 = cudaSuccess;
  for (size_t gi = 0; gi < ng && !e1; ++gi) e1 = cudaStreamCreateWithFlags(&gs[gi], cudaStreamNonBlocking);
  for (size_t k = 0; k <= ng && !e1; ++k) e1 = cudaEventCreateWithFlags(&ev[k], cudaEventDisableTiming);
  auto release = [&] {
    for (auto x : gs)
      if (x) cudaStreamDestroy(x);
    for (auto x : ev)
      if (x) cudaEventDestroy(x);
    if (own) cudaStreamDestroy(own);
  };
  if (e1) {
    release();
    G.release();
    return cuda_fail(e1, "batch streams");
  }
  cudaGraph_t graph;
  if ((e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal))) {
    release();
    G.release();
    return cuda_fail(e, "batch capture");
  }
  const int nst = kind == 0 ? 1 : 4;
  e1 = cudaEventRecord(ev[ng], cs);
  for (size_t gi = 0; gi < ng && !e1; ++gi) {
    const BatchGroup& g = b->groups[gi];
    if ((e1 = cudaStreamWaitEvent(gs[gi], ev[ng], 0))) break;
    for (int st = 0; st < nst && !e1; ++st) {
      BatchMesh* tab = G.d_tables[st * ng + gi];
      if (!g.members.empty()) {
        if ((e1 = launch_batch(g.dim, g.p + 1, 0, tab, g.d_pitems, (int)g.pitems.size(), g.pgrid, g.pthreads,
                               g.psmem, gs[gi])))
          break;
        if ((e1 = launch_batch(g.dim, g.p + 1, 1, tab, g.d_ritems, (int)g.ritems.size(), g.rgrid, g.rthreads,
                               g.rsmem, gs[gi])))
          break;
      }
      for (int i : g.solo) {   // the group's large meshes: their own launches, same stage
        esd_mesh m = b->meshes[i];
        double* u = const_cast<double*>(G.u[i]);
        const double* in = u;
        Epilogue ep{};
        if (kind == 0) {
          ep.mode = 0;
          ep.dudt = const_cast<double*>(G.u[b->meshes.size() + i]);
        } else {
          const double ra[4] = {0.5, 0.5, 1.0, 0.0};
          const double rb[4] = {1.0 / 6.0, 1.0 / 3.0, 1.0 / 3.0, 1.0 / 6.0};
          in = st == 0 ? u : m->ws_stage;
          ep.mode = 1;
          ep.u0 = u;
          ep.acc_in = st == 0 ? u : m->ws_acc;
          ep.acc_out = st == 3 ? u : m->ws_acc;
          ep.stage_out = st == 3 ? nullptr : m->ws_stage;
          ep.ca = ra[st] * G.dt[i];
          ep.cb = rb[st] * G.dt[i];
        }
        if ((e1 = launch_project(m->R, m->M, m->L, in, nullptr, gs[gi]))) break;
        if ((e1 = launch_residual(m->R, m->M, m->L, ep, gs[gi]))) break;
      }
    }
    if (!e1) e1 = cudaEventRecord(ev[gi], gs[gi]);
    if (!e1) e1 = cudaStreamWaitEvent(cs, ev[gi], 0);
  }
  e = cudaStreamEndCapture(cs, &graph);
  if (e1 || e) {
    if (!e) cudaGraphDestroy(graph);
    release();
    G.release();
    return e1 ? cuda_fail(e1, "batch launch") : cuda_fail(e, "batch end capture");
  }
  e = cudaGraphInstantiate(&G.exec, graph, 0);
  cudaGraphDestroy(graph);
  release();
  if (e) {
    G.exec = nullptr;
    G.release();
    return cuda_fail(e, "batch graph instantiate");
  }
  if (b->graphs.size() >= kMaxCachedGraphs) {
    cudaDeviceSynchronize();   // the evicted graph's launches still read its device tables
    b->graphs.front().release();
    b->graphs.erase(b->graphs.begin());
  }
  b->graphs.push_back(G);
  e = cudaGraphLaunch(G.exec, s);
  return e ? cuda_fail(e, "batch graph launch") : ESD_OK;
}

esd_status esd_batch_rhs(esd_batch b, const double* const* u, double* const* dudt, void* stream) {
  if (b && !b->meshes.empty())
    if (esd_status ds = check_device(b->meshes[0]->device)) return ds;
  ESD_RANGE("esd_batch_rhs");
  if (!b || !u || !dudt) return fail(ESD_ERR_ARG, "null argument");
  const size_t n = b->meshes.size();
  std::vector<const double*> ptrs(2 * n);
  esd_status st;
  for (size_t i = 0; i < n; ++i) {
    if ((st = check_dev(u[i], "u[i]")) || (st = check_dev(dudt[i], "dudt[i]"))) return st;
    if (u[i] == dudt[i]) return fail(ESD_ERR_ARG, "u[i] and dudt[i] must not alias");
    ptrs[i] = u[i];
    ptrs[n + i] = dudt[i];
  }
  return batch_run(b, 0, ptrs, {}, (cudaStream_t)stream);
}

esd_status esd_batch_rk_step(esd_batch b, double* const* u, const double* dt, void* stream) {
  if (b && !b->meshes.empty())
    if (esd_status ds = check_device(b->meshes[0]->device)) return ds;
  ESD_RANGE("esd_batch_rk_step");
  if (!b || !u || !dt) return fail(ESD_ERR_ARG, "null argument");
  const size_t n = b->meshes.size();
  std::vector<const double*> ptrs(n);
  std::vector<double> dts(n);
  esd_status st;
  for (size_t i = 0; i < n; ++i) {
    if ((st = check_dev(u[i], "u[i]"))) return st;
    if (!(dt[i] > 0.0)) return fail(ESD_ERR_ARG, "dt[i] must be positive");
    ptrs[i] = u[i];
    dts[i] = dt[i];
  }
  return batch_run(b, 1, ptrs, dts, (cudaStream_t)stream);
}

// ---------------------------------------------------------------------------
// esd_rhs_static_scratch: the same two kernels as esd_rhs, with the per-node
// state scratch taken from a fixed array in device global memory instead of
// the mesh's workspace.  The array is reserved on every device when the
// library loads and is held until the process exits.
// ---------------------------------------------------------------------------
namespace {
constexpr size_t kStaticScratchBytes = size_t(32) << 20;   // 32 MiB
constexpr size_t kStaticScratchDoubles = kStaticScratchBytes / sizeof(double);
static __device__ __align__(256) double g_static_scratch[kStaticScratchDoubles];

// Device address of g_static_scratch on the current device.  In host code the
// symbol's name is only a host-side stand-in, so the address is looked up with the
// device current.  The lookup is repeated on every call (it is a host-side table lookup
// once the library's device code is loaded on the device): an address cached across calls
// would go stale if the device's context were reset and the code reloaded elsewhere.
esd_status static_scratch_address(double** out) {
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
  if (e != cudaSuccess || p == nullptr) return cuda_fail(e, "cudaGetSymbolAddress(static scratch)");
  *out = static_cast<double*>(p);
  return ESD_OK;
}
}  // namespace

esd_status esd_rhs_static_scratch(esd_mesh m, const double* u, double* dudt, void* stream) {
  if (!m) return fail(ESD_ERR_ARG, "null mesh");
  if (esd_status ds = check_device(m->device)) return ds;
  if (esd_status ps = reject_partition(m, "esd_rhs_static_scratch")) return ps;
  esd_status st;
  if ((st = check_dev(u, "u")) || (st = check_dev(dudt, "dudt"))) return st;
  if (u == dudt) return fail(ESD_ERR_ARG, "u and dudt must not alias");
  const size_t n_states = (size_t)m->E * nfields(m->dim) * m->ref.Ntot;
  const size_t n_cfac = (size_t)m->E * m->ref.Nfn;
  const size_t n_cfac_off = (n_states + 31) / 32 * 32;          // keep the second block 256-byte aligned
  if (n_cfac_off + n_cfac > kStaticScratchDoubles) {
    char msg[256];
    std::snprintf(msg, sizeof msg,
                  "mesh needs %zu bytes of state scratch; esd_rhs_static_scratch is limited to %zu bytes "
                  "(use esd_rhs for larger meshes)",
                  (n_cfac_off + n_cfac) * sizeof(double), kStaticScratchBytes);
    return fail(ESD_ERR_UNSUPPORTED, msg);
  }
  double* scratch = nullptr;
  if ((st = static_scratch_address(&scratch))) return st;
  DevMesh M = m->M;
  M.states = scratch;               // fully rewritten by the projection kernel before it is read
  M.cfac = scratch + n_cfac_off;
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = launch_project(m->R, M, m->L, u, nullptr, s);
  if (e) return cuda_fail(e, "project launch");
  Epilogue ep{};
  ep.mode = 0;
  ep.dudt = dudt;
  e = launch_residual(m->R, M, m->L, ep, s);
  return e ? cuda_fail(e, "residual launch") : ESD_OK;
}

// ---------------------------------------------------------------------------
// Autotuner: elements per CTA (and threads for the projection) chosen by timing the
// kernels on this mesh.  Every element is computed by the same per-element code
// whatever the tiling, so the results do not depend on the choice.
// ---------------------------------------------------------------------------
static float time_launches(const std::function<cudaError_t()>& f, cudaStream_t s, int reps) {
  if (f() != cudaSuccess) return 1e30f;   // warm-up
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  cudaEventRecord(a, s);
  for (int i = 0; i < reps; ++i)
    if (f() != cudaSuccess) {
      cudaEventDestroy(a);
      cudaEventDestroy(b);
      return 1e30f;
    }
  cudaEventRecord(b, s);
  cudaEventSynchronize(b);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, a, b);
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  return ms / reps;
}

esd_status esd_autotune(esd_mesh m, const double* u, void* stream) {
  return esd_autotune_kernels(m, u, ESD_TUNE_ALL, stream);
}

esd_status esd_autotune_kernels(esd_mesh m, const double* u, int kernels, void* stream) {
  ESD_RANGE("esd_autotune_kernels");
  if (!m) return fail(ESD_ERR_ARG, "null mesh");
  if (esd_status ds = check_device(m->device)) return ds;
  if (kernels & ~ESD_TUNE_ALL) return fail(ESD_ERR_ARG, "unknown kernel bits");
  esd_status st;
  if ((st = check_dev(u, "u"))) return st;
  cudaStream_t s = (cudaStream_t)stream;
  const RefTables& r = m->ref;
  const size_t budget = 227 * 1024;
  LaunchCfg best = m->L;
  const char* ev = std::getenv("ESD_AUTOTUNE_VERBOSE");   // print every candidate's time
  const bool verbose = ev && ev[0] == '1';
  // projection: elements per CTA x threads
  if (kernels & ESD_TUNE_PROJECT) {
    float tbest = 1e30f;
    const int emax = std::max(1, (int)(budget / smem_project(r, 1)));
    for (int e = emax; e >= 1; e = e > 1 ? e / 2 : 0) {
      for (int thr : {128, 256, 512}) {
        LaunchCfg L = m->L;
        L.ea = e;
        L.ta = thr;
        L.sa = smem_project(r, e);
        float t = time_launches([&] { return launch_project(m->R, m->M, L, u, nullptr, s); }, s, 3);
        if (verbose) std::fprintf(stderr, "esd_autotune: project  elems/CTA %3d threads %4d  %.4f ms\n", e, thr, t);
        if (t < tbest) {
          tbest = t;
          best.ea = L.ea;
          best.ta = L.ta;
          best.sa = L.sa;
        }
      }
      if (e == 1) break;
    }
  }
  // residual: elements per CTA (threads follow: E * line tasks * lanes per task, rounded to warps)
  if (kernels & ESD_TUNE_RESIDUAL) {
    cudaError_t e0 = launch_project(m->R, m->M, best, u, nullptr, s);
    if (e0) return cuda_fail(e0, "autotune projection");
    Epilogue ep{};
    ep.mode = 0;
    ep.dudt = m->ws_stage;   // scratch output (the RK stage buffer; autotuning drops captured graphs)
    float tbest = 1e30f;
    const int emax = std::min(std::max(1, (int)(budget / smem_residual(r, 1))),
                              std::max(1, 1024 / (residual_line_lanes(r.dim, r.n) * r.T)));
    for (int e = 1; e <= emax; ++e) {
      LaunchCfg L = best;
      L.eb = e;
      L.tb = residual_threads(r.dim, r.n, r.T, e);
      L.sb = smem_residual(r, e);
      float t = time_launches([&] { return launch_residual(m->R, m->M, L, ep, s); }, s, 3);
      if (verbose) std::fprintf(stderr, "esd_autotune: residual elems/CTA %3d threads %4d  %.4f ms\n", e, L.tb, t);
      if (t < tbest) {
        tbest = t;
        best.eb = L.eb;
        best.tb = L.tb;
        best.sb = L.sb;
      }
    }
  }
  // projection adjoint (esd_rhs_vjp): elements per CTA x threads, with the residual
  // adjoint's current shape (meshes with stored pair tables)
  if ((kernels & ESD_TUNE_ADJOINT) && !m->M.gvol) {
    float tbest = 1e30f;
    const int emax = std::max(1, (int)(budget / smem_project(r, 1)));
    for (int e = emax; e >= 1; e = e > 1 ? e / 2 : 0) {
      for (int thr : {128, 256, 512}) {
        LaunchCfg L = best;
        L.eq = e;
        L.tq = thr;
        L.sq = smem_project(r, e);
        float t = time_launches([&] {
          return launch_vjp(m->R, m->M, L, u, m->ws_adj[0], m->ws_adj[1], m->ws_qbar, m->ws_qext, s);
        }, s, 2);
        if (verbose) std::fprintf(stderr, "esd_autotune: vjp-proj elems/CTA %3d threads %4d  %.4f ms\n", e, thr, t);
        if (t < tbest) {
          tbest = t;
          best.eq = L.eq;
          best.tq = L.tq;
          best.sq = L.sq;
        }
      }
      if (e == 1) break;
    }
  }
  // residual adjoint (esd_rhs_vjp): elements per CTA (meshes with stored pair tables)
  if ((kernels & ESD_TUNE_ADJOINT) && !m->M.gvol) {
    float tbest = 1e30f;
    const int emax = std::max(1, (int)(budget / smem_residual_adj(r, 1)));
    for (int e = 1; e <= emax; ++e) {
      if (e > 1 && adj_threads_host(r, e) > 512) break;   // 128 registers per thread
      LaunchCfg L = best;
      L.ev = e;
      L.tv = std::max(64, adj_threads_host(r, e));
      L.sv = smem_residual_adj(r, e);
      float t = time_launches([&] {
        return launch_vjp(m->R, m->M, L, u, m->ws_adj[0], m->ws_adj[1], m->ws_qbar, m->ws_qext, s);
      }, s, 2);
      if (verbose) std::fprintf(stderr, "esd_autotune: vjp      elems/CTA %3d threads %4d  %.4f ms\n", e, L.tv, t);
      if (t < tbest) {
        tbest = t;
        best.ev = L.ev;
        best.tv = L.tv;
        best.sv = L.sv;
      }
    }
  }
  cudaError_t e = cudaStreamSynchronize(s);
  cudaGetLastError();
  if (e) return cuda_fail(e, "autotune");
  m->L = best;
  for (auto& g : m->graphs) cudaGraphExecDestroy(g.exec);   // captured graphs hold the old launch shapes
  m->graphs.clear();
  return ESD_OK;
}

esd_status esd_launch_stage(esd_mesh m, int stage, const double* u, double* out, void* stream) {
  if (!m) return fail(ESD_ERR_ARG, "null mesh");
  if (esd_status ds = check_device(m->device)) return ds;
  cudaStream_t s = (cudaStream_t)stream;
  esd_status st;
  if (stage == 0) {
    if ((st = check_dev(u, "u"))) return st;
    cudaError_t e = launch_project(m->R, m->M, m->L, u, nullptr, s);
    return e ? cuda_fail(e, "project launch") : ESD_OK;
  }
  if (stage == 1) {
    if ((st = check_dev(out, "out"))) return st;
    Epilogue ep{};
    ep.mode = 0;
    ep.dudt = out;
    cudaError_t e = launch_residual(m->R, m->M, m->L, ep, s);
    return e ? cuda_fail(e, "residual launch") : ESD_OK;
  }
  return fail(ESD_ERR_ARG, "stage must be 0 or 1");
}

esd_status esd_ref_info(int dim, int p, esd_info* o) {
  if (!o) return fail(ESD_ERR_ARG, "null output");
  RefTables r;
  std::string err;
  esd_status st = build_ref(dim, p, &r, &err);
  if (st != ESD_OK) return fail(st, err);
  std::memset(o, 0, sizeof(*o));
  o->dim = r.dim; o->p = r.p; o->n_c = dim + 2; o->n_modes = r.Np; o->n_vol_nodes = r.Nq;
  o->n_facets = r.Nf; o->n_facet_nodes = r.Nqf;
  o->vol_pairs_per_elem = r.nvp;
  o->facet_pairs_per_elem = r.nfp;
  const int64_t q = r.p, n = q + 1;
  o->paper_flux_count_per_elem = r.dim == 2 ? (q * n * n) / 2 + q * n * n + 3 * n * n
                                            : 3 * q * n * n * n + 3 * n * n * n + n * n * n * n;
  return ESD_OK;
}

esd_status esd_debug_host_setup(const esd_mesh_desc* d, double* wj, double* bj, double* nrm, double* vdir,
                                double* fdir, int32_t* nbr, int32_t* nbr_node, double* xvol) {
  if (!d) return fail(ESD_ERR_ARG, "null descriptor");
  if (d->n_elem <= 0 || !d->map_nodes || !d->nbr_elem || !d->nbr_face) return fail(ESD_ERR_ARG, "bad mesh arrays");
  HostMesh H;
  std::string err;
  esd_status st = build_host_mesh(*d, &H, &err);
  if (st != ESD_OK) return fail(st, err);
  auto cp = [](auto* dst, const auto& v) {
    if (dst) std::memcpy(dst, v.data(), v.size() * sizeof(v[0]));
  };
  cp(wj, H.wj); cp(bj, H.bj); cp(nrm, H.nrm); cp(vdir, H.vdir); cp(fdir, H.fdir);
  cp(nbr, H.nbr_e); cp(nbr_node, H.nbr_f); cp(xvol, H.xvol);
  return ESD_OK;
}

esd_status esd_debug_check_layouts(void) {
  std::string err;
  if (!audit_layouts(&err)) return fail(ESD_ERR_UNSUPPORTED, err.c_str());
  return ESD_OK;
}

esd_status esd_debug_math(int which, const double* x, double* y, int64_t n, void* stream) {
  if (which != 0 && which != 1) return fail(ESD_ERR_ARG, "which must be 0 (log) or 1 (exp)");
  esd_status st;
  if ((st = check_dev(x, "x")) || (st = check_dev(y, "y"))) return st;
  static std::mutex mu;
  static double* tab[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) return fail(ESD_ERR_UNSUPPORTED, "device index");
  {
    std::lock_guard<std::mutex> lock(mu);
    if (!tab[dev]) {
      std::vector<double> h(kMathTabSize);
      build_math_table(h.data());
      void* p = nullptr;
      cudaError_t e = cudaMalloc(&p, h.size() * sizeof(double));
      if (e) return cuda_fail(e, "math table");
      e = cudaMemcpy(p, h.data(), h.size() * sizeof(double), cudaMemcpyHostToDevice);
      if (e) return cuda_fail(e, "math table");
      tab[dev] = static_cast<double*>(p);
    }
  }
  cudaError_t e = launch_math_probe(which, tab[dev], x, y, n, (cudaStream_t)stream);
  return e ? cuda_fail(e, "math probe") : ESD_OK;
}

esd_status esd_measure_fp64_peak(double* flops, void* stream) {
  if (!flops) return fail(ESD_ERR_ARG, "null output");
  cudaError_t e = measure_fp64(flops, (cudaStream_t)stream);
  return e ? cuda_fail(e, "fp64 probe") : ESD_OK;
}

// ---------------------------------------------------------------------------
// The skew-symmetric form of Eq. (rhs_skew): a mesh with the form's line-pair
// coefficients, a trace kernel (u = V u~ and its facet traces, the cross-element input)
// and the line-task residual kernel.
// ---------------------------------------------------------------------------
struct esd_skew_s {
  esd_mesh m = nullptr;
  SkewModel P{};
  int nc = 0;
  int et = 1, tt = 128;  size_t st = 0;   // trace kernel: elements/CTA, threads, smem
  int er = 1, tr = 128;  size_t sr = 0;   // residual kernel
  ~esd_skew_s() { delete m; }
};

esd_status esd_skew_create(const esd_mesh_desc* d, const esd_skew_model* model, esd_skew* out) {
  ESD_RANGE("esd_skew_create");
  if (!d || !model || !out) return fail(ESD_ERR_ARG, "null argument");
  *out = nullptr;
  if (model->model != ESD_SKEW_EULER && model->model != ESD_SKEW_ADVECTION)
    return fail(ESD_ERR_ARG, "model must be ESD_SKEW_EULER or ESD_SKEW_ADVECTION");
  if (model->model == ESD_SKEW_ADVECTION && model->upwind != 0 && model->upwind != 1)
    return fail(ESD_ERR_ARG, "upwind must be 0 or 1");
  esd_mesh m = nullptr;
  esd_status st = mesh_create(d, kTablesSkew, &m);
  if (st) return st;
  esd_skew k = new esd_skew_s();
  k->m = m;
  k->nc = model->model == ESD_SKEW_EULER ? d->dim + 2 : 1;
  k->P.gamma = d->gamma;
  for (int i = 0; i < 3; ++i) k->P.a[i] = i < d->dim ? model->a[i] : 0.0;
  k->P.sigma = model->model == ESD_SKEW_ADVECTION && model->upwind ? 1.0 : 0.0;
  const RefTables& r = m->ref;
  const int nc = k->nc;
  constexpr size_t kBudget = 227 * 1024;
  // trace kernel: the projection kernel's tile (its layout with nc variables)
  const size_t pe_t = (size_t)nc * (r.Np + 3 * r.Nq + r.Nfn) * sizeof(double);
  k->et = std::max(1, std::min(32, (int)(kBudget / pe_t)));
  k->tt = 256;
  k->st = k->et * pe_t;
  // residual kernel: E elements x T line tasks; E maximises the threads doing line work per
  // SM within shared memory and registers
  const SkewLayout Ly = r.dim == 2 ? skew_layout<2>(nc, r.Nq, r.Np, r.n) : skew_layout<3>(nc, r.Nq, r.Np, r.n);
  const size_t pe_r = (size_t)Ly.pe * sizeof(double);
  int regs = 255, max_thr = 256;
  cudaError_t e = r.dim == 2 ? skew_residual_attrs_d2(r.n, nc, (int)kBudget, &regs, &max_thr)
                             : skew_residual_attrs_d3(r.n, nc, (int)kBudget, &regs, &max_thr);
  if (!e) e = r.dim == 2 ? skew_trace_attrs_d2((int)kBudget) : skew_trace_attrs_d3((int)kBudget);
  if (e) {
    delete k;
    return cuda_fail(e, "skew kernel attributes");
  }
  int best = 1;
  double best_score = -1.0;
  const int emax = std::max(1, std::min((int)(kBudget / pe_r), 1024 / r.T));
  const int regs_alloc = (std::max(regs, 1) + 7) / 8 * 8;   // registers are allocated in groups of 8
  for (int el = 1; el <= emax; ++el) {
    const int thr = ((el * r.T + 31) / 32) * 32;
    if (el > 1 && (thr > max_thr || (size_t)thr * regs_alloc > 65536)) break;   // the block must fit
    const int by_smem = (int)(kBudget / (el * pe_r));
    const int by_regs = std::max(1, 65536 / (regs_alloc * thr));
    const int ctas = std::max(1, std::min(std::min(by_smem, by_regs), 32));
    const double score = (double)ctas * el * r.T + 1e-3 * (double)(el * r.T) / thr;
    if (score > best_score) {
      best_score = score;
      best = el;
    }
  }
  k->er = best;
  k->tr = std::max(32, ((best * r.T + 31) / 32) * 32);
  k->sr = best * pe_r;
  *out = k;
  return ESD_OK;
}

esd_status esd_skew_destroy(esd_skew k) {
  if (!k) return fail(ESD_ERR_ARG, "null handle");
  cudaDeviceSynchronize();
  delete k;
  return ESD_OK;
}

esd_status esd_skew_check(esd_skew k, void* stream) {
  if (!k) return fail(ESD_ERR_ARG, "null handle");
  return esd_mesh_check(k->m, stream);
}

esd_status esd_rhs_skew(esd_skew k, const double* u, double* dudt, void* stream) {
  ESD_RANGE("esd_rhs_skew");
  if (!k) return fail(ESD_ERR_ARG, "null handle");
  esd_mesh m = k->m;
  if (esd_status ds = check_device(m->device)) return ds;
  esd_status st;
  if ((st = check_dev(u, "u")) || (st = check_dev(dudt, "dudt"))) return st;
  if (u == dudt) return fail(ESD_ERR_ARG, "u and dudt must not alias");
  cudaStream_t s = (cudaStream_t)stream;
  const int n = m->ref.n, nc = k->nc;
  cudaError_t e = m->dim == 2 ? launch_skew_trace_d2(nc, m->R, m->M, k->P, k->et, k->tt, k->st, u, s)
                              : launch_skew_trace_d3(nc, m->R, m->M, k->P, k->et, k->tt, k->st, u, s);
  if (e) return cuda_fail(e, "skew trace launch");
  e = m->dim == 2 ? launch_skew_residual_d2(n, nc, m->R, m->M, k->P, m->sdir, k->er, k->tr, k->sr, u, dudt, s)
                  : launch_skew_residual_d3(n, nc, m->R, m->M, k->P, m->sdir, k->er, k->tr, k->sr, u, dudt, s);
  return e ? cuda_fail(e, "skew residual launch") : ESD_OK;
}

esd_status esd_skew_info(esd_skew k, int* n_vars, int* elems_per_cta, int* threads_per_cta) {
  if (!k) return fail(ESD_ERR_ARG, "null handle");
  if (n_vars) *n_vars = k->nc;
  if (elems_per_cta) *elems_per_cta = k->er;
  if (threads_per_cta) *threads_per_cta = k->tr;
  return ESD_OK;
}

}  // extern "C"
