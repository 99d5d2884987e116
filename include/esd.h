/*
 * esd.h -- C ABI of a GB300 (sm_103a) FP64 library for the entropy-stable modal
 * discontinuous spectral-element method with tensor-product summation-by-parts
 * operators on curved triangles and tetrahedra (Montoya & Zingg, arXiv 2312.07874).
 *
 * Conventions used by every entry point
 * -------------------------------------
 * - Arithmetic is IEEE FP64 throughout.
 * - Modal state arrays ("u", "dudt", "w_modal", cotangents) are device pointers
 *   to double, C-contiguous with layout [n_elem][N_c][N_p*], N_c = dim + 2,
 *   N_p* = C(p+dim, dim).  Variables are ordered (rho, rho v_1 .. rho v_dim, E)
 *   (Eq. (euler), Section 7.1).  Modes are the normalized PKD polynomials of
 *   Eq. (modal_basis_2d) / Eq. (modal_basis_3d) (Section 4.3), multi-indices
 *   alpha in lexicographic order with alpha_1 slowest:
 *     for a1 in 0..p: for a2 in 0..p-a1: [for a3 in 0..p-a1-a2:]
 * - Device arrays must be allocated by the caller (cudaMalloc or a framework
 *   allocator), be 8-byte aligned, and stay alive until the stream work that
 *   uses them completes.  The library never allocates or frees memory in the
 *   per-step calls; everything it needs is allocated by esd_mesh_create (the batch
 *   calls allocate their small per-launch tables once per new set of arguments).
 * - "stream" is a cudaStream_t passed as void*; NULL is the legacy default
 *   stream.  All device calls are asynchronous on that stream; a returned
 *   ESD_OK means the work was enqueued.
 * - Errors are returned as esd_status, never thrown or trapped on the device.
 *   esd_last_error() returns a human-readable message for the calling thread.
 *   Argument errors (null/host pointers, bad sizes) are detected before any
 *   launch.  A non-admissible state (rho <= 0, p <= 0 or non-finite values at a
 *   quadrature node) sets a device flag that esd_mesh_check() reports as
 *   ESD_ERR_STATE.
 * - A mesh handle may be used from one host thread at a time.  It belongs to the
 *   device that was current when it was created (its tables and workspace live there):
 *   every call that touches the device must be made with that device current, else it
 *   returns ESD_ERR_ARG before enqueuing anything.
 * - Test and measurement hooks (timing one kernel, the FP64 peak, host-table export,
 *   failure-path probes) are declared separately in esd_test.h.
 */
#ifndef ESD_H
#define ESD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  ESD_OK = 0,
  ESD_ERR_ARG = -1,         /* invalid argument (null, host pointer, misaligned, out of range) */
  ESD_ERR_MESH = -2,        /* J <= 0, non-conforming facets, bad connectivity */
  ESD_ERR_CUDA = -3,        /* a CUDA runtime call failed */
  ESD_ERR_STATE = -4,       /* non-admissible state seen by a kernel (rho <= 0, p <= 0, NaN/Inf) */
  ESD_ERR_TIMEOUT = -5,     /* a bounded device-side wait gave up */
  ESD_ERR_NOMEM = -6,       /* device allocation failed at create time */
  ESD_ERR_UNSUPPORTED = -7  /* degree or size outside what the library supports */
} esd_status;

enum { ESD_FLUX_EC = 0, ESD_FLUX_LF = 1 };

typedef struct esd_mesh_s* esd_mesh;
typedef struct esd_batch_s* esd_batch;

/* Mesh description (all pointers are HOST pointers, read during esd_mesh_create only).
 *
 * map_nodes: [n_elem][N*_p][dim] physical positions of the degree-p mapping nodes
 *   of every element (isoparametric p_g = q = p, Section 7.3).  The nodes are the
 *   equispaced lattice of the reference simplex, first lattice index fastest:
 *     triangle:    for j in 0..p: for i in 0..p-j:            xi = (-1+2i/p, -1+2j/p)
 *     tetrahedron: for k: for j: for i (i+j+k <= p): xi = (-1+2i/p, -1+2j/p, -1+2k/p)
 *   Reference simplex: triangle (-1,-1),(1,-1),(-1,1) (Eq. (reference_triangle));
 *   tetrahedron (-1,-1,-1),(1,-1,-1),(-1,1,-1),(-1,-1,1) (Eq. (reference_tetrahedron)).
 * nbr_elem/nbr_face: [n_elem][N_f], the element and local facet across each local facet
 *   (facets numbered as in Eq. (tri_facets) / Eq. (tet_facets)).  Every facet must have a
 *   neighbour (periodic meshes).  Tetrahedra must be oriented so that both sides of
 *   a facet collapse its quadrature rule onto the same vertex (Remark 5); the facet
 *   node correspondence (identity or reversal of the first facet coordinate) is
 *   found from node positions, which may differ by one constant periodic shift.
 * gamma: ratio of specific heats (Section 7.1).
 * flux: ESD_FLUX_LF (entropy stable, Eq. (num_flux) with Eq. (wave_speed)) or
 *   ESD_FLUX_EC (entropy conservative: no dissipative term).
 */
typedef struct {
  int dim;                  /* 2 (triangles) or 3 (tetrahedra) */
  int p;                    /* polynomial degree p = q = p_g; 1..10 (triangles and tetrahedra) */
  int64_t n_elem;
  const double* map_nodes;
  const int32_t* nbr_elem;
  const int8_t* nbr_face;
  double gamma;
  int flux;
} esd_mesh_desc;

typedef struct {
  int dim, p, n_c, n_modes, n_vol_nodes, n_facets, n_facet_nodes;
  int64_t n_elem;
  int64_t vol_pairs_per_elem;          /* line-based volume pairs, dim*q(q+1)^dim/2 */
  int64_t facet_pairs_per_elem;        /* nnz of R^T B summed over facets */
  int64_t paper_flux_count_per_elem;   /* Eq. (num_fluxes) */
  size_t device_bytes;                 /* device memory held by the handle */
  int elems_per_cta_project, elems_per_cta_residual;
} esd_info;

/* Build reference tables, curved geometry (exact adjugate metrics in 2D, conservative
 * curl form of Eq. (conservative_curl) in 3D, Nanson normals Eq. (nanson), interpolated
 * Jacobian Eq. (jacobian_approx)), facet connectivity, and mesh-static pair
 * coefficients; validates J > 0 (Eq. (jacobian_positive)) and Assumption 2; uploads
 * everything and allocates the workspace.  Synchronous.  Errors: ESD_ERR_ARG,
 * ESD_ERR_MESH, ESD_ERR_UNSUPPORTED, ESD_ERR_NOMEM, ESD_ERR_CUDA. */
esd_status esd_mesh_create(const esd_mesh_desc* desc, esd_mesh* out);

/* esd_mesh_create with a choice of how the flux-differencing kernel obtains its pair
 * directions (not in the paper's text, a storage/arithmetic trade of Section 5):
 *   ESD_MESH_PAIR_TABLES         (= esd_mesh_create) the directions n_ij of every line pair,
 *                                Eq. (avg_volume_metric), and of every facet-correction pair,
 *                                Eq. (facet_correction), precomputed per element (O(p^(d+1))
 *                                doubles per element; 42 KB per tetrahedron at p = 4);
 *   ESD_MESH_METRICS_ON_THE_FLY  only the metric terms G at the volume nodes and J^zeta n at
 *                                the facet nodes are stored (O(p^d) per element, the paper's
 *                                storage); the kernel forms every direction from them.
 * esd_rhs, esd_rk_step, esd_diagnostics and esd_rhs_static_scratch accept both kinds of mesh
 * and give the same results up to rounding; esd_rhs_vjp, esd_rk_step_vjp and the batch calls
 * need ESD_MESH_PAIR_TABLES (ESD_ERR_UNSUPPORTED otherwise). */
enum { ESD_MESH_PAIR_TABLES = 0, ESD_MESH_METRICS_ON_THE_FLY = 1 };
esd_status esd_mesh_create_ex(const esd_mesh_desc* desc, int options, esd_mesh* out);
esd_status esd_mesh_destroy(esd_mesh mesh);
esd_status esd_mesh_info(esd_mesh mesh, esd_info* out);

/* Synchronize the stream, then report (and clear) the device error flag: ESD_OK,
 * ESD_ERR_TIMEOUT, ESD_ERR_STATE (a non-admissible state) or ESD_ERR_ARG (an
 * esd_part_export element index outside the partition).
 * ESD_ERR_TIMEOUT means that a shared-memory staging copy of some block did not complete
 * within its bounded wait of about one second: that block skipped its work (its outputs
 * hold stale values) after waiting once more, for the same time, for its copies to land.
 * If they had still not landed, a copy may complete into shared memory after the block
 * has exited.  Treat the outputs of every call since the previous check as invalid, and a
 * device that times out as unreliable for the rest of the process. */
esd_status esd_mesh_check(esd_mesh mesh, void* stream);

/* Physical coordinates of the volume quadrature nodes, HOST output
 * [n_elem][N_q][dim] in the library's node order (the same order esd_l2_project
 * expects).  Used to evaluate initial data. */
esd_status esd_mesh_volume_nodes(esd_mesh mesh, double* x_host);

/* Reference L2 projection u~ = V^T W u of nodal data given at the volume nodes
 * (input layout [n_elem][N_c][N_q], device) -- an input-preparation helper. */
esd_status esd_l2_project(esd_mesh mesh, const double* u_nodal, double* u_modal, void* stream);

/* Entropy projection, Eq. (entropy_expansion): w~ = M~^{-1} V^T W J W(V u~) with the
 * weight-adjusted inverse M~^{-1} = V^T W J^{-1} V of Eq. (weight_adjusted_inverse)
 * (M = I).  u: [n_elem][N_c][N_p*] in, w_modal: same layout out (device). */
esd_status esd_project_entropy(esd_mesh mesh, const double* u, double* w_modal, void* stream);

/* Time derivative of Eq. (dudt_modal), d u~/dt = M~^{-1} V^T r, with the nodal
 * residual r of Eq. (entropy_stable): line-based flux differencing along the
 * collapsed-coordinate lines, facet correction Eq. (facet_correction), interface flux
 * Eq. (interface_flux).  u, dudt: device, [n_elem][N_c][N_p*]; u and dudt must not alias. */
esd_status esd_rhs(esd_mesh mesh, const double* u, double* dudt, void* stream);

/* esd_rhs for callers that cannot allocate device memory (the paper has no counterpart).
 *
 * Some callers cannot call cudaMalloc: plug-ins running inside a host application that
 * owns the whole device-memory budget through its own allocator, or fixed-footprint
 * deployments that forbid any allocation after start-up.  This entry point computes
 * exactly what esd_rhs computes, with the same kernels, but takes the per-node state
 * scratch (entropy-projected states and facet sound speeds) from a fixed array in device
 * global memory that the library reserves on every GPU when it is loaded (32 MiB, held
 * until the process exits) instead of from the mesh's workspace.  It allocates nothing.
 * The caller still passes the inputs (mesh, u) and the output (dudt).
 * - Limit: the mesh needs n_elem * ((dim+5) * (N_q + N_f*N_fq) + N_f*N_fq) doubles of
 *   scratch (about 15 KB per element for tetrahedra at p = 4, 2.4 KB for triangles at
 *   p = 4); larger meshes are rejected with ESD_ERR_UNSUPPORTED before any launch.
 * - Each call looks up the array's device address on the current device (the mesh's
 *   device: see above).  The first call on a device also loads the library's device
 *   code there if nothing has loaded it yet; make that first call before any stream
 *   capture.
 * - Every call shares the one array and leaves the last call's contents in it.  Nothing
 *   in it needs to start at zero (each call overwrites every value it reads), but calls
 *   that overlap on the GPU (different streams, or concurrent host threads) race on it.
 * u, dudt: device [n_elem][N_c][N_p*]; they must not alias. */
esd_status esd_rhs_static_scratch(esd_mesh mesh, const double* u, double* dudt, void* stream);

/* Vector-Jacobian product of esd_rhs with respect to u: grad = (d rhs / d u)^T cot.
 * The paper has no counterpart (it is the adjoint of Eq. (dudt_modal)).  u, cot, grad:
 * device [n_elem][N_c][N_p*]; grad must not alias u or cot. */
esd_status esd_rhs_vjp(esd_mesh mesh, const double* u, const double* cot, double* grad, void* stream);

/* One classical RK4 step of size dt in place on u (not in the paper, which uses DP8).
 * stage_ckpt: NULL or device [4][n_elem][N_c][N_p*]; when given, the four stage
 * inputs are stored there for esd_rk_step_vjp.  The launch sequence is captured in a
 * CUDA graph per (u, dt, stage_ckpt, stream) and replayed on later calls; the 16 most
 * recently captured graphs are kept per mesh. */
esd_status esd_rk_step(esd_mesh mesh, double* u, double dt, double* stage_ckpt, void* stream);

/* Discrete adjoint of one esd_rk_step: given the stage checkpoints written by the forward
 * step and the cotangent of the step's output, write the cotangent of its input.
 * cot_out, cot_in: device [n_elem][N_c][N_p*]; they may alias (in place). */
esd_status esd_rk_step_vjp(esd_mesh mesh, const double* stage_ckpt, double dt, const double* cot_out,
                           double* cot_in, void* stream);

/* Reverse mode with a saved forward pass.  esd_rhs_vjp and esd_rk_step_vjp first recompute
 * the entropy projection of their input state (Eq. (entropy_expansion) and the states
 * U(w) at every volume and facet node), which the adjoint kernels read.  A caller that can
 * hold those per-node states from the forward call skips that work: the _save calls run
 * the same kernels as esd_rhs / esd_rk_step but leave the projection of each right-hand
 * side in a caller-owned tape, and the _saved VJPs read it instead of recomputing it.
 * Results are identical (bitwise) to the recomputing calls.
 *
 * A tape holds esd_tape_doubles() doubles: the entropy-projected states with their
 * derived fields [n_elem][dim+5][N_q + N_f N_fq] and the facet sound speeds [n_elem][N_f N_fq],
 * each padded to a multiple of 32 doubles (about 15 KB per tetrahedron at p = 4, 11 times
 * the modal state).  tape / tapes: device, 16-byte aligned (ESD_ERR_ARG otherwise: the
 * kernels stage each element's states with bulk copies), owned by the caller.  A tape is
 * valid for the state it was written from until it is overwritten; the library cannot
 * check that the u passed to a _saved VJP is that state.  Meshes created with
 * ESD_MESH_METRICS_ON_THE_FLY have no VJP (ESD_ERR_UNSUPPORTED). */
esd_status esd_tape_doubles(esd_mesh mesh, int64_t* n_doubles);

/* esd_rhs, keeping the forward tape of u in tape (esd_tape_doubles doubles). */
esd_status esd_rhs_save(esd_mesh mesh, const double* u, double* dudt, double* tape, void* stream);

/* esd_rhs_vjp at the state u whose tape esd_rhs_save wrote (the projection is not
 * recomputed).  u, cot, grad as for esd_rhs_vjp; tape is only read. */
esd_status esd_rhs_vjp_saved(esd_mesh mesh, const double* u, const double* tape, const double* cot, double* grad,
                             void* stream);

/* esd_rk_step with stage_ckpt (required here) and the four stages' forward tapes in
 * tapes: device [4][esd_tape_doubles].  Graph-replayed like esd_rk_step; the graph cache
 * key includes tapes. */
esd_status esd_rk_step_save(esd_mesh mesh, double* u, double dt, double* stage_ckpt, double* tapes, void* stream);

/* esd_rk_step_vjp reading the tapes that esd_rk_step_save wrote with the same stage_ckpt. */
esd_status esd_rk_step_vjp_saved(esd_mesh mesh, const double* stage_ckpt, const double* tapes, double dt,
                                 const double* cot_out, double* cot_in, void* stream);

/* Diagnostics of Theorems 2 and 4: out (device, N_c + 2 doubles) receives
 * sum_kappa 1^T r^(kappa,e) for each variable e (equal to sum 1^T W J V d u~/dt), then
 * sum_kappa sum_e w^T r (the entropy rate, zero for ESD_FLUX_EC on periodic meshes), then
 * sum |w_i r_i| as its scale. */
esd_status esd_diagnostics(esd_mesh mesh, const double* u, double* out, void* stream);

/* Totals over the mesh of the state u (device [n_elem][N_c][N_p*]): out (device, N_c + 1
 * doubles) receives sum_kappa 1^T W J V u~ for each conserved variable (the quantities
 * Theorem 2 conserves; constant over RK steps up to rounding on periodic meshes), then
 * sum_kappa 1^T W J S(V u~), the total of the entropy function S = -rho s / (gamma - 1),
 * s = ln(p / rho^gamma) (Section 7.1; constant in time for ESD_FLUX_EC up to the time
 * integration error, non-increasing for ESD_FLUX_LF).  Quadrature of the mass matrix
 * (interpolated J).  Used for conservation and entropy time series over a run. */
esd_status esd_integrals(esd_mesh mesh, const double* u, double* out, void* stream);

/* Element partitions.  The semi-discretisation couples elements only through the interface
 * flux of Eq. (num_flux) at shared facets (Section 4.3), i.e. through the neighbours' facet
 * traces, so a mesh split into partitions needs one exchange of facet traces per right-hand
 * side (and, for the VJP, one exchange of the interface cotangents).  These calls expose
 * that structure: each partition is a mesh of its own, the phases of the evaluation are
 * separate calls, and the traces travel in caller-owned device buffers between them (on
 * several GPUs a collective or peer copy moves them; on one GPU a plain buffer does).
 *
 * esd_part_create: desc describes n_elem = n_local + n_ghost elements, the n_ghost ghosts
 * last, with their map nodes.  Local elements are computed; ghosts are not and exist only
 * to supply traces.  A local element's facet may face a ghost (nbr_elem in [n_local,
 * n_elem)); that ghost's nbr_elem / nbr_face entry for the shared facet must point back.
 * Other ghost facets are not read and may hold any value.  Facet nodes are matched as for
 * esd_mesh_create.  u, dudt, grad of a partition are [n_local][N_c][N_p*].  n_ghost = 0
 * gives an ordinary mesh.
 *
 * Calls that evaluate a whole right-hand side at once (esd_rhs, esd_rhs_save,
 * esd_rhs_static_scratch, esd_rk_step*, esd_rhs_vjp*, esd_rk_step_vjp*, esd_diagnostics,
 * esd_batch_create) return ESD_ERR_UNSUPPORTED on a partition with ghosts.  Instead:
 *   d u~/dt:  esd_rhs_begin(u)  (entropy projection, Eq. (entropy_expansion), of the local
 *             elements) -> esd_part_export(ESD_TRACE_STATES) of the elements the other
 *             partitions hold as ghosts, esd_part_import(ESD_TRACE_STATES) of this
 *             partition's ghosts -> esd_rhs_end(dudt)  (Eq. (dudt_modal));
 *   VJP:      esd_rhs_begin(u) -> exchange ESD_TRACE_STATES -> esd_rhs_vjp_mid(cot) ->
 *             exchange ESD_TRACE_COTANGENTS -> esd_rhs_vjp_end(u, grad).
 * Each partition's result equals the unpartitioned call's rows for its elements bit for
 * bit.  The phases also work on ordinary meshes (no exchange needed).  The mesh workspace
 * carries the state between phases: one evaluation at a time per mesh.
 *
 * esd_part_info: n_ghost, and the doubles per element of a trace message:
 *   ESD_TRACE_STATES      (dim + 6) N_f N_fq: the entropy-projected states with their
 *                         derived fields at the facet nodes, then the facet sound speeds;
 *   ESD_TRACE_COTANGENTS  (dim + 2) N_f N_fq: the cotangents of the neighbour's facet states
 *                         produced by the residual adjoint.
 * esd_part_export: elems (device int64 [n]) are local element indices; buf (device
 * [n][trace doubles]) receives their messages in that order.  An index outside [0, n_local)
 * sends zeros and makes the next esd_mesh_check return ESD_ERR_ARG.
 * esd_part_import: buf (device [n][trace doubles]) fills ghosts first .. first + n - 1
 * (ghost g is element n_local + g of the descriptor); ESD_ERR_ARG if the range leaves
 * [0, n_ghost).  Buffers must not overlap the mesh's own memory. */
enum { ESD_TRACE_STATES = 0, ESD_TRACE_COTANGENTS = 1 };
esd_status esd_part_create(const esd_mesh_desc* desc, int64_t n_ghost, esd_mesh* out);
esd_status esd_part_info(esd_mesh mesh, int64_t* n_ghost, int64_t* trace_doubles, int64_t* cotangent_doubles);
esd_status esd_rhs_begin(esd_mesh mesh, const double* u, void* stream);
esd_status esd_rhs_end(esd_mesh mesh, double* dudt, void* stream);
esd_status esd_rhs_vjp_mid(esd_mesh mesh, const double* cot, void* stream);
esd_status esd_rhs_vjp_end(esd_mesh mesh, const double* u, double* grad, void* stream);
esd_status esd_part_export(esd_mesh mesh, int kind, const int64_t* elems, int64_t n, double* buf, void* stream);
esd_status esd_part_import(esd_mesh mesh, int kind, const double* buf, int64_t first, int64_t n, void* stream);

/* The skew-symmetric nodal form of Section 4.4, Eq. (rhs_skew), with the modal update of
 * Eq. (modal) through the weight-adjusted inverse (M = I):
 *   r = 1/2 sum_l (Q^(l)T sum_m G^(l,m) f_m - sum_m G^(l,m) Q^(l) f_m)
 *       - sum_zeta R^T B J^zeta (f* - 1/2 sum_m N^(zeta,m) R f_m),  d u~/dt = M~^{-1} V^T r,
 * with the fluxes f_m evaluated at the nodal solution u = V u~ (no entropy projection and
 * no two-point flux: a different scheme from esd_rhs, the one Section 4.4 derives the
 * entropy-stable form from).  Two flux models:
 *   ESD_SKEW_EULER      the compressible Euler equations (Section 7.1), N_c = dim + 2, the
 *                       interface flux of Eq. (num_flux) (ESD_FLUX_LF) or its
 *                       entropy-conservative part (ESD_FLUX_EC), chosen by desc->flux;
 *   ESD_SKEW_ADVECTION  scalar linear advection f_m(u) = a_m u, N_c = 1, interface flux
 *                       (a.n)(u- + u+)/2 - sigma |a.n| (u+ - u-)/2, sigma = 1 with `upwind`
 *                       (energy stable on curved elements), 0 for the central flux.
 * esd_skew_create builds the mesh (as esd_mesh_create, from the same description) with the
 * form's mesh-static line-pair coefficients instead of the entropy-stable pair tables.
 * u, dudt: device [n_elem][N_c][N_p*]; they must not alias.  The handle belongs to the
 * device current at creation (as a mesh).  esd_skew_check reports the admissibility
 * flag (Euler: rho <= 0 or p <= 0 at a facet trace) as esd_mesh_check does. */
typedef struct esd_skew_s* esd_skew;
enum { ESD_SKEW_EULER = 0, ESD_SKEW_ADVECTION = 1 };
typedef struct {
  int model;      /* ESD_SKEW_EULER or ESD_SKEW_ADVECTION */
  double a[3];    /* advection velocity (components beyond dim ignored) */
  int upwind;     /* advection: 1 upwind, 0 central interface flux */
} esd_skew_model;
esd_status esd_skew_create(const esd_mesh_desc* desc, const esd_skew_model* model, esd_skew* out);
esd_status esd_skew_destroy(esd_skew skew);
esd_status esd_rhs_skew(esd_skew skew, const double* u, double* dudt, void* stream);
esd_status esd_skew_check(esd_skew skew, void* stream);
/* Number of variables N_c of the model and the residual kernel's launch shape (any output may
 * be NULL). */
esd_status esd_skew_info(esd_skew skew, int* n_vars, int* elems_per_cta, int* threads_per_cta);

/* Batched, persistent execution of many independent meshes (not in the paper).
 * Meshes are grouped by (dim, p).  In each group, the meshes whose residual launch would not
 * fill the GPU once share one persistent projection launch and one persistent residual
 * launch per stage; larger meshes keep their own launches.  One CUDA graph holds all groups
 * as concurrent branches.  Results equal the per-mesh calls bit for bit.  The batch keeps
 * references to the meshes, which must outlive it. */
esd_status esd_batch_create(const esd_mesh* meshes, int n, esd_batch* out);
esd_status esd_batch_destroy(esd_batch batch);
/* u[i], dudt[i]: device state arrays of mesh i (layouts as above). */
esd_status esd_batch_rhs(esd_batch batch, const double* const* u, double* const* dudt, void* stream);
/* One RK4 step of every mesh; dt[i] is a HOST array of step sizes.  Both batch calls
 * capture their launches in a CUDA graph per (pointers, step sizes, stream), replayed on
 * later calls with the same arguments; the 16 most recent are kept per batch (dropping
 * one waits for the device).  An RK4 step uses each member mesh's workspace, so two
 * batches (or a batch and a direct call) sharing a mesh must not overlap on the GPU. */
esd_status esd_batch_rk_step(esd_batch batch, double* const* u, const double* dt, void* stream);

/* Autotuner (not in the paper): time the projection kernel over elements-per-CTA x
 * threads-per-CTA, and the residual kernel and the residual adjoint (esd_rhs_vjp) over
 * elements-per-CTA, on this mesh and state u
 * (device, [n_elem][N_c][N_p*], admissible), keep the fastest, and drop captured RK4
 * graphs.  Per-element arithmetic is independent of the tiling, so results are unchanged.
 * Synchronous.  Batches built afterwards use the tuned tiles.  With the environment
 * variable ESD_AUTOTUNE_VERBOSE=1 every candidate's time is printed to stderr. */
esd_status esd_autotune(esd_mesh mesh, const double* u, void* stream);

/* The same for a subset of the kernels: `kernels` is a bitwise or of the ESD_TUNE_* bits
 * (ESD_ERR_ARG for other bits); esd_autotune == ESD_TUNE_ALL.  Shapes of the kernels not
 * selected are kept. */
enum { ESD_TUNE_PROJECT = 1, ESD_TUNE_RESIDUAL = 2, ESD_TUNE_ADJOINT = 4, ESD_TUNE_ALL = 7 };
esd_status esd_autotune_kernels(esd_mesh mesh, const double* u, int kernels, void* stream);

/* Per-element sizes for a (dim, p) pair without building a mesh (n_elem = 0,
 * device_bytes = 0, launch fields 0).  Host only. */
esd_status esd_ref_info(int dim, int p, esd_info* out);

const char* esd_status_string(esd_status s);
const char* esd_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* ESD_H */
