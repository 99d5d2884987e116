/*
 * esd_test.h -- test and measurement hooks of libesd.so (not part of the product ABI
 * declared in esd.h; the library exports them for its own test suite and benchmark).
 * None of them has a counterpart in the paper.  Status codes, stream and pointer
 * conventions are those of esd.h.
 */
#ifndef ESD_TEST_H
#define ESD_TEST_H

#include "esd.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Measurement hook: launch one kernel of the esd_rhs pipeline alone, so that it can be
 * timed with events on `stream`.  stage 0: the projection kernel on u (entropy projection
 * and entropy-projected states at all nodes, written to the handle's workspace; `out`
 * unused, may be NULL); stage 1: the residual kernel on the workspace states left by the
 * last stage-0 launch, writing d u~/dt to `out` (device).  esd_rhs == stage 0 then 1. */
esd_status esd_launch_stage(esd_mesh mesh, int stage, const double* u, double* out, void* stream);

/* Measurement helper: sustained FP64 FMA throughput of this device, in FP64
 * operations (1 FMA = 2) per second, measured with a register-resident FMA chain
 * on the given stream (synchronous). */
esd_status esd_measure_fp64_peak(double* flops_per_s, void* stream);


/* Test hook: run only the host part of esd_mesh_create (no device is touched) and
 * copy selected host tables out.  Every output is optional (NULL skips it); sizes,
 * with the library's internal node order (volume node c1 + n*(c2 + n*c3), facet
 * node zeta*Nqf + a + n*b, see the kernels for the pair order):
 *   wj [n_elem][N_q] (W J), bj [n_elem][N_f*Nqf] (B J^(kappa,zeta)),
 *   nrm [n_elem][dim][N_f*Nqf] (unit normals), vdir [n_elem][vol_pairs*dim],
 *   fdir [n_elem][facet_pairs*dim] (pair directions), nbr [n_elem][N_f*Nqf]
 *   (neighbour element), nbr_node (neighbour facet node), xvol [n_elem][N_q][dim]. */
esd_status esd_debug_host_setup(const esd_mesh_desc* desc, double* wj, double* bj, double* nrm, double* vdir,
                                double* fdir, int32_t* nbr, int32_t* nbr_node, double* xvol);

/* Test hook: y = log(x) (which = 0) or exp(x) (which = 1) elementwise with the library's
 * table-driven device implementations; x, y device arrays of n doubles. */
esd_status esd_debug_math(int which, const double* x, double* y, int64_t n, void* stream);

/* Host-side audit (no device needed): for every supported (dim, p), the shared-memory
 * layouts of the residual and adjoint kernels are in bounds and disjoint where live
 * together, bulk copies are 16-byte sized and aligned, and the default launch shapes fit
 * one CTA.  ESD_OK, or ESD_ERR_UNSUPPORTED with the first violation in esd_last_error(). */
esd_status esd_debug_check_layouts(void);

/* Test hook for the failure path of the bounded waits (not in the paper): launches one
 * block that waits on a shared-memory barrier that nothing completes; after `seconds`
 * (0 < seconds <= 10) the wait gives up and sets the mesh's error flag, so that the next
 * esd_mesh_check returns ESD_ERR_TIMEOUT.  The kernels' staging copies use the same
 * bounded wait (about one second). */
esd_status esd_debug_staging_timeout(esd_mesh mesh, double seconds, void* stream);

/* Test hook: overwrite the device index recorded in the mesh handle at creation, so that
 * the check that every compute call runs with the mesh's device current can be exercised
 * on a machine with one GPU (the next compute call then returns ESD_ERR_ARG without
 * launching anything).  Pass the true index to restore the handle. */
esd_status esd_debug_set_mesh_device(esd_mesh mesh, int device);

/* Test hook: the size (in waves of residual CTAs over the GPU) from which esd_batch_create
 * runs a member mesh with its own launches inside the batch graph instead of the group's
 * persistent launch (default 1).  0 runs every mesh on its own; a large value runs every
 * mesh in the persistent launches.  Applies to batches created afterwards; ESD_ERR_ARG if
 * negative. */
esd_status esd_debug_batch_solo_waves(int waves);

#ifdef __cplusplus
}
#endif
#endif /* ESD_TEST_H */
