"""Python binding of the esd C-ABI library (include/esd.h; test hooks in include/esd_test.h).

Argument marshalling only: every step of the computation runs in the CUDA
kernels of libesd.so.  Torch tensors provide device memory and streams.  The
functions mirror the C names; ``Mesh`` is a small convenience wrapper.

The library must have been built (``python -m paper_2312_07874_gb300.build`` or
``__graft_entry__.build()``); importing fails loudly otherwise.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libesd.so")

ESD_FLUX_EC, ESD_FLUX_LF = 0, 1


class EsdError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{msg} (status {status})")
        self.status = status


class esd_mesh_desc(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("p", ctypes.c_int), ("n_elem", ctypes.c_int64),
                ("map_nodes", ctypes.POINTER(ctypes.c_double)), ("nbr_elem", ctypes.POINTER(ctypes.c_int32)),
                ("nbr_face", ctypes.POINTER(ctypes.c_int8)), ("gamma", ctypes.c_double), ("flux", ctypes.c_int)]


class esd_info(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("p", ctypes.c_int), ("n_c", ctypes.c_int), ("n_modes", ctypes.c_int),
                ("n_vol_nodes", ctypes.c_int), ("n_facets", ctypes.c_int), ("n_facet_nodes", ctypes.c_int),
                ("n_elem", ctypes.c_int64), ("vol_pairs_per_elem", ctypes.c_int64),
                ("facet_pairs_per_elem", ctypes.c_int64), ("paper_flux_count_per_elem", ctypes.c_int64),
                ("device_bytes", ctypes.c_size_t), ("elems_per_cta_project", ctypes.c_int),
                ("elems_per_cta_residual", ctypes.c_int)]


class esd_skew_model(ctypes.Structure):
    _fields_ = [("model", ctypes.c_int), ("a", ctypes.c_double * 3), ("upwind", ctypes.c_int)]


ESD_SKEW_EULER, ESD_SKEW_ADVECTION = 0, 1

SYMBOLS = {
    "esd_mesh_create": ([ctypes.POINTER(esd_mesh_desc), ctypes.POINTER(ctypes.c_void_p)], ctypes.c_int),
    "esd_mesh_create_ex": ([ctypes.POINTER(esd_mesh_desc), ctypes.c_int, ctypes.POINTER(ctypes.c_void_p)],
                           ctypes.c_int),
    "esd_mesh_destroy": ([ctypes.c_void_p], ctypes.c_int),
    "esd_mesh_info": ([ctypes.c_void_p, ctypes.POINTER(esd_info)], ctypes.c_int),
    "esd_mesh_check": ([ctypes.c_void_p, ctypes.c_void_p], ctypes.c_int),
    "esd_mesh_volume_nodes": ([ctypes.c_void_p, ctypes.c_void_p], ctypes.c_int),
    "esd_l2_project": ([ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p], ctypes.c_int),
    "esd_project_entropy": ([ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p], ctypes.c_int),
    "esd_rhs": ([ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p], ctypes.c_int),
    "esd_rhs_vjp": ([ctypes.c_void_p] * 5, ctypes.c_int),
    "esd_rhs_static_scratch": ([ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p], ctypes.c_int),
    "esd_rk_step": ([ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double, ctypes.c_void_p, ctypes.c_void_p], ctypes.c_int),
    "esd_rk_step_vjp": ([ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double, ctypes.c_void_p, ctypes.c_void_p,
                         ctypes.c_void_p], ctypes.c_int),
    "esd_tape_doubles": ([ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64)], ctypes.c_int),
    "esd_rhs_save": ([ctypes.c_void_p] * 5, ctypes.c_int),
    "esd_rhs_vjp_saved": ([ctypes.c_void_p] * 6, ctypes.c_int),
    "esd_rk_step_save": ([ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double, ctypes.c_void_p, ctypes.c_void_p,
                          ctypes.c_void_p], ctypes.c_int),
    "esd_rk_step_vjp_saved": ([ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double, ctypes.c_void_p,
                               ctypes.c_void_p, ctypes.c_void_p], ctypes.c_int),
    "esd_part_create": ([ctypes.POINTER(esd_mesh_desc), ctypes.c_int64, ctypes.POINTER(ctypes.c_void_p)],
                        ctypes.c_int),
    "esd_part_info": ([ctypes.c_void_p] + [ctypes.POINTER(ctypes.c_int64)] * 3, ctypes.c_int),
    "esd_rhs_begin": ([ctypes.c_void_p] * 3, ctypes.c_int),
    "esd_rhs_end": ([ctypes.c_void_p] * 3, ctypes.c_int),
    "esd_rhs_vjp_mid": ([ctypes.c_void_p] * 3, ctypes.c_int),
    "esd_rhs_vjp_end": ([ctypes.c_void_p] * 4, ctypes.c_int),
    "esd_part_export": ([ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                         ctypes.c_void_p], ctypes.c_int),
    "esd_part_import": ([ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64,
                         ctypes.c_void_p], ctypes.c_int),
    "esd_diagnostics": ([ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p], ctypes.c_int),
    "esd_integrals": ([ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p], ctypes.c_int),
    "esd_batch_create": ([ctypes.POINTER(ctypes.c_void_p), ctypes.c_int, ctypes.POINTER(ctypes.c_void_p)], ctypes.c_int),
    "esd_batch_destroy": ([ctypes.c_void_p], ctypes.c_int),
    "esd_batch_rhs": ([ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_void_p),
                       ctypes.c_void_p], ctypes.c_int),
    "esd_batch_rk_step": ([ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_double),
                           ctypes.c_void_p], ctypes.c_int),
    "esd_autotune": ([ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p], ctypes.c_int),
    "esd_autotune_kernels": ([ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p], ctypes.c_int),
    "esd_launch_stage": ([ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p],
                         ctypes.c_int),
    "esd_measure_fp64_peak": ([ctypes.POINTER(ctypes.c_double), ctypes.c_void_p], ctypes.c_int),
    "esd_ref_info": ([ctypes.c_int, ctypes.c_int, ctypes.POINTER(esd_info)], ctypes.c_int),
    "esd_debug_host_setup": ([ctypes.POINTER(esd_mesh_desc)] + [ctypes.c_void_p] * 8, ctypes.c_int),
    "esd_debug_staging_timeout": ([ctypes.c_void_p, ctypes.c_double, ctypes.c_void_p], ctypes.c_int),
    "esd_debug_check_layouts": ([], ctypes.c_int),
    "esd_debug_math": ([ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p],
                       ctypes.c_int),
    "esd_debug_set_mesh_device": ([ctypes.c_void_p, ctypes.c_int], ctypes.c_int),
    "esd_debug_batch_solo_waves": ([ctypes.c_int], ctypes.c_int),
    "esd_skew_create": ([ctypes.POINTER(esd_mesh_desc), ctypes.POINTER(esd_skew_model),
                         ctypes.POINTER(ctypes.c_void_p)], ctypes.c_int),
    "esd_skew_destroy": ([ctypes.c_void_p], ctypes.c_int),
    "esd_rhs_skew": ([ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p], ctypes.c_int),
    "esd_skew_check": ([ctypes.c_void_p, ctypes.c_void_p], ctypes.c_int),
    "esd_skew_info": ([ctypes.c_void_p] + [ctypes.POINTER(ctypes.c_int)] * 3, ctypes.c_int),
    "esd_status_string": ([ctypes.c_int], ctypes.c_char_p),
    "esd_last_error": ([], ctypes.c_char_p),
}

_lib = None


def lib():
    """Load libesd.so (raises if the CUDA library has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libesd.so not built: run __graft_entry__.build() ({LIB_PATH} missing)")
        L = ctypes.CDLL(LIB_PATH)
        for name, (args, res) in SYMBOLS.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _lib = L
    return _lib


def _check(status):
    if status != 0:
        msg = lib().esd_last_error().decode()
        raise EsdError(status, msg or lib().esd_status_string(status).decode())


def _ptr(t):
    """Device pointer of a contiguous float64 CUDA tensor."""
    import torch
    if not isinstance(t, torch.Tensor):
        raise TypeError("expected a torch.Tensor")
    if t.dtype != torch.float64 or not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous float64 CUDA tensor")
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


# ---- C-named entry points (thin marshalling) -----------------------------------------
ESD_MESH_PAIR_TABLES, ESD_MESH_METRICS_ON_THE_FLY = 0, 1


def esd_mesh_create(dim, p, map_nodes, nbr_elem, nbr_face, gamma=1.4, flux=ESD_FLUX_LF,
                    options=ESD_MESH_PAIR_TABLES, n_ghost=0):
    X = np.ascontiguousarray(map_nodes, dtype=np.float64)
    ne = np.ascontiguousarray(nbr_elem, dtype=np.int32)
    nf = np.ascontiguousarray(nbr_face, dtype=np.int8)
    d = esd_mesh_desc(dim, p, X.shape[0], X.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                      ne.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), nf.ctypes.data_as(ctypes.POINTER(ctypes.c_int8)),
                      gamma, flux)
    h = ctypes.c_void_p()
    if n_ghost:
        if options != ESD_MESH_PAIR_TABLES:
            raise ValueError("partition meshes use the stored pair tables")
        _check(lib().esd_part_create(ctypes.byref(d), int(n_ghost), ctypes.byref(h)))
    elif options == ESD_MESH_PAIR_TABLES:
        _check(lib().esd_mesh_create(ctypes.byref(d), ctypes.byref(h)))
    else:
        _check(lib().esd_mesh_create_ex(ctypes.byref(d), int(options), ctypes.byref(h)))
    return h


def esd_ref_info(dim, p):
    i = esd_info()
    _check(lib().esd_ref_info(dim, p, ctypes.byref(i)))
    return {k: getattr(i, k) for k, _ in esd_info._fields_}


def esd_debug_host_setup(dim, p, map_nodes, nbr_elem, nbr_face, gamma=1.4, flux=ESD_FLUX_LF):
    """Host part of mesh creation only (no device); returns the host tables as numpy arrays."""
    X = np.ascontiguousarray(map_nodes, dtype=np.float64)
    ne = np.ascontiguousarray(nbr_elem, dtype=np.int32)
    nf = np.ascontiguousarray(nbr_face, dtype=np.int8)
    E = X.shape[0]
    info = esd_ref_info(dim, p)
    Nq, Nfn = info["n_vol_nodes"], info["n_facets"] * info["n_facet_nodes"]
    out = dict(wj=np.empty((E, Nq)), bj=np.empty((E, Nfn)), nrm=np.empty((E, dim, Nfn)),
               vdir=np.empty((E, info["vol_pairs_per_elem"] * dim)),
               fdir=np.empty((E, info["facet_pairs_per_elem"] * dim)),
               nbr=np.empty((E, Nfn), dtype=np.int32), nbr_node=np.empty((E, Nfn), dtype=np.int32),
               xvol=np.empty((E, Nq, dim)))
    d = esd_mesh_desc(dim, p, E, X.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                      ne.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), nf.ctypes.data_as(ctypes.POINTER(ctypes.c_int8)),
                      gamma, flux)
    args = [out[k].ctypes.data_as(ctypes.c_void_p) for k in ("wj", "bj", "nrm", "vdir", "fdir", "nbr", "nbr_node", "xvol")]
    _check(lib().esd_debug_host_setup(ctypes.byref(d), *args))
    return out, info


def esd_mesh_destroy(h):
    _check(lib().esd_mesh_destroy(h))


def esd_mesh_info(h):
    i = esd_info()
    _check(lib().esd_mesh_info(h, ctypes.byref(i)))
    return {k: getattr(i, k) for k, _ in esd_info._fields_}


def esd_mesh_check(h, stream=None):
    _check(lib().esd_mesh_check(h, _stream(stream)))


def esd_mesh_volume_nodes(h, n_elem, n_q, dim):
    x = np.empty((n_elem, n_q, dim))
    _check(lib().esd_mesh_volume_nodes(h, x.ctypes.data_as(ctypes.c_void_p)))
    return x


def esd_l2_project(h, u_nodal, u_modal, stream=None):
    _check(lib().esd_l2_project(h, _ptr(u_nodal), _ptr(u_modal), _stream(stream)))


def esd_project_entropy(h, u, w_modal, stream=None):
    _check(lib().esd_project_entropy(h, _ptr(u), _ptr(w_modal), _stream(stream)))


def esd_rhs(h, u, dudt, stream=None):
    _check(lib().esd_rhs(h, _ptr(u), _ptr(dudt), _stream(stream)))


def esd_rhs_static_scratch(h, u, dudt, stream=None):
    """esd_rhs without any allocation: state scratch from the library's fixed device array."""
    _check(lib().esd_rhs_static_scratch(h, _ptr(u), _ptr(dudt), _stream(stream)))


def esd_rhs_vjp(h, u, cot, grad, stream=None):
    _check(lib().esd_rhs_vjp(h, _ptr(u), _ptr(cot), _ptr(grad), _stream(stream)))


def esd_rk_step(h, u, dt, stage_ckpt=None, stream=None):
    ck = _ptr(stage_ckpt) if stage_ckpt is not None else ctypes.c_void_p()
    _check(lib().esd_rk_step(h, _ptr(u), float(dt), ck, _stream(stream)))


def esd_rk_step_vjp(h, stage_ckpt, dt, cot_out, cot_in, stream=None):
    _check(lib().esd_rk_step_vjp(h, _ptr(stage_ckpt), float(dt), _ptr(cot_out), _ptr(cot_in), _stream(stream)))


def esd_tape_doubles(h):
    """Doubles of one forward tape (the entropy-projected states of one right-hand side)."""
    n = ctypes.c_int64()
    _check(lib().esd_tape_doubles(h, ctypes.byref(n)))
    return n.value


def esd_rhs_save(h, u, dudt, tape, stream=None):
    _check(lib().esd_rhs_save(h, _ptr(u), _ptr(dudt), _ptr(tape), _stream(stream)))


def esd_rhs_vjp_saved(h, u, tape, cot, grad, stream=None):
    _check(lib().esd_rhs_vjp_saved(h, _ptr(u), _ptr(tape), _ptr(cot), _ptr(grad), _stream(stream)))


def esd_rk_step_save(h, u, dt, stage_ckpt, tapes, stream=None):
    _check(lib().esd_rk_step_save(h, _ptr(u), float(dt), _ptr(stage_ckpt), _ptr(tapes), _stream(stream)))


def esd_rk_step_vjp_saved(h, stage_ckpt, tapes, dt, cot_out, cot_in, stream=None):
    _check(lib().esd_rk_step_vjp_saved(h, _ptr(stage_ckpt), _ptr(tapes), float(dt), _ptr(cot_out), _ptr(cot_in),
                                       _stream(stream)))


ESD_TRACE_STATES, ESD_TRACE_COTANGENTS = 0, 1


def esd_part_info(h):
    """(n_ghost, doubles per element of a state trace, of a cotangent trace)."""
    a, b, c = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    _check(lib().esd_part_info(h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
    return a.value, b.value, c.value


def esd_rhs_begin(h, u, stream=None):
    _check(lib().esd_rhs_begin(h, _ptr(u), _stream(stream)))


def esd_rhs_end(h, dudt, stream=None):
    _check(lib().esd_rhs_end(h, _ptr(dudt), _stream(stream)))


def esd_rhs_vjp_mid(h, cot, stream=None):
    _check(lib().esd_rhs_vjp_mid(h, _ptr(cot), _stream(stream)))


def esd_rhs_vjp_end(h, u, grad, stream=None):
    _check(lib().esd_rhs_vjp_end(h, _ptr(u), _ptr(grad), _stream(stream)))


def _ptr_i64(t):
    """Device pointer of a contiguous int64 CUDA tensor."""
    import torch
    if t.dtype != torch.int64 or not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous int64 CUDA tensor")
    return ctypes.c_void_p(t.data_ptr())


def esd_part_export(h, kind, elems, buf, stream=None):
    _check(lib().esd_part_export(h, int(kind), _ptr_i64(elems), elems.numel(), _ptr(buf), _stream(stream)))


def esd_part_import(h, kind, buf, first, n, stream=None):
    _check(lib().esd_part_import(h, int(kind), _ptr(buf), int(first), int(n), _stream(stream)))


def esd_diagnostics(h, u, out, stream=None):
    _check(lib().esd_diagnostics(h, _ptr(u), _ptr(out), _stream(stream)))


def esd_integrals(h, u, out, stream=None):
    _check(lib().esd_integrals(h, _ptr(u), _ptr(out), _stream(stream)))


ESD_TUNE_PROJECT, ESD_TUNE_RESIDUAL, ESD_TUNE_ADJOINT, ESD_TUNE_ALL = 1, 2, 4, 7


def esd_autotune(h, u, stream=None):
    _check(lib().esd_autotune(h, _ptr(u), _stream(stream)))


def esd_autotune_kernels(h, u, kernels, stream=None):
    _check(lib().esd_autotune_kernels(h, _ptr(u), int(kernels), _stream(stream)))


def esd_launch_stage(h, stage, u=None, out=None, stream=None):
    _check(lib().esd_launch_stage(h, int(stage), _ptr(u) if u is not None else None,
                                  _ptr(out) if out is not None else None, _stream(stream)))


def esd_debug_check_layouts():
    """Host-side audit of the kernels' shared-memory layouts for every supported degree."""
    _check(lib().esd_debug_check_layouts())


def esd_debug_staging_timeout(handle, seconds=0.05, stream=None):
    """Failure-path hook: a wait that nothing completes gives up after `seconds`; the next
    esd_mesh_check reports ESD_ERR_TIMEOUT."""
    _check(lib().esd_debug_staging_timeout(handle, float(seconds), _stream(stream)))


def esd_debug_math(which, x, y, stream=None):
    _check(lib().esd_debug_math(int(which), _ptr(x), _ptr(y), x.numel(), _stream(stream)))


def esd_measure_fp64_peak(stream=None):
    v = ctypes.c_double()
    _check(lib().esd_measure_fp64_peak(ctypes.byref(v), _stream(stream)))
    return v.value


def esd_batch_create(handles):
    arr = (ctypes.c_void_p * len(handles))(*[h.value for h in handles])
    b = ctypes.c_void_p()
    _check(lib().esd_batch_create(arr, len(handles), ctypes.byref(b)))
    return b


def esd_batch_destroy(b):
    _check(lib().esd_batch_destroy(b))


def esd_batch_rhs(b, us, dudts, stream=None):
    ua = (ctypes.c_void_p * len(us))(*[t.data_ptr() for t in us])
    da = (ctypes.c_void_p * len(dudts))(*[t.data_ptr() for t in dudts])
    _check(lib().esd_batch_rhs(b, ua, da, _stream(stream)))


def esd_batch_rk_step(b, us, dts, stream=None):
    ua = (ctypes.c_void_p * len(us))(*[t.data_ptr() for t in us])
    da = (ctypes.c_double * len(dts))(*[float(x) for x in dts])
    _check(lib().esd_batch_rk_step(b, ua, da, _stream(stream)))


# ---- convenience wrapper ------------------------------------------------------------
class Mesh:
    """Owns an esd_mesh handle; state tensors are float64 CUDA [n_elem, N_c, N_p*]."""

    def __init__(self, dim, p, map_nodes, nbr_elem, nbr_face, gamma=1.4, flux="LF", metrics_on_the_fly=False,
                 n_ghost=0):
        """n_ghost > 0: a partition mesh whose last n_ghost elements are ghosts
        (esd_part_create; paper_2312_07874_gb300.partition builds the descriptions)."""
        self.handle = esd_mesh_create(dim, p, map_nodes, nbr_elem, nbr_face, gamma,
                                      ESD_FLUX_LF if flux == "LF" else ESD_FLUX_EC,
                                      ESD_MESH_METRICS_ON_THE_FLY if metrics_on_the_fly else ESD_MESH_PAIR_TABLES,
                                      n_ghost)
        self.info = esd_mesh_info(self.handle)
        self.dim, self.p = dim, p
        self.n_elem = self.info["n_elem"]
        self.nc = self.info["n_c"]
        self.n_modes = self.info["n_modes"]
        self.n_q = self.info["n_vol_nodes"]

    def close(self):
        if self.handle is not None:
            esd_mesh_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def empty_state(self):
        import torch
        return torch.empty((self.n_elem, self.nc, self.n_modes), dtype=torch.float64, device="cuda")

    def empty_tapes(self, *shape):
        """Forward tapes (esd_rhs_save / esd_rk_step_save): a float64 tensor of shape
        shape + (esd_tape_doubles,) on the device; torch allocations are 256-byte aligned and
        each tape is a multiple of 32 doubles, so every tape in it is 16-byte aligned."""
        import torch
        return torch.empty(tuple(shape) + (esd_tape_doubles(self.handle),), dtype=torch.float64, device="cuda")

    def volume_nodes(self):
        return esd_mesh_volume_nodes(self.handle, self.n_elem, self.n_q, self.dim)

    def l2_project(self, u_nodal):
        out = self.empty_state()
        esd_l2_project(self.handle, u_nodal.contiguous(), out)
        return out

    def project_entropy(self, u):
        out = self.empty_state()
        esd_project_entropy(self.handle, u, out)
        return out

    def rhs(self, u, out=None):
        out = self.empty_state() if out is None else out
        esd_rhs(self.handle, u, out)
        return out

    def rk_step(self, u, dt, stage_ckpt=None):
        esd_rk_step(self.handle, u, dt, stage_ckpt)
        return u

    def diagnostics(self, u):
        import torch
        out = torch.empty(self.nc + 2, dtype=torch.float64, device="cuda")
        esd_diagnostics(self.handle, u, out)
        return out

    def integrals(self, u):
        """[N_c + 1]: totals of the conserved variables, then of the entropy function."""
        import torch
        out = torch.empty(self.nc + 1, dtype=torch.float64, device="cuda")
        esd_integrals(self.handle, u, out)
        return out

    def run_diagnostics(self, u, dt, n_steps, every=1):
        """Advance u in place by n_steps RK4 steps, sampling before the first step and
        after every `every` steps the totals (esd_integrals) and the rates (esd_diagnostics):
        returns (steps [K], totals [K, N_c + 1], rates [K, N_c + 2]) as numpy arrays."""
        import numpy as np
        import torch
        steps, tot, rates = [], [], []

        def sample(k):
            steps.append(k)
            tot.append(self.integrals(u))
            rates.append(self.diagnostics(u))
        sample(0)
        for k in range(1, n_steps + 1):
            self.rk_step(u, dt)
            if k % every == 0 or k == n_steps:
                sample(k)
        torch.cuda.synchronize()
        self.check()
        return (np.array(steps), torch.stack(tot).cpu().numpy(), torch.stack(rates).cpu().numpy())

    def check(self):
        esd_mesh_check(self.handle)

    def autotune(self, u, kernels=ESD_TUNE_ALL):
        """Time launch shapes on this mesh and state u and keep the fastest (esd_autotune);
        `kernels` selects the projection / residual / adjoint kernels (ESD_TUNE_* bits)."""
        esd_autotune_kernels(self.handle, u, kernels)
        self.info = esd_mesh_info(self.handle)
        return self.info


# ---- skew-symmetric form (Eq. (rhs_skew)) ----------------------------------------------
def esd_skew_create(dim, p, map_nodes, nbr_elem, nbr_face, model=ESD_SKEW_EULER, a=(0.0, 0.0, 0.0),
                    upwind=False, gamma=1.4, flux=ESD_FLUX_LF):
    X = np.ascontiguousarray(map_nodes, dtype=np.float64)
    ne = np.ascontiguousarray(nbr_elem, dtype=np.int32)
    nf = np.ascontiguousarray(nbr_face, dtype=np.int8)
    d = esd_mesh_desc(dim, p, X.shape[0], X.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                      ne.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), nf.ctypes.data_as(ctypes.POINTER(ctypes.c_int8)),
                      gamma, flux)
    av = (list(a) + [0.0, 0.0, 0.0])[:3]
    m = esd_skew_model(int(model), (ctypes.c_double * 3)(*av), int(bool(upwind)))
    h = ctypes.c_void_p()
    _check(lib().esd_skew_create(ctypes.byref(d), ctypes.byref(m), ctypes.byref(h)))
    return h


def esd_skew_destroy(h):
    _check(lib().esd_skew_destroy(h))


def esd_rhs_skew(h, u, dudt, stream=None):
    _check(lib().esd_rhs_skew(h, _ptr(u), _ptr(dudt), _stream(stream)))


def esd_skew_check(h, stream=None):
    _check(lib().esd_skew_check(h, _stream(stream)))


def esd_skew_info(h):
    nv, ec, tc = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(lib().esd_skew_info(h, ctypes.byref(nv), ctypes.byref(ec), ctypes.byref(tc)))
    return dict(n_vars=nv.value, elems_per_cta=ec.value, threads_per_cta=tc.value)


class Skew:
    """Owns an esd_skew handle (the skew-symmetric form of Eq. (rhs_skew)); states are float64
    CUDA [n_elem, N_c, N_p*] with N_c = dim + 2 (Euler) or 1 (linear advection)."""

    def __init__(self, dim, p, map_nodes, nbr_elem, nbr_face, model="euler", a=(0.0, 0.0, 0.0), upwind=False,
                 gamma=1.4, flux="LF"):
        kind = ESD_SKEW_EULER if model == "euler" else ESD_SKEW_ADVECTION
        self.handle = esd_skew_create(dim, p, map_nodes, nbr_elem, nbr_face, kind, a, upwind, gamma,
                                      ESD_FLUX_LF if flux == "LF" else ESD_FLUX_EC)
        info = esd_ref_info(dim, p)
        self.dim, self.p = dim, p
        self.n_elem = np.asarray(map_nodes).shape[0]
        self.n_modes = info["n_modes"]
        self.info = esd_skew_info(self.handle)
        self.nc = self.info["n_vars"]

    def close(self):
        if self.handle is not None:
            esd_skew_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def rhs(self, u, out=None):
        import torch
        if out is None:
            out = torch.empty((self.n_elem, self.nc, self.n_modes), dtype=torch.float64, device="cuda")
        esd_rhs_skew(self.handle, u, out)
        return out

    def check(self):
        esd_skew_check(self.handle)
