"""Child process of tests/test_zz_no_alloc.py (run on its own, without torch): calls
esd_rhs_static_scratch and esd_rhs on the same mesh and input, resets the device's
context with cudaDeviceReset (which ends only this process's context), rebuilds the mesh
and buffers, and compares again.  The entry point must find its fixed scratch array in
the new context.  Device memory comes from cudaMalloc of the CUDA runtime the library
itself loaded.  Prints one line per round: 'round k err e0 e1 ...'."""
import ctypes
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import esd_inputs as I                       # noqa: E402
import paper_2312_07874_gb300 as E           # noqa: E402

H2D, D2H = 1, 2


def main():
    L = E.lib()
    rt = ctypes.CDLL("libcudart.so.13")      # the runtime instance libesd.so was linked with
    rt.cudaMalloc.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.c_size_t]
    rt.cudaMemcpy.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int]
    rt.cudaFree.argtypes = [ctypes.c_void_p]

    def ok(code, what):
        if code != 0:
            raise SystemExit(f"{what} failed with {code}: {L.esd_last_error().decode()}")

    def dev(nbytes):
        p = ctypes.c_void_p()
        ok(rt.cudaMalloc(ctypes.byref(p), nbytes), "cudaMalloc")
        return p

    dim, M, p = 3, 3, 3
    mesh, X = I.config_mesh(dim, M, 2 * np.pi, p, True)
    for rnd in range(2):
        h = E.esd_mesh_create(dim, p, X, mesh.nbr_elem, mesh.nbr_face)
        info = E.esd_mesh_info(h)
        Eel, nq, npm, nc = info["n_elem"], info["n_vol_nodes"], info["n_modes"], info["n_c"]
        x = E.esd_mesh_volume_nodes(h, Eel, nq, dim)
        un = np.ascontiguousarray(np.transpose(I.taylor_green(x, 0.1), (0, 2, 1)))
        nb_nod, nb_mod = un.nbytes, Eel * nc * npm * 8
        d_un, d_u, d_ref, d_got = dev(nb_nod), dev(nb_mod), dev(nb_mod), dev(nb_mod)
        ok(rt.cudaMemcpy(d_un, un.ctypes.data, nb_nod, H2D), "cudaMemcpy")
        ok(L.esd_l2_project(h, d_un, d_u, None), "esd_l2_project")
        ok(L.esd_rhs(h, d_u, d_ref, None), "esd_rhs")
        ok(L.esd_rhs_static_scratch(h, d_u, d_got, None), "esd_rhs_static_scratch")
        ok(L.esd_mesh_check(h, None), "esd_mesh_check")
        ref = np.empty((Eel, nc, npm))
        got = np.empty((Eel, nc, npm))
        ok(rt.cudaMemcpy(ref.ctypes.data, d_ref, nb_mod, D2H), "cudaMemcpy")
        ok(rt.cudaMemcpy(got.ctypes.data, d_got, nb_mod, D2H), "cudaMemcpy")
        err = np.abs(got - ref).max(axis=(0, 2)) / np.abs(ref).max(axis=(0, 2))
        print(f"round {rnd} err " + " ".join(f"{e:.3e}" for e in err), flush=True)
        E.esd_mesh_destroy(h)
        for d in (d_un, d_u, d_ref, d_got):
            ok(rt.cudaFree(d), "cudaFree")
        if rnd == 0:
            ok(rt.cudaDeviceReset(), "cudaDeviceReset")


if __name__ == "__main__":
    main()
