"""The synthetic workloads (meshes, degrees, states) used by tests and benchmarks.

Named by what they are:
  tri_vortex_affine  : [0,2pi]^2, 8x8x2 = 128 affine triangles, p = 2, vortex at the centre
  tri_vortex_curved  : [0,1]^2, 64x64x2 = 8192 triangles, sine warp, p in {4,6,8,10},
                       vortex at (1/2,1/2) plus seeded U(-1e-3,1e-3) on nodal density
  tet_tgv_curved     : [0,2pi]^3, 16^3 x 6 = 24576 tetrahedra, sine warp, p in {2,4,6}, TGV Ma = 0.1
  tet_tgv_adjoint    : [0,2pi]^3, 8^3 x 6 = 3072 tetrahedra, p = 3, TGV + seeded N(0,1e-3) on modes
Smaller M gives the same workload family at test sizes.
"""
import numpy as np
from .mesh import periodic_tri_mesh, periodic_tet_mesh, mapping_nodes, warp_tri_sine, warp_tet_sine
from . import states

CONFIGS = {
    "tri_vortex_affine": dict(dim=2, M=8, L=2 * np.pi, p=2, warp=False, state="vortex"),
    "tri_vortex_curved": dict(dim=2, M=64, L=1.0, p=4, warp=True, state="vortex"),
    "tet_tgv_curved": dict(dim=3, M=16, L=2 * np.pi, p=4, warp=True, state="tgv"),
    "tet_tgv_adjoint": dict(dim=3, M=8, L=2 * np.pi, p=3, warp=True, state="tgv"),
}


def config_mesh(dim, M, L, p, warp):
    """Mesh and degree-p mapping nodes of a periodic split-Cartesian mesh."""
    if dim == 2:
        mesh = periodic_tri_mesh(M, L)
        w = warp_tri_sine(L) if warp else None
    else:
        mesh = periodic_tet_mesh(M, L)
        w = warp_tet_sine(L) if warp else None
    return mesh, mapping_nodes(mesh, p, w)


def config_state_fn(dim, L, state):
    if state == "vortex":
        return lambda x: states.isentropic_vortex(x, (L / 2, L / 2), L)
    if state == "tgv":
        return lambda x: states.taylor_green(x, 0.1)
    if state == "density_wave":
        return lambda x: states.density_wave(x, L)
    raise ValueError(state)
