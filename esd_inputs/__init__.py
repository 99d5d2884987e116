"""Seeded synthetic inputs shared by the oracle-side tests and the CUDA path.

This module generates *inputs only*: split-Cartesian periodic meshes (vertex
positions, connectivity, curved mapping-node positions), analytic initial
conditions evaluated at caller-supplied physical points, and seeded random
perturbations.  It holds none of the discretisation's arithmetic (no
quadrature, no basis, no operators, no fluxes).

Conventions shared with the C ABI (``include/esd.h``):

* Reference simplex vertices: triangle (-1,-1), (1,-1), (-1,1);
  tetrahedron (-1,-1,-1), (1,-1,-1), (-1,1,-1), (-1,-1,1)  (Section 3.1, 3.2).
* Local facets (Section 3.1, 3.2): triangle  F1 = {v1,v2} (xi2=-1), F2 = {v2,v3}
  (xi1+xi2=0), F3 = {v1,v3} (xi1=-1); tetrahedron F1 = {v1,v2,v4} (xi2=-1),
  F2 = {v2,v3,v4} (xi1+xi2+xi3=-1), F3 = {v1,v3,v4} (xi1=-1), F4 = {v1,v2,v3}
  (xi3=-1).
* Mapping nodes (Eq. for the polynomial mapping, Section 4.1) are the
  equispaced lattice of degree P on the reference simplex, ordered with the
  first index fastest:  triangle  for j in 0..P, for i in 0..P-j:
  xi = (-1+2i/P, -1+2j/P);  tetrahedron  for k, for j, for i with i+j+k <= P.
"""
from .mesh import (REF_VERTICES, LOCAL_FACETS, lattice_nodes, periodic_tri_mesh,
                   periodic_tet_mesh, mapping_nodes, warp_tri_sine, warp_tet_sine, Mesh)
from .states import (isentropic_vortex, taylor_green, density_wave, conservative_from_primitive,
                     seeded_uniform, seeded_normal, max_wave_speed_sampled)
from .configs import config_mesh, config_state_fn, CONFIGS
