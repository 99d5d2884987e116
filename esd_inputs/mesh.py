"""Split-Cartesian periodic meshes of triangles and tetrahedra (Section 7.3).

Each square is split into two triangles and each cube into six tetrahedra
(Kuhn split: all six share the cube's main diagonal, so the split is
conforming across cells and across the periodic boundary).  Tetrahedron
vertices are ordered by ascending global vertex id (ids taken from the
periodically wrapped lattice index), and the first two local vertices are
swapped when that ordering is negatively oriented.  With that ordering every
facet's collapse vertex (local v4 for F1..F3, local v3 for F4) is the facet
vertex of largest id, seen identically from both sides of the facet, which is
the orientation rule of Sherwin & Karniadakis / Warburton et al. that Remark 5
(conforming facets, Assumption 2) relies on.  Triangles keep counter-clockwise
order; their Gauss facet nodes are symmetric, so no further rule is needed.
"""
from dataclasses import dataclass
import itertools
import numpy as np

REF_VERTICES = {
    2: np.array([[-1.0, -1.0], [1.0, -1.0], [-1.0, 1.0]]),
    3: np.array([[-1.0, -1.0, -1.0], [1.0, -1.0, -1.0], [-1.0, 1.0, -1.0], [-1.0, -1.0, 1.0]]),
}
LOCAL_FACETS = {
    2: [(0, 1), (1, 2), (0, 2)],
    3: [(0, 1, 3), (1, 2, 3), (0, 2, 3), (0, 1, 2)],
}


@dataclass
class Mesh:
    dim: int
    L: float
    M: int
    verts: np.ndarray      # [n_elem, dim+1, dim] physical vertex positions (unwrapped)
    nbr_elem: np.ndarray   # [n_elem, n_facets] int32
    nbr_face: np.ndarray   # [n_elem, n_facets] int8

    @property
    def n_elem(self):
        return self.verts.shape[0]


def lattice_nodes(dim, P):
    """Equispaced lattice of degree P on the reference simplex, first index fastest."""
    pts = []
    if dim == 2:
        for j in range(P + 1):
            for i in range(P + 1 - j):
                pts.append((-1.0 + 2.0 * i / P, -1.0 + 2.0 * j / P))
    else:
        for k in range(P + 1):
            for j in range(P + 1 - k):
                for i in range(P + 1 - j - k):
                    pts.append((-1.0 + 2.0 * i / P, -1.0 + 2.0 * j / P, -1.0 + 2.0 * k / P))
    return np.array(pts)


def _connect(elem_vids, dim):
    """Neighbour (element, facet) for every facet, matching facets by vertex-id set."""
    n = len(elem_vids)
    nf = dim + 1
    nbr_e = -np.ones((n, nf), dtype=np.int32)
    nbr_f = -np.ones((n, nf), dtype=np.int8)
    seen = {}
    for e in range(n):
        for f, loc in enumerate(LOCAL_FACETS[dim]):
            key = tuple(sorted(int(elem_vids[e][v]) for v in loc))
            if key in seen:
                e2, f2 = seen.pop(key)
                nbr_e[e, f], nbr_f[e, f] = e2, f2
                nbr_e[e2, f2], nbr_f[e2, f2] = e, f
            else:
                seen[key] = (e, f)
    if seen:
        raise ValueError("mesh has unmatched facets")
    return nbr_e, nbr_f


def periodic_tri_mesh(M, L=1.0):
    """2*M*M counter-clockwise triangles on the periodic square [0,L]^2 (M >= 3)."""
    if M < 3:
        raise ValueError("periodic meshes need M >= 3 so that facets are identified uniquely")
    h = L / M
    verts, vids = [], []
    for j in range(M):
        for i in range(M):
            c = [(i, j), (i + 1, j), (i + 1, j + 1), (i, j + 1)]
            for tri in ((0, 1, 2), (0, 2, 3)):
                idx = [c[t] for t in tri]
                verts.append([[a * h, b * h] for a, b in idx])
                vids.append([(a % M) + M * (b % M) for a, b in idx])
    verts = np.array(verts)
    nbr_e, nbr_f = _connect(vids, 2)
    return Mesh(2, L, M, verts, nbr_e, nbr_f)


def periodic_tet_mesh(M, L=1.0):
    """6*M^3 tetrahedra (Kuhn split) on the periodic cube [0,L]^3 (M >= 3), oriented as above."""
    if M < 3:
        raise ValueError("periodic meshes need M >= 3 so that facets are identified uniquely")
    h = L / M
    verts, vids = [], []
    eye = np.eye(3, dtype=int)
    for k in range(M):
        for j in range(M):
            for i in range(M):
                base = np.array([i, j, k])
                for perm in itertools.permutations(range(3)):
                    path = [base.copy()]
                    cur = base.copy()
                    for ax in perm:
                        cur = cur + eye[ax]
                        path.append(cur.copy())
                    ids = [int((p[0] % M) + M * ((p[1] % M) + M * (p[2] % M))) for p in path]
                    order = sorted(range(4), key=lambda t: ids[t])
                    P = [path[t] * h for t in order]
                    I = [ids[t] for t in order]
                    det = np.linalg.det(np.array([P[1] - P[0], P[2] - P[0], P[3] - P[0]], dtype=float))
                    if det < 0:
                        P[0], P[1] = P[1], P[0]
                        I[0], I[1] = I[1], I[0]
                    verts.append(np.array(P, dtype=float))
                    vids.append(I)
    verts = np.array(verts)
    nbr_e, nbr_f = _connect(vids, 3)
    return Mesh(3, L, M, verts, nbr_e, nbr_f)


def mapping_nodes(mesh, P, warp=None):
    """Physical positions of the degree-P lattice nodes of every element: [n_elem, N*_P, dim].

    The straight-sided element is the affine image of the reference simplex
    (reference vertex k -> physical vertex k); ``warp`` (a function of an
    [..., dim] array) then perturbs the node positions (Section 7.3).
    """
    lat = lattice_nodes(mesh.dim, P)                   # [n, dim]
    bary = (lat + 1.0) / 2.0                           # weights of v2.. relative to v1
    v0 = mesh.verts[:, :1, :]                          # [E,1,dim]
    edges = mesh.verts[:, 1:, :] - v0                  # [E,dim,dim]
    x = v0 + np.einsum("nk,ekd->end", bary, edges)
    if warp is not None:
        x = warp(x)
    return np.ascontiguousarray(x)


def warp_tri_sine(L, amp=0.05):
    """x + amp*L*sin(pi x/L) sin(pi y/L) in both components (vanishes on the boundary)."""
    def f(x):
        s = amp * L * np.sin(np.pi * x[..., 0] / L) * np.sin(np.pi * x[..., 1] / L)
        return x + s[..., None]
    return f


def warp_tet_sine(L, amp=0.05):
    """x_k + amp*L*sin(2 pi x1/L) sin(2 pi x2/L) sin(2 pi x3/L), k = 1..3 (periodic)."""
    def f(x):
        s = amp * L * (np.sin(2 * np.pi * x[..., 0] / L) * np.sin(2 * np.pi * x[..., 1] / L)
                       * np.sin(2 * np.pi * x[..., 2] / L))
        return x + s[..., None]
    return f
