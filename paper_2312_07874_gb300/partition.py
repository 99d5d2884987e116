"""Element partitions of a mesh and the facet-trace exchange between them.

The semi-discretisation couples elements only through the interface flux at shared facets,
so a partitioned mesh needs, per right-hand side, one exchange of the facet traces of the
elements that border another partition (and, per VJP, one exchange of the interface
cotangents).  `split` builds, from the global connectivity and an owner per element, each
partition's mesh description (local elements, then ghosts grouped by owning partition) and
the send lists / receive ranges of the exchange.  The exchange itself runs either between
partition meshes held by one process (`exchange_local`, device buffers on one GPU) or
between ranks of torch.distributed (`exchange_dist`), with the export and import steps
passed in as functions so that the host logic runs without a GPU.

Host-side bookkeeping only: the traces are gathered and scattered by the library's
esd_part_export / esd_part_import kernels.
"""
import numpy as np


class Part:
    """One partition.

    local:   global ids of the local elements, in local order (0 .. n_local-1)
    ghosts:  global ids of the ghosts, in ghost order (element n_local + g of the description),
             grouped by owning partition in increasing order
    nbr_elem, nbr_face: the description's connectivity over local elements then ghosts;
             ghost facets that face no local element hold -1
    recv:    {q: (first, n)}: ghosts first .. first+n-1 come from partition q
    send:    {q: local indices}: local elements that partition q holds as ghosts, in q's ghost order
    """

    def __init__(self, rank, local, ghosts, nbr_elem, nbr_face, recv, send):
        self.rank, self.local, self.ghosts = rank, local, ghosts
        self.nbr_elem, self.nbr_face, self.recv, self.send = nbr_elem, nbr_face, recv, send

    @property
    def n_local(self):
        return len(self.local)

    @property
    def n_ghost(self):
        return len(self.ghosts)

    def elements(self):
        """Global ids of the description's elements: local, then ghosts."""
        return np.concatenate([self.local, self.ghosts])

    def map_nodes(self, X):
        """The description's mapping nodes, gathered from the global [n_elem][N_p][dim] X."""
        return np.ascontiguousarray(X[self.elements()])


def split(nbr_elem, nbr_face, owner):
    """Partitions of a mesh with connectivity nbr_elem / nbr_face ([n_elem][N_f]) and
    owner[e] in 0..P-1.  Returns the list of P Part objects."""
    nbr_elem = np.asarray(nbr_elem, dtype=np.int64)
    nbr_face = np.asarray(nbr_face, dtype=np.int64)
    owner = np.asarray(owner, dtype=np.int64)
    E, Nf = nbr_elem.shape
    P = int(owner.max()) + 1
    parts = []
    for r in range(P):
        local = np.flatnonzero(owner == r)
        if len(local) == 0:
            raise ValueError(f"partition {r} has no elements")
        nb = nbr_elem[local]
        gh = np.unique(nb[owner[nb] != r])
        ghosts = np.concatenate([gh[owner[gh] == q] for q in range(P)]) if len(gh) else gh
        index = -np.ones(E, dtype=np.int64)
        index[local] = np.arange(len(local))
        index[ghosts] = len(local) + np.arange(len(ghosts))
        ne = np.full((len(local) + len(ghosts), Nf), -1, dtype=np.int64)
        nf = np.full((len(local) + len(ghosts), Nf), -1, dtype=np.int64)
        ne[:len(local)] = index[nb]
        nf[:len(local)] = nbr_face[local]
        if len(ghosts):
            gn = nbr_elem[ghosts]
            faces_local = owner[gn] == r           # ghost facets that face a local element
            ne[len(local):][faces_local] = index[gn[faces_local]]
            nf[len(local):][faces_local] = nbr_face[ghosts][faces_local]
        recv = {}
        for q in range(P):
            sel = np.flatnonzero(owner[ghosts] == q)
            if len(sel):
                recv[q] = (int(sel[0]), len(sel))
        parts.append(Part(r, local, ghosts, ne.astype(np.int32), nf.astype(np.int8), recv, {}))
    for r, part in enumerate(parts):   # what r sends to q: q's ghosts owned by r, in q's order
        for q, other in enumerate(parts):
            if q == r or r not in other.recv:
                continue
            first, n = other.recv[r]
            gl = other.ghosts[first:first + n]
            pos = np.searchsorted(part.local, gl)
            part.send[q] = pos.astype(np.int64)
    return parts


class LocalExchange:
    """A planned exchange between partition meshes of this process (one GPU): the element
    lists of every ordered pair (q -> r) and their message buffers are set up once on the
    device, and each call only launches the export and import kernels (q exports the traces
    of r's ghosts it owns into a buffer, r imports them into its ghost range).  kind:
    ESD_TRACE_STATES or ESD_TRACE_COTANGENTS."""

    def __init__(self, meshes, parts, kind):
        import torch
        from . import ESD_TRACE_STATES, esd_part_info
        self.meshes, self.kind, self.plan = meshes, kind, []
        for r, part in enumerate(parts):
            for q, (first, n) in part.recv.items():
                _, per_s, per_c = esd_part_info(meshes[q].handle)
                per = per_s if kind == ESD_TRACE_STATES else per_c
                elems = torch.from_numpy(parts[q].send[r]).to("cuda")
                buf = torch.empty((n, per), dtype=torch.float64, device="cuda")
                self.plan.append((q, r, elems, buf, first, n))

    def __call__(self, stream=None):
        from . import esd_part_export, esd_part_import
        for q, r, elems, buf, first, n in self.plan:
            esd_part_export(self.meshes[q].handle, self.kind, elems, buf, stream)
            esd_part_import(self.meshes[r].handle, self.kind, buf, first, n, stream)


def exchange_local(meshes, parts, kind, stream=None):
    """One exchange between partition meshes of this process (a LocalExchange used once)."""
    LocalExchange(meshes, parts, kind)(stream)


def exchange_dist(part, export, import_, per, dist, device="cpu", dtype=None):
    """One exchange between ranks of torch.distributed, rank r holding partition `part`
    (part.rank == r): for every peer, the messages are exported with export(elems, buf)
    (elems: local indices as an int64 tensor on `device`, buf: [n][per] float64), sent with
    point-to-point calls, and imported with import_(buf, first, n).  With the GPU library,
    export / import wrap esd_part_export / esd_part_import and the process group is NCCL;
    the host logic is the same with gloo and CPU buffers."""
    import torch
    dtype = dtype or torch.float64
    ops, recvs = [], []
    for q, elems_np in sorted(part.send.items()):
        elems = torch.from_numpy(elems_np).to(device)
        buf = torch.empty((len(elems_np), per), dtype=dtype, device=device)
        export(elems, buf)
        ops.append(dist.P2POp(dist.isend, buf, q))
    for q, (first, n) in sorted(part.recv.items()):
        buf = torch.empty((n, per), dtype=dtype, device=device)
        recvs.append((buf, first, n))
        ops.append(dist.P2POp(dist.irecv, buf, q))
    if ops:
        for req in dist.batch_isend_irecv(ops):
            req.wait()
    for buf, first, n in recvs:
        import_(buf, first, n)
