"""Host logic of element partitions (paper_2312_07874_gb300.partition) on the CPU: the
partition descriptions and exchange lists built by `split`, and the trace exchange between
torch.distributed ranks (gloo, 2 and 3 ranks) with export / import functions that stand in
for the library's kernels."""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from esd_inputs.configs import config_mesh  # noqa: E402
from paper_2312_07874_gb300.partition import split  # noqa: E402


def _owners(mesh, X, kind, P):
    E = X.shape[0]
    if kind == "round_robin":
        return np.arange(E) % P
    c = X.mean(axis=1)[:, 0]               # slabs of the first coordinate
    edges = np.quantile(c, np.linspace(0, 1, P + 1)[1:-1])
    return np.searchsorted(edges, c, side="right")


@pytest.mark.parametrize("dim,M", [(2, 4), (3, 3)])
@pytest.mark.parametrize("kind,P", [("slab", 2), ("round_robin", 3), ("slab", 4)])
def test_split_descriptions_and_exchange_lists(dim, M, kind, P):
    mesh, X = config_mesh(dim, M, 2 * np.pi, 2, True)
    ne, nf = np.asarray(mesh.nbr_elem), np.asarray(mesh.nbr_face)
    owner = _owners(mesh, X, kind, P)
    parts = split(ne, nf, owner)
    assert len(parts) == P
    # every element is local to exactly one partition
    allloc = np.sort(np.concatenate([p.local for p in parts]))
    assert np.array_equal(allloc, np.arange(X.shape[0]))
    Nf = ne.shape[1]
    for r, p in enumerate(parts):
        ids = p.elements()
        assert np.all(owner[p.local] == r) and np.all(owner[p.ghosts] != r)
        # ghosts grouped by owner, each group contiguous and described by recv
        for q, (first, n) in p.recv.items():
            assert np.all(owner[p.ghosts[first:first + n]] == q)
        assert sum(n for _, n in p.recv.values()) == p.n_ghost
        # local facets: same neighbour (global id) and face as the global mesh; symmetric
        for e in range(p.n_local):
            for z in range(Nf):
                e2, z2 = p.nbr_elem[e, z], p.nbr_face[e, z]
                assert 0 <= e2 < len(ids)
                assert ids[e2] == ne[p.local[e], z] and z2 == nf[p.local[e], z]
                assert p.nbr_elem[e2, z2] == e and p.nbr_face[e2, z2] == z
        # every ghost borders a local element (no superfluous ghosts)
        touched = set(p.nbr_elem[:p.n_local].ravel().tolist())
        assert all(p.n_local + g in touched for g in range(p.n_ghost))
        # ghost facets facing no local element are marked -1
        for g in range(p.n_ghost):
            for z in range(Nf):
                if owner[ne[p.ghosts[g], z]] != r:
                    assert p.nbr_elem[p.n_local + g, z] == -1
        # what q sends to r is exactly r's ghost range from q, in that order
        for q, (first, n) in p.recv.items():
            sent = parts[q].local[parts[q].send[r]]
            assert np.array_equal(sent, p.ghosts[first:first + n])
    # map nodes follow the description's element order
    p0 = parts[0]
    assert np.array_equal(p0.map_nodes(X)[p0.n_local:], X[p0.ghosts])


def test_split_rejects_empty_partition():
    mesh, X = config_mesh(2, 3, 1.0, 1, False)
    owner = np.zeros(X.shape[0], dtype=np.int64)
    owner[0] = 2                              # partition 1 is empty
    with pytest.raises(ValueError):
        split(mesh.nbr_elem, mesh.nbr_face, owner)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


PER = 5   # doubles per element of the stand-in messages


def _rank_main(rank, world, port, out_path):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    from paper_2312_07874_gb300.partition import exchange_dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    mesh, X = config_mesh(3, 3, 2 * np.pi, 1, False)
    owner = _owners(mesh, X, "round_robin", world)
    part = split(mesh.nbr_elem, mesh.nbr_face, owner)[rank]
    ghost_rows = torch.full((part.n_ghost, PER), np.nan, dtype=torch.float64)

    def export(elems, buf):    # stand-in for esd_part_export: global id and a per-column tag
        g = torch.from_numpy(part.local)[elems].to(torch.float64)
        buf.copy_(g[:, None] * 10.0 + torch.arange(PER, dtype=torch.float64)[None, :])

    def import_(buf, first, n):   # stand-in for esd_part_import
        ghost_rows[first:first + n] = buf

    exchange_dist(part, export, import_, PER, dist)
    expect = torch.from_numpy(part.ghosts).to(torch.float64)[:, None] * 10.0 + \
        torch.arange(PER, dtype=torch.float64)[None, :]
    ok = bool(torch.equal(ghost_rows, expect))
    with open(f"{out_path}.{rank}", "w") as f:
        f.write(f"{int(ok)} {part.n_ghost}")
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_trace_exchange_over_gloo_ranks(tmp_path, world):
    """Each rank holds one partition; after one exchange every ghost row holds the message
    of the right element from the right rank."""
    import torch.multiprocessing as mp
    out = str(tmp_path / "r")
    mp.start_processes(_rank_main, args=(world, _free_port(), out), nprocs=world, start_method="spawn", join=True)
    for r in range(world):
        ok, ng = open(f"{out}.{r}").read().split()
        assert ok == "1" and int(ng) > 0
