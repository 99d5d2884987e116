"""The boundary is a C ABI: a C99 program compiled with gcc against include/esd.h links
with libesd.so and calls it (entry points that need no GPU), on the CPU."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
LIB_DIR = os.path.join(ROOT, "paper_2312_07874_gb300")
LIB = os.path.join(LIB_DIR, "libesd.so")

pytestmark = pytest.mark.skipif(not os.path.exists(LIB) or shutil.which("gcc") is None,
                                reason="libesd.so not built or no gcc")


def test_c99_program_links_and_calls(tmp_path):
    exe = tmp_path / "abi_check"
    cmd = ["gcc", "-std=c99", "-Wall", "-Wextra", "-Werror", "-pedantic",
           "-I" + os.path.join(ROOT, "include"), os.path.join(ROOT, "tests", "c_abi", "abi_check.c"),
           "-L" + LIB_DIR, "-lesd", "-Wl,-rpath," + LIB_DIR, "-o", str(exe)]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    out = dict(line.split(" ", 1) for line in r.stdout.strip().splitlines())
    q, n = 4, 5
    assert int(out["n_modes"]) == 35                       # C(p + 3, 3)
    assert int(out["n_vol_nodes"]) == n ** 3
    assert int(out["n_facet_nodes"]) == n ** 2
    assert int(out["vol_pairs"]) == 3 * q * n ** 3 // 2     # line pairs, one flux per pair
    assert int(out["facet_pairs"]) == 3 * n ** 3 + n ** 4   # faces 1-3 on lines, face 4 on planes
    assert int(out["paper_flux_count"]) == 4 * n ** 4      # Eq. (num_fluxes), tetrahedra
    assert int(out["unsupported_degree"]) == -7            # ESD_ERR_UNSUPPORTED
    assert int(out["null_output"]) == -1
    assert int(out["null_mesh_rhs"]) == -1
    assert int(out["layouts"]) == 0
    assert out["status_string"].startswith("ESD_ERR_STATE")
