"""Benchmark: FP64 DOF-residual updates/s of the entropy-stable tensor-product DSEM.

Workload (one GPU): periodic [0,2pi]^3, 16^3 x 6 = 24576 curved tetrahedra (sine
warp, amplitude 0.05 L), degree p = 4 (N_p* = 35 modes, N_c = 5), Taylor-Green
vortex at Mach 0.1 with Lax-Friedrichs interface dissipation, FP64.  One "step" is
one classical RK4 step (four evaluations of d u~/dt, every row of the hot path),
replayed from a CUDA graph.  DOF = n_elem * N_p* * N_c; value = 4 * DOF per step.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the oracle (plain numpy, test infrastructure) on the host on a
bounded sample of the same workload.  Under torchrun each rank runs an independent
replica (weak scaling, no collective); rank 0 prints one JSON line.
"""
import argparse
import json
import os
import subprocess
import sys
import time

# the oracle's CPU baseline runs single-threaded: pin every BLAS/OpenMP pool before numpy loads
for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "BLIS_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import esd_inputs as I  # noqa: E402

WORKLOAD = dict(dim=3, M=16, L=2 * np.pi, p=4, state="tgv", flux="LF")
METRIC = "FP64 DOF-residual updates/s at p=4 tets (% FP64 roofline); adjoint/forward ratio"
# nominal FP64 rate of GB300: 2 FMA lanes per clock per SM x 152 SMs x 2.07 GHz x 2 flops
NOMINAL_FP64_TFLOPS = 2 * 152 * 2.07e9 * 2 / 1e12
UNIT = "DOF-residual updates/s"


# ---------------------------------------------------------------------------------
# algorithmic FP64 flop counts (formula level: add/mul/div = 1, FMA = 2)
# ---------------------------------------------------------------------------------
def pair_flops(D):
    """One directional two-point flux (Section 7.2) plus its accumulation to both ends."""
    NC = D + 2
    log_means = 2 * 12            # s, d, f = d/s, u = f^2, 3-term Horner series (6), division, select
    dots = 3 * (2 * D - 1)        # v^-.n, v^+.n, v^-.v^+
    f_rho = 3                     # rho_ln * (vn^- + vn^+)/2
    p_avg = 2
    momentum = 5 * D              # f_rho {{v_k}} + {{p}} n_k
    energy = 9
    accumulate = 2 * NC
    return log_means + dots + f_rho + p_avg + momentum + energy + accumulate


def interface_flops(D):
    NC = D + 2
    flux = pair_flops(D) - 2 * NC
    lf = 2 * (2 * D - 1) + 5 + 2 * (2 * D + 2) + 2 * D + 3 * NC   # speeds, jumps of U, damping
    return flux + lf + NC                                          # times B J


def transform_fmas(D, p):
    n = p + 1
    Np = (p + 1) * (p + 2) // 2 if D == 2 else (p + 1) * (p + 2) * (p + 3) // 6
    S12 = (p + 1) * (p + 2) // 2
    Nq = n ** D
    if D == 2:
        V = Np * n + Nq * (p + 1)
        VT = (p + 1) * n * n + Np * n
    else:
        V = Np * n + S12 * n * n + Nq * (p + 1)
        VT = (p + 1) * n ** 3 + S12 * n * n + Np * n
    return V, VT, Nq, Np


def residual_kernel_flops(D, p):
    """Per element: interface flux, volume + facet-correction pairs, lift, weight-adjusted inverse."""
    n = p + 1
    NC = D + 2
    V, VT, Nq, Np = transform_fmas(D, p)
    vol_pairs = D * n ** (D - 1) * (p * (p + 1) // 2)
    fac_pairs = 3 * n * n if D == 2 else 3 * n ** 3 + n ** 4
    Nfn = (D + 1) * n ** (D - 1)
    lift = (7 * Nq) if D == 2 else (2 * n ** 3 + 9 * Nq)
    reduce4 = 0 if D == 2 else NC * n * n * (n - 1)
    dudt = 2 * (VT + V + VT) + Nq
    return ((vol_pairs + fac_pairs) * pair_flops(D) + Nfn * interface_flops(D)
            + NC * (lift + dudt) + reduce4), vol_pairs + fac_pairs + Nfn


def skew_node_flux_flops(D, nc):
    """f_m(u) at one node: Euler (reciprocal with two Newton steps, v, p, the D flux
    vectors), or a_m u for linear advection."""
    if nc == 1:
        return D
    return 9 + 3 * D + 4 + D * (1 + 2 * D + 1)


def skew_residual_flops(D, p, nc):
    """Per element, the skew-symmetric residual kernel (Eq. (rhs_skew)): u = V u~, the line
    pairs (one FMA per ordered pair, direction and variable), the node fluxes formed in each
    phase and for the facet traces, the facet terms and lifts, d u~/dt = [V^T (W/J) V] V^T r."""
    n = p + 1
    V, VT, Nq, Np = transform_fmas(D, p)
    T = n ** (D - 1)
    pairs = 2 * D * T * n * (n - 1) * D * nc
    flux_evals = D * Nq + (3 * T * n if D == 3 else 3 * n * n) + (T * n if D == 3 else 0)
    fluxes = flux_evals * skew_node_flux_flops(D, nc)
    traces = 2 * D * nc * ((3 * T * n) + (2 * T * n if D == 3 else 0))
    Nfn = (D + 1) * n ** (D - 1)
    fstar = Nfn * ((interface_flops(D) if nc > 1 else 12) + 2 * D * nc + 2 * nc)
    lift = 2 * nc * ((3 * T * n) + (2 * T * n if D == 3 else 0))
    dudt = 2 * nc * (V + VT + V + VT) + nc * Nq
    return pairs + fluxes + traces + fstar + lift + dudt


def project_kernel_flops(D, p):
    n = p + 1
    NC = D + 2
    V, VT, Nq, Np = transform_fmas(D, p)
    Nfn = (D + 1) * n ** (D - 1)
    R = 6 * n * n if D == 2 else 10 * n ** 3       # facet extrapolation R (face 4 in two stages)
    entropy_vars = Nq * (4 * D + 16)          # primitive recovery, two logs, W(u), times W J
    cons_from_w = (Nq + Nfn) * (3 * D + 14)   # U(w): log, exp, primitive fields
    return NC * (2 * (3 * V + 2 * VT) + Nq + R) + entropy_vars + cons_from_w


# ---------------------------------------------------------------------------------
def reduce_max(x, device):
    """Maximum of a per-rank float over all ranks of the default process group (the
    slowest rank's time); x itself when no group is initialised."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def build_inputs(torch, E, dev):
    w = WORKLOAD
    mesh, X = I.config_mesh(w["dim"], w["M"], w["L"], w["p"], True)
    if w["M"] != 16:
        print(f"note: reduced mesh M={w['M']} (profiling case, not a bench line)", file=sys.stderr)
    gm = E.Mesh(w["dim"], w["p"], X, mesh.nbr_elem, mesh.nbr_face, flux=w["flux"])
    x = gm.volume_nodes()
    un = np.ascontiguousarray(np.transpose(I.taylor_green(x, 0.1), (0, 2, 1)))
    u0 = gm.l2_project(torch.from_numpy(un).to(dev))
    torch.cuda.synchronize()
    lam = I.max_wave_speed_sampled(lambda y: I.taylor_green(y, 0.1), 3, w["L"])
    dt = 0.1 * (w["L"] / w["M"]) / (lam * (2 * w["p"] + 1))
    return mesh, gm, u0, dt


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        # the raw samples go to a scratch file (BENCH_CLOCKS_DIR, default the system temp dir)
        import tempfile
        d = os.environ.get("BENCH_CLOCKS_DIR") or tempfile.gettempdir()
        self.path = os.path.join(d, f"esd_bench_clocks_rank{index}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [s.strip() for s in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def profiled_range(torch, on):
    """Opens (on) or closes the launch range that `ncu --profile-from-start off` captures:
    the timed RK4 steps and the timed VJP calls.  Without a profiler attached it has no
    effect."""
    (torch.cuda.profiler.start if on else torch.cuda.profiler.stop)()


def run_ours(args):
    import torch
    import paper_2312_07874_gb300 as E
    rank, world, local = dist_env()
    # the oracle on all host cores runs first: its workers are forked before any CUDA call
    all_cores = None
    if world == 1 and args.cpu_seconds > 0:
        all_cores = cpu_baseline_all_cores()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    mesh, gm, u0, dt = build_inputs(torch, E, dev)
    # launch shapes timed on this mesh (setup, outside the timed region)
    info = gm.info if args.no_autotune else gm.autotune(u0)
    D, p = WORKLOAD["dim"], WORKLOAD["p"]
    nE = info["n_elem"]
    dof = nE * info["n_modes"] * info["n_c"]
    stream = torch.cuda.Stream(device=dev)
    u = u0.clone()

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    # ---- warm-up (graph capture happens on the first call) ----
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            gm.rk_step(u, dt)
    stream.synchronize()
    gm.check()
    # ---- timed region: K RK4 steps ----
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        profiled_range(torch, True)
        ev0.record(stream)
        for _ in range(args.steps):
            gm.rk_step(u, dt)
        ev1.record(stream)
        profiled_range(torch, False)
    stream.synchronize()
    barrier()
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1) / args.steps
    clk = clocks.stop()
    gm.check()
    ms = reduce_max(ms, dev)
    value = 4.0 * dof * world / (ms * 1e-3)

    # ---- dominant kernel (residual) alone, on the launching stream ----
    out = torch.empty_like(u)
    nrep = max(3, args.steps)
    with torch.cuda.stream(stream):
        E.esd_launch_stage(gm.handle, 0, u, None, stream)
        E.esd_launch_stage(gm.handle, 1, None, out, stream)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(nrep):
            E.esd_launch_stage(gm.handle, 1, None, out, stream)
        b.record(stream)
        c, d = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        c.record(stream)
        for _ in range(nrep):
            E.esd_launch_stage(gm.handle, 0, u, None, stream)
        d.record(stream)
    stream.synchronize()
    res_ms = a.elapsed_time(b) / nrep
    proj_ms = c.elapsed_time(d) / nrep
    # adjoint / forward: esd_rhs_vjp against esd_rhs on the same state (same stream)
    cot = torch.empty_like(u).normal_(generator=torch.Generator(device=dev).manual_seed(4))
    grad = torch.empty_like(u)
    with torch.cuda.stream(stream):
        E.esd_rhs(gm.handle, u, out, stream)
        E.esd_rhs_vjp(gm.handle, u, cot, grad, stream)
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        for _ in range(nrep):
            E.esd_rhs(gm.handle, u, out, stream)
        f1.record(stream)
        g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        profiled_range(torch, True)
        g0.record(stream)
        for _ in range(nrep):
            E.esd_rhs_vjp(gm.handle, u, cot, grad, stream)
        g1.record(stream)
        profiled_range(torch, False)
    stream.synchronize()
    fwd_ms = f0.elapsed_time(f1) / nrep
    adj_ms = g0.elapsed_time(g1) / nrep
    # reverse mode with the forward's tape kept (esd_rhs_save) and read by the VJP
    # (esd_rhs_vjp_saved): the adjoint does not recompute the entropy projection
    tape = gm.empty_tapes()
    with torch.cuda.stream(stream):
        E.esd_rhs_save(gm.handle, u, out, tape, stream)
        E.esd_rhs_vjp_saved(gm.handle, u, tape, cot, grad, stream)
        h0, h1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        h0.record(stream)
        for _ in range(nrep):
            E.esd_rhs_save(gm.handle, u, out, tape, stream)
        h1.record(stream)
        k0, k1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        k0.record(stream)
        for _ in range(nrep):
            E.esd_rhs_vjp_saved(gm.handle, u, tape, cot, grad, stream)
        k1.record(stream)
    stream.synchronize()
    fwd_save_ms = h0.elapsed_time(h1) / nrep
    adj_saved_ms = k0.elapsed_time(k1) / nrep
    del tape
    rflops, npairs = residual_kernel_flops(D, p)
    achieved = rflops * nE / (res_ms * 1e-3)
    peak = E.esd_measure_fp64_peak(stream)
    traffic = None
    tpath = os.path.join(ROOT, "profiles", "residual_kernel_tet_p4_traffic.json")
    if os.path.exists(tpath):
        tj = json.load(open(tpath))
        if tj.get("kernel_source_sha256") == _kernel_hash():
            # captured on tetrahedra at p = 4; traffic grows in proportion to the elements
            traffic = tj["dram_bytes_per_element"] * nE
    pflops = project_kernel_flops(D, p)

    # ---- end to end through the public API: pinned H2D, RK4 step, D2H ----
    host_in = u0.cpu().pin_memory()
    host_out = torch.empty_like(host_in).pin_memory()
    ue = torch.empty_like(u)
    with torch.cuda.stream(stream):
        for _ in range(2):
            ue.copy_(host_in, non_blocking=True)
            gm.rk_step(ue, dt)
            host_out.copy_(ue, non_blocking=True)
    stream.synchronize()
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        e0.record(stream)
        for _ in range(args.steps):
            ue.copy_(host_in, non_blocking=True)
            gm.rk_step(ue, dt)
            host_out.copy_(ue, non_blocking=True)
        e1.record(stream)
    stream.synchronize()
    e2e_ms = e0.elapsed_time(e1) / args.steps
    e2e_ms = reduce_max(e2e_ms, dev)
    nbytes = host_in.numel() * 8

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded analytic TGV state, no dataset)",
        "config": {"workload": "tet_tgv_curved p=4: periodic [0,2pi]^3, 16^3x6 = 24576 curved tets, TGV Ma=0.1, "
                               "LF interface flux, RK4 step (4 residual evaluations) from a CUDA graph",
                   "n_elem": nE, "p": p, "dof": dof, "dt": dt,
                   "l2": "inputs larger than L2: per step the kernels stream ~1.4 GB of pair tables and states",
                   "parallelism": f"replicas x{world} (independent meshes, no collective)",
                   "launch": {k: info[k] for k in ("elems_per_cta_project", "elems_per_cta_residual")}},
        "roofline": {"bound": "alu", "achieved": achieved / 1e12, "peak": peak / 1e12, "unit": "TFLOP/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "kernel": "residual_kernel<3> (interface flux, line-based flux differencing, facet "
                               "correction, lift, weight-adjusted inverse)",
                     "peak_source": "measured live: FP64 FMA chain (esd_measure_fp64_peak), FMA = 2 flops",
                     "nominal_peak": NOMINAL_FP64_TFLOPS,
                     "frac_of_nominal": achieved / 1e12 / NOMINAL_FP64_TFLOPS,
                     "algorithmic_flops_per_elem": rflops, "kernel_ms": res_ms,
                     "project_kernel_ms": proj_ms, "project_flops_per_elem": pflops},
        "two_point_fluxes_per_s": 4.0 * npairs * nE * world / (ms * 1e-3),
        "paper_flux_count_equivalent_per_s": 4.0 * info["paper_flux_count_per_elem"] * nE * world / (ms * 1e-3),
        "adjoint_forward_ratio": adj_ms / fwd_ms,
        "adjoint_forward_ratio_saved_tape": adj_saved_ms / fwd_save_ms,
        "adjoint": {"rhs_ms": fwd_ms, "rhs_vjp_ms": adj_ms, "rhs_save_ms": fwd_save_ms,
                    "rhs_vjp_saved_ms": adj_saved_ms,
                    "note": "adjoint_forward_ratio: esd_rhs_vjp (recomputes the entropy projection) / esd_rhs; "
                            "_saved_tape: esd_rhs_vjp_saved (reads the forward's tape) / esd_rhs_save"},
        "e2e": {"value": 4.0 * dof * world / (e2e_ms * 1e-3), "unit": UNIT, "ms_per_step": e2e_ms,
                "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes},
        "gpu_launches": 8 * args.steps,
        "clocks": clk,
    }
    if rank == 0:
        # the host baselines are taken at N = 1 only (at N > 1 the other ranks would wait)
        line["cpu_baseline"] = (cpu_baseline(seconds=args.cpu_seconds)
                                if args.cpu_seconds > 0 and world == 1 else None)
        line["cpu_baseline_all_cores"] = all_cores
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()


KERNEL_SOURCES = ("device.cuh", "residual_inst.cuh", "residual_d3.cu", "esd_internal.h")


def _code_tokens(src):
    """C/C++ source without comments, with blank lines, indentation and runs of blanks
    collapsed: a comment or layout edit leaves it unchanged, a code edit changes it."""
    import re
    out, i, n = [], 0, len(src)
    while i < n:
        c = src[i]
        if src.startswith("//", i):
            j = src.find("\n", i)
            i = n if j < 0 else j
            out.append(" ")
        elif src.startswith("/*", i):
            j = src.find("*/", i + 2)
            j = n if j < 0 else j + 2
            out.append("\n" if "\n" in src[i:j] else " ")
            i = j
        elif c in "\"'":
            j = i + 1
            while j < n and src[j] != c:
                j += 2 if src[j] == "\\" else 1
            out.append(src[i:j + 1])
            i = j + 1
        else:
            out.append(c)
            i += 1
    code = re.sub(r"[ \t]+", " ", "".join(out))
    return re.sub(r" ?\n\s*", "\n", code).strip()


def _kernel_hash(read=None):
    """Hash of the code (comments and layout excluded) of residual_kernel<3, N>'s sources;
    the adjoint and projection kernels live elsewhere.  `read(name)` returns a file's text."""
    import hashlib
    read = read or (lambda f: open(os.path.join(ROOT, "paper_2312_07874_gb300", "csrc", f)).read())
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        h.update(_code_tokens(read(f)).encode())
    return h.hexdigest()


# ---------------------------------------------------------------------------------
# oracle on the host (CPU baseline and the reference arm)
# ---------------------------------------------------------------------------------
_ORACLE = {}


def _oracle_setup():
    if "D" not in _ORACLE:
        from oracle.residual import Discretization
        w = WORKLOAD
        mesh, X = I.config_mesh(w["dim"], w["M"], w["L"], w["p"], True)
        D = Discretization(w["dim"], w["p"], X, mesh.nbr_elem, mesh.nbr_face, flux=w["flux"])
        um = np.einsum("ij,i,eic->ecj", D.V, D.ref.w, I.taylor_green(D.geo.x_vol, 0.1))
        _ORACLE.update(D=D, um=um)
    return _ORACLE["D"], _ORACLE["um"]


def _oracle_sample(D, um, n_el):
    """d u~/dt of the sampled elements by the oracle's sparse route (the paper's algorithm):
    entropy projection of the sample and its face neighbours, then the residual."""
    from oracle.residual import Discretization  # noqa: F401
    el = np.arange(n_el)
    t0 = time.perf_counter()
    D.rhs(um, "sparse", elems=el, chunk=n_el)
    return time.perf_counter() - t0


def cpu_baseline(seconds=15.0, n_el=None):
    """Time the oracle as it stands on a bounded sample of the workload's elements."""
    D, um = _oracle_setup()
    n_el = n_el or 16
    t = _oracle_sample(D, um, n_el)
    while t < 0.25 * seconds and n_el < D.E:
        n_el = min(D.E, n_el * 2)
        t = _oracle_sample(D, um, n_el)
    dof = n_el * D.Np * D.Nc
    return {"value": dof / t, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{n_el} of {D.E} elements of the benchmark mesh, one d u~/dt each (sparse route); "
                      f"{t:.1f} s (entropy projection of the sample and its neighbours included)"}


def _oracle_block(args):
    """Worker of cpu_baseline_all_cores: one d u~/dt of elements [k n, (k + 1) n)."""
    k, n = args
    D, um = _ORACLE["D"], _ORACLE["um"]
    el = np.arange(k * n, (k + 1) * n)
    t0 = time.perf_counter()
    D.rhs(um, "sparse", elems=el, chunk=n)
    return time.perf_counter() - t0


def _oracle_pool(n_el):
    """One forked worker per host core (at most 64) and the block size each one takes:
    up to n_el distinct elements.  Fork only in a process that has made no CUDA call."""
    import multiprocessing as mp
    D, _ = _oracle_setup()
    cores = max(1, min(64, len(os.sched_getaffinity(0))))
    n = max(1, min(n_el, D.E // cores))
    return mp.get_context("fork").Pool(cores), cores, n


def _oracle_pool_step(pool, cores, n):
    """Wall time of one d u~/dt of cores x n distinct elements, one block per worker."""
    t0 = time.perf_counter()
    worker_s = pool.map(_oracle_block, [(k, n) for k in range(cores)])
    return time.perf_counter() - t0, max(worker_s)


def cpu_baseline_all_cores(n_el=1536):
    """The same oracle on every host core at once: one forked worker per core, each on its
    own block of up to n_el elements (the elements are independent); value = all sampled
    elements' DOF / wall time.  Must run before the process makes its first CUDA call (the
    workers are forked and run numpy only)."""
    D, _ = _oracle_setup()
    pool, cores, n = _oracle_pool(n_el)
    try:
        wall, slowest = _oracle_pool_step(pool, cores, n)
    finally:
        pool.close()
        pool.join()
    dof = cores * n * D.Np * D.Nc
    return {"value": dof / wall, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{cores} forked workers x {n} distinct elements of the benchmark mesh, one d u~/dt "
                      f"each (sparse route, entropy projection of each block and its neighbours included); "
                      f"{wall:.1f} s wall, slowest worker {slowest:.1f} s"}


def run_reference(args):
    """The oracle as it stands on all host cores (this process makes no CUDA call): each
    step is one d u~/dt of cores x n distinct elements of the benchmark mesh, one block per
    forked worker."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    D, um = _oracle_setup()
    pool, cores, n = _oracle_pool(512)   # ~1 s of oracle work per worker and step
    try:
        for _ in range(args.warmup):
            _oracle_pool_step(pool, cores, n)
        times = [_oracle_pool_step(pool, cores, n)[0] for _ in range(args.steps)]
    finally:
        pool.close()
        pool.join()
    t = float(np.mean(times))
    dof = cores * n * D.Np * D.Nc
    value = dof / t
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded analytic TGV state, no dataset)",
        "impl": "reference",
        "config": {"workload": f"tet_tgv_curved p=4: periodic [0,2pi]^3, {D.E} curved tets, TGV Ma=0.1, LF "
                               f"interface flux (oracle: one d u~/dt of {cores} x {n} elements per step, "
                               f"one block per host core)",
                   "n_elem": D.E, "p": WORKLOAD["p"]},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{cores} forked workers x {n} distinct elements per step, sparse route"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------------
# batched execution: 64 independent meshes, one persistent launch per kernel and degree
# ---------------------------------------------------------------------------------
def batch_mix(seed=5, n=64, small=False):
    """Seeded mix: triangles on uniform 2D grids (2 M^2 in [200, 20000]), tetrahedra from
    uniform cube splits (6 M^3 in [384, 24576]), p uniform in {2..10} for both, vortex or
    Taylor-Green states (about 110 GB of device memory in total).  small=True: the same
    recipe with small meshes only (triangles M in [10, 30], tetrahedra M in [3, 6]), where
    launch overheads are a visible part of a step."""
    rng = np.random.default_rng(seed)
    tri_m, tet_m = ((10, 31), (3, 7)) if small else ((10, 101), (4, 17))
    mix = []
    for i in range(n):
        if i % 2 == 0:
            M = int(rng.integers(*tri_m))
            mix.append((2, M, int(rng.integers(2, 11)), "vortex"))
        else:
            M = int(rng.integers(*tet_m))
            mix.append((3, M, int(rng.integers(2, 11)), "tgv"))
    return mix


def run_batch(args):
    import torch
    import paper_2312_07874_gb300 as E
    dev = torch.device("cuda", 0)
    meshes, states, dts, dof = [], [], [], 0
    t0 = time.time()
    mix = batch_mix(small=args.batch_small)
    for dim, M, p, state in mix:
        L = 2 * np.pi
        mesh, X = I.config_mesh(dim, M, L, p, True)
        gm = E.Mesh(dim, p, X, mesh.nbr_elem, mesh.nbr_face)
        x = gm.volume_nodes()
        f = I.config_state_fn(dim, L, state)
        un = np.ascontiguousarray(np.transpose(f(x), (0, 2, 1)))
        u = gm.l2_project(torch.from_numpy(un).to(dev))
        lam = I.max_wave_speed_sampled(f, dim, L, n=32)
        gm.autotune(u, E.ESD_TUNE_PROJECT | E.ESD_TUNE_RESIDUAL)   # element tiling; the batch inherits it
        meshes.append(gm)
        states.append(u)
        dts.append(0.1 * (L / M) / (lam * (2 * p + 1)))
        dof += gm.n_elem * gm.nc * gm.n_modes
    setup_s = time.time() - t0
    b = E.esd_batch_create([m.handle for m in meshes])
    stream = torch.cuda.Stream(device=dev)
    ua = [u.clone() for u in states]
    ub = [u.clone() for u in states]

    def timed(fn):
        with torch.cuda.stream(stream):
            for _ in range(args.warmup):
                fn()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(args.steps):
                fn()
            e1.record(stream)
        stream.synchronize()
        return e0.elapsed_time(e1) / args.steps

    ms_batch = timed(lambda: E.esd_batch_rk_step(b, ua, dts, stream))
    ms_plain = timed(lambda: [m.rk_step(u, dt) for m, u, dt in zip(meshes, ub, dts)])
    # where the per-mesh path's time goes: each mesh's RK4 step alone (its graph), and the
    # share of the meshes too small to fill the GPU (fewer residual CTAs than two per SM),
    # the only time that batching can recover
    per_mesh = [timed(lambda m=m, u=u, dt=dt: m.rk_step(u, dt)) for m, u, dt in zip(meshes, ub, dts)]
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    small = [i for i, m in enumerate(meshes)
             if (m.n_elem + m.info["elems_per_cta_residual"] - 1) // m.info["elems_per_cta_residual"] < 2 * sms]
    small_ms = sum(per_mesh[i] for i in small)
    order = sorted(range(len(meshes)), key=lambda i: -per_mesh[i])
    line = {"metric": "FP64 DOF-residual updates/s, 64-mesh batch (RK4 steps)", "unit": UNIT,
            "per_mesh_breakdown": {
                "sum_of_single_mesh_steps_ms": sum(per_mesh),
                "largest_8": [{"mesh": f"{'tri' if mix[i][0] == 2 else 'tet'} M={mix[i][1]} p={mix[i][2]}",
                               "n_elem": meshes[i].n_elem, "ms": per_mesh[i]} for i in order[:8]],
                "share_of_largest_8": sum(per_mesh[i] for i in order[:8]) / sum(per_mesh),
                "meshes_under_two_ctas_per_sm": len(small), "their_ms": small_ms,
                "speedup_bound_if_their_time_vanished": sum(per_mesh) / max(sum(per_mesh) - small_ms, 1e-9)},
            "batched": {"value": 4.0 * dof / (ms_batch * 1e-3), "ms_per_step": ms_batch,
                        "launches_per_step": None},
            "plain_per_mesh": {"value": 4.0 * dof / (ms_plain * 1e-3), "ms_per_step": ms_plain,
                               "launches_per_step": 8 * len(meshes)},
            "speedup": ms_plain / ms_batch, "n_meshes": len(meshes), "dof": dof,
            "mix": [f"{'tri' if d == 2 else 'tet'} M={M} p={p}" for d, M, p, _ in mix],
            "meshes": "small (launch-bound)" if args.batch_small else "batching workload",
            "setup_s": setup_s, "steps": args.steps, "warmup": args.warmup}
    print(json.dumps(line), flush=True)
    E.esd_batch_destroy(b)


# ---------------------------------------------------------------------------------
# per-configuration sweep: single-residual and RK4 throughput with the residual kernel's
# roofline fraction (not the headline line; one JSON line per configuration)
# ---------------------------------------------------------------------------------
SWEEP = ([("tri_vortex_curved", 2, 64, 1.0, p, "vortex") for p in (4, 6, 8, 10)]
         + [("tet_tgv_curved", 3, 16, 2 * np.pi, p, "tgv") for p in (2, 4, 6)]
         + [("tet_tgv_curved_8", 3, 8, 2 * np.pi, p, "tgv") for p in (8, 10)])   # 3072 tets, high degree


def _time_flushed(torch, stream, fn, reps, flush):
    """Mean device time of fn() over reps launches, L2 flushed (a 256 MB write) before each."""
    tot = 0.0
    with torch.cuda.stream(stream):
        fn()
        for _ in range(reps):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            stream.synchronize()
            tot += a.elapsed_time(b)
    return tot / reps


def run_sweep(args):
    import torch
    import paper_2312_07874_gb300 as E
    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(32 * 1024 * 1024, dtype=torch.float64, device=dev)
    peak = E.esd_measure_fp64_peak(stream)
    reps = max(3, args.steps)
    for name, dim, M, L, p, state in SWEEP:
        mesh, X = I.config_mesh(dim, M, L, p, True)
        gm = E.Mesh(dim, p, X, mesh.nbr_elem, mesh.nbr_face, flux="LF")
        f = I.config_state_fn(dim, L, state)
        x = gm.volume_nodes()
        nod = f(x)
        if dim == 2:   # seeded U(-1e-3, 1e-3) on nodal density
            nod[..., 0] += I.seeded_uniform(1, nod[..., 0].shape, -1e-3, 1e-3)
        u = gm.l2_project(torch.from_numpy(np.ascontiguousarray(np.transpose(nod, (0, 2, 1)))).to(dev))
        launch = gm.autotune(u)   # elements per CTA and threads, timed on this mesh (untimed setup)
        lam = I.max_wave_speed_sampled(f, dim, L)
        dt = 0.1 * (L / M) / (lam * (2 * p + 1))
        info = gm.info
        nE = info["n_elem"]
        dof = nE * info["n_modes"] * info["n_c"]
        out = torch.empty_like(u)
        rhs_ms = _time_flushed(torch, stream, lambda: E.esd_rhs(gm.handle, u, out, stream), reps, flush)
        E.esd_launch_stage(gm.handle, 0, u, None, stream)
        res_ms = _time_flushed(torch, stream, lambda: E.esd_launch_stage(gm.handle, 1, None, out, stream),
                               reps, flush)
        proj_ms = _time_flushed(torch, stream, lambda: E.esd_launch_stage(gm.handle, 0, u, None, stream),
                                reps, flush)
        ur = u.clone()
        rk_ms = _time_flushed(torch, stream, lambda: gm.rk_step(ur, dt), reps, flush)
        gm.check()
        rflops, npairs = residual_kernel_flops(dim, p)
        line = {"kind": "sweep", "workload": f"{name} p={p}", "n_elem": nE, "p": p, "dof": dof,
                "rhs": {"ms": rhs_ms, "dof_residual_updates_per_s": dof / (rhs_ms * 1e-3),
                        "two_point_fluxes_per_s": npairs * nE / (rhs_ms * 1e-3)},
                "rk4_step": {"ms": rk_ms, "dof_residual_updates_per_s": 4 * dof / (rk_ms * 1e-3)},
                "residual_kernel": {"ms": res_ms, "achieved_tflops": rflops * nE / (res_ms * 1e-3) / 1e12,
                                    "peak_tflops": peak / 1e12, "frac": rflops * nE / (res_ms * 1e-3) / peak,
                                    "bound": "alu", "algorithmic_flops_per_elem": rflops},
                "project_kernel_ms": proj_ms,
                "launch": {k: launch[k] for k in ("elems_per_cta_project", "elems_per_cta_residual")},
                "l2": "flushed (256 MB write) before every timed launch", "dtype": "f64"}
        print(json.dumps(line), flush=True)
        del gm, u, ur, out
        torch.cuda.empty_cache()
    # differentiation workload: VJP of esd_rhs on 3072 curved tets at p = 3, and a 20-step
    # RK4 rollout with per-stage checkpoints through torch.autograd
    from paper_2312_07874_gb300.autograd import rollout
    mesh, X = I.config_mesh(3, 8, 2 * np.pi, 3, True)
    gm = E.Mesh(3, 3, X, mesh.nbr_elem, mesh.nbr_face, flux="LF")
    x = gm.volume_nodes()
    nod = np.transpose(I.taylor_green(x, 0.1), (0, 2, 1))
    u = gm.l2_project(torch.from_numpy(np.ascontiguousarray(nod)).to(dev))
    u += torch.from_numpy(I.seeded_normal(21, tuple(u.shape), 1e-3)).to(dev)
    cot = torch.from_numpy(I.seeded_normal(22, tuple(u.shape), 1.0)).to(dev)
    out, grad = torch.empty_like(u), torch.empty_like(u)
    fwd = _time_flushed(torch, stream, lambda: E.esd_rhs(gm.handle, u, out, stream), reps, flush)
    adj = _time_flushed(torch, stream, lambda: E.esd_rhs_vjp(gm.handle, u, cot, grad, stream), reps, flush)
    tape = gm.empty_tapes()
    fwd_s = _time_flushed(torch, stream, lambda: E.esd_rhs_save(gm.handle, u, out, tape, stream), reps, flush)
    adj_s = _time_flushed(torch, stream, lambda: E.esd_rhs_vjp_saved(gm.handle, u, tape, cot, grad, stream),
                          reps, flush)
    lam = I.max_wave_speed_sampled(lambda y: I.taylor_green(y, 0.1), 3, 2 * np.pi)
    dt = 0.1 * (2 * np.pi / 8) / (lam * 7)

    def fwd_only(mode):
        with torch.no_grad():
            rollout(u, gm, dt, 20, mode)

    def fwd_bwd(mode):
        u0 = u.clone().requires_grad_(True)
        (cot * rollout(u0, gm, dt, 20, mode)).sum().backward()
    # the same 20 steps without checkpoints: the rollout's per-step checkpoint copies cost the
    # difference
    ur = u.clone()

    def plain20():
        for _ in range(20):
            gm.rk_step(ur, dt)
    t_plain = _time_flushed(torch, stream, plain20, 2, flush)
    roll = {}
    for mode in ("stages", "tapes"):
        t_f = _time_flushed(torch, stream, lambda: fwd_only(mode), 2, flush)
        t_fb = _time_flushed(torch, stream, lambda: fwd_bwd(mode), 2, flush)
        roll[mode] = {"rollout_20_steps_ms": t_f, "rollout_20_steps_forward_backward_ms": t_fb,
                      "rollout_backward_forward_ratio": (t_fb - t_f) / t_f}
    print(json.dumps({"kind": "sweep", "workload": "vjp tet_tgv_curved p=3 (8^3 x 6 = 3072 tets, TGV + N(0,1e-3))",
                      "rhs_ms": fwd, "rhs_vjp_ms": adj, "adjoint_forward_ratio": adj / fwd,
                      "rhs_save_ms": fwd_s, "rhs_vjp_saved_ms": adj_s, "adjoint_forward_ratio_saved_tape": adj_s / fwd_s,
                      "rollout_20_steps_ms": roll["stages"]["rollout_20_steps_ms"],
                      "rollout_20_steps_forward_backward_ms": roll["stages"]["rollout_20_steps_forward_backward_ms"],
                      "rollout_backward_forward_ratio": roll["stages"]["rollout_backward_forward_ratio"],
                      "checkpoint": "stages", "rollout_checkpoint_tapes": roll["tapes"],
                      "plain_20_steps_ms": t_plain,
                      "l2": "flushed (256 MB write) before every timed call", "dtype": "f64"}), flush=True)


def run_partition(args):
    """The element partition with its facet-trace exchange on one GPU: the benchmark mesh
    (24576 curved tetrahedra, p = 4, TGV) evaluated whole (esd_rhs) and split into 2 slabs
    and into 8 round-robin partitions, each partition phase by phase (esd_rhs_begin, trace
    export / import, esd_rhs_end) on one stream; results checked bitwise against the whole
    mesh.  One line per split; L2 flushed before every timed call."""
    import torch
    import paper_2312_07874_gb300 as E
    from paper_2312_07874_gb300.partition import split, LocalExchange
    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(32 * 1024 * 1024, dtype=torch.float64, device=dev)
    mesh, gm, u0, dt = build_inputs(torch, E, dev)
    gm.autotune(u0)
    X = I.config_mesh(3, WORKLOAD["M"], WORKLOAD["L"], WORKLOAD["p"], True)[1]
    ref = torch.empty_like(u0)
    whole_ms = _time_flushed(torch, stream, lambda: E.esd_rhs(gm.handle, u0, ref, stream), args.steps, flush)
    E.esd_rhs(gm.handle, u0, ref, stream)
    stream.synchronize()
    c = X.mean(axis=1)[:, 0]
    for name, owner in (("2 slabs", (c >= np.median(c)).astype(np.int64)),
                        ("8 round-robin partitions", np.arange(len(X)) % 8)):
        parts = split(mesh.nbr_elem, mesh.nbr_face, owner)
        ms = [E.Mesh(3, WORKLOAD["p"], pt.map_nodes(X), pt.nbr_elem, pt.nbr_face, n_ghost=pt.n_ghost) for pt in parts]
        loc = [torch.from_numpy(pt.local).to(dev) for pt in parts]
        us = [u0[i].contiguous() for i in loc]
        for m, up in zip(ms, us):
            m.autotune(up, E.ESD_TUNE_PROJECT | E.ESD_TUNE_RESIDUAL)
        outs = [torch.empty_like(up) for up in us]
        exchange = LocalExchange(ms, parts, E.ESD_TRACE_STATES)   # index lists and buffers set up once

        def phased():
            for m, up in zip(ms, us):
                E.esd_rhs_begin(m.handle, up, stream)
            exchange(stream)
            for m, o in zip(ms, outs):
                E.esd_rhs_end(m.handle, o, stream)
        with torch.cuda.stream(stream):
            ms_split = _time_flushed(torch, stream, phased, args.steps, flush)
            phased()
        stream.synchronize()
        exact = all(bool(torch.equal(o, ref[i])) for o, i in zip(outs, loc))
        _, per_s, _ = E.esd_part_info(ms[0].handle)
        ghosts = sum(pt.n_ghost for pt in parts)
        print(json.dumps({"kind": "partition", "workload": f"tet_tgv_curved p={WORKLOAD['p']} ({len(X)} elements), {name}",
                          "esd_rhs_ms": whole_ms, "phased_ms": ms_split, "overhead": ms_split / whole_ms - 1.0,
                          "ghost_elements": ghosts, "trace_bytes_per_rhs": ghosts * per_s * 8,
                          "bitwise_equal_to_whole_mesh": exact,
                          "l2": "flushed (256 MB write) before every timed call", "dtype": "f64"}), flush=True)
        del ms


def run_skew(args):
    """The skew-symmetric form (esd_rhs_skew, Eq. (rhs_skew)) against the entropy-stable
    esd_rhs on the same meshes and states: 24576 curved tetrahedra (TGV) and 8192 curved
    triangles (vortex) at p = 4, Euler with LF facets, and linear advection (upwind) of the
    density.  One line per workload; L2 flushed before every timed call."""
    import torch
    import paper_2312_07874_gb300 as E
    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(32 * 1024 * 1024, dtype=torch.float64, device=dev)
    peak = E.esd_measure_fp64_peak(stream)
    reps = max(3, args.steps)
    for name, dim, M, L, p, state in [("tet_tgv_curved", 3, 16, 2 * np.pi, 4, "tgv"),
                                      ("tri_vortex_curved", 2, 64, 1.0, 4, "vortex")]:
        mesh, X = I.config_mesh(dim, M, L, p, True)
        gm = E.Mesh(dim, p, X, mesh.nbr_elem, mesh.nbr_face, flux="LF")
        x = gm.volume_nodes()
        f = I.config_state_fn(dim, L, state)
        u = gm.l2_project(torch.from_numpy(np.ascontiguousarray(np.transpose(f(x), (0, 2, 1)))).to(dev))
        gm.autotune(u, E.ESD_TUNE_PROJECT | E.ESD_TUNE_RESIDUAL)
        out = torch.empty_like(u)
        es_ms = _time_flushed(torch, stream, lambda: E.esd_rhs(gm.handle, u, out, stream), reps, flush)
        nE = gm.info["n_elem"]
        line = {"kind": "skew", "workload": f"{name} p={p} ({nE} elements)", "esd_rhs_ms": es_ms}
        for model in ("euler", "advection"):
            sk = E.Skew(dim, p, X, mesh.nbr_elem, mesh.nbr_face, model=model, a=(1.0, 0.6, -0.35)[:dim],
                        upwind=True, flux="LF")
            us = u if model == "euler" else u[:, :1].contiguous()
            so = torch.empty_like(us)
            ms = _time_flushed(torch, stream, lambda: E.esd_rhs_skew(sk.handle, us, so, stream), reps, flush)
            sk.check()
            nc = sk.nc
            dof = nE * gm.n_modes * nc
            fl = skew_residual_flops(dim, p, nc)
            line[model] = {"esd_rhs_skew_ms": ms, "dof_residual_updates_per_s": dof / (ms * 1e-3),
                           "skew_residual_flops_per_elem": fl,
                           "whole_call_tflops": fl * nE / (ms * 1e-3) / 1e12,
                           "whole_call_frac_of_measured_fp64": fl * nE / (ms * 1e-3) / peak,
                           "launch": sk.info}
            del sk, us, so
        line.update({"fp64_peak_tflops": peak / 1e12, "l2": "flushed (256 MB write) before every timed call",
                     "dtype": "f64"})
        print(json.dumps(line), flush=True)
        del gm, u, out
        torch.cuda.empty_cache()


def otf_direction_flops(D, p):
    """Extra flops per element of forming the pair directions on the fly: per volume pair the
    D coefficients (Q_ij - Q_ji)/4 (FMA + MUL each) and D^2 (ADD + FMA); per facet pair
    D (D FMA + MUL) -- the arithmetic the stored tables replace by 3 loads."""
    n = p + 1
    vol_pairs = D * n ** (D - 1) * (p * (p + 1) // 2)
    fac_pairs = 3 * n * n if D == 2 else 3 * n ** 3 + n ** 4
    return vol_pairs * (3 * D + 3 * D * D) + fac_pairs * D * (2 * D + 1)


def run_directions(args):
    """The pair-direction trade measured both ways: the residual kernel with the stored
    per-element pair tables (ESD_MESH_PAIR_TABLES) and with directions formed on the fly from
    per-node metric terms (ESD_MESH_METRICS_ON_THE_FLY), on the same mesh and state; device
    memory of each mesh, kernel time (L2 flushed), fraction of the measured FP64 peak."""
    import torch
    import paper_2312_07874_gb300 as E
    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(32 * 1024 * 1024, dtype=torch.float64, device=dev)
    peak = E.esd_measure_fp64_peak(stream)
    reps = max(3, args.steps)
    cases = [("tet_tgv_curved", 3, 16, 2 * np.pi, 4, "tgv"), ("tet_tgv_curved_8", 3, 8, 2 * np.pi, 10, "tgv"),
             ("tet_tgv_curved", 3, 16, 2 * np.pi, 10, "tgv"), ("tri_vortex_curved", 2, 64, 1.0, 4, "vortex"),
             ("tri_vortex_curved", 2, 64, 1.0, 10, "vortex")]
    for name, dim, M, L, p, state in cases:
        mesh, X = I.config_mesh(dim, M, L, p, True)
        f = I.config_state_fn(dim, L, state)
        line = {"kind": "pair_directions", "workload": f"{name} p={p}"}
        outs = {}
        for tag, otf in (("stored_pair_tables", False), ("metrics_on_the_fly", True)):
            gm = E.Mesh(dim, p, X, mesh.nbr_elem, mesh.nbr_face, flux="LF", metrics_on_the_fly=otf)
            x = gm.volume_nodes()
            u = gm.l2_project(torch.from_numpy(np.ascontiguousarray(np.transpose(f(x), (0, 2, 1)))).to(dev))
            gm.autotune(u, E.ESD_TUNE_PROJECT | E.ESD_TUNE_RESIDUAL)
            out = torch.empty_like(u)
            E.esd_launch_stage(gm.handle, 0, u, None, stream)
            ms = _time_flushed(torch, stream, lambda: E.esd_launch_stage(gm.handle, 1, None, out, stream), reps, flush)
            gm.check()
            nE = gm.info["n_elem"]
            fl, _ = residual_kernel_flops(dim, p)
            extra = otf_direction_flops(dim, p) if otf else 0
            outs[tag] = out.cpu().numpy()
            line[tag] = {"residual_kernel_ms": ms, "device_bytes_per_elem": gm.info["device_bytes"] / nE,
                         "frac_of_measured_fp64": fl * nE / (ms * 1e-3) / peak,
                         "frac_incl_direction_flops": (fl + extra) * nE / (ms * 1e-3) / peak,
                         "elems_per_cta": gm.info["elems_per_cta_residual"]}
            line["n_elem"] = nE
            del gm, u, out
            torch.cuda.empty_cache()
        a, b = outs["stored_pair_tables"], outs["metrics_on_the_fly"]
        line["max_rel_difference"] = float((np.abs(a - b).max(axis=(0, 2)) / np.abs(a).max(axis=(0, 2))).max())
        line["time_ratio_otf_over_stored"] = (line["metrics_on_the_fly"]["residual_kernel_ms"]
                                              / line["stored_pair_tables"]["residual_kernel_ms"])
        line.update({"fp64_peak_tflops": peak / 1e12, "l2": "flushed (256 MB write) before every timed launch",
                     "dtype": "f64"})
        print(json.dumps(line), flush=True)


def run_diagnostics_series(args):
    """Conservation and entropy over a run: Taylor-Green vortex at Mach 0.1 on 4^3 x 6 = 384
    curved tetrahedra, p = 4, entropy-conservative (EC) and Lax-Friedrichs (LF) interface
    fluxes, RK4 at CFL 0.1, totals and rates sampled every 10 steps (one line per flux)."""
    import torch
    import paper_2312_07874_gb300 as E
    L, M, p = 2 * np.pi, 4, 4
    mesh, X = I.config_mesh(3, M, L, p, True)
    lam = I.max_wave_speed_sampled(lambda y: I.taylor_green(y, 0.1), 3, L)
    dt = 0.1 * (L / M) / (lam * (2 * p + 1))
    n_steps = max(20, args.steps) if args.steps != 10 else 200
    for flux in ("EC", "LF"):
        gm = E.Mesh(3, p, X, mesh.nbr_elem, mesh.nbr_face, flux=flux)
        x = gm.volume_nodes()
        un = np.ascontiguousarray(np.transpose(I.taylor_green(x, 0.1), (0, 2, 1)))
        u = gm.l2_project(torch.from_numpy(un).cuda())
        t0 = time.time()
        steps, tot, rates = gm.run_diagnostics(u, dt, n_steps, every=10)
        wall = time.time() - t0
        nc = 5
        cons = np.abs(tot[:, :nc] - tot[0, :nc]).max(axis=0) / np.abs(tot[0, :nc]).max()
        ent_rate = rates[:, nc] / rates[:, nc + 1]
        S = tot[:, nc]
        print(json.dumps({"kind": "diagnostics", "workload": f"tet_tgv_curved p={p} M={M} (384 tets), {flux} facets",
                          "steps": int(steps[-1]), "dt": dt, "t_final": float(steps[-1] * dt),
                          "samples": int(len(steps)),
                          "max_conserved_drift_rel": cons.tolist(),
                          "entropy_rate_rel": {"min": float(ent_rate.min()), "max": float(ent_rate.max())},
                          "entropy_total_change_rel": float((S[-1] - S[0]) / abs(S[0])),
                          "entropy_monotone": bool(np.all(np.diff(S) <= 1e-12 * abs(S[0]))),
                          "wall_s": wall}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-seconds", type=float, default=15.0, help="0 skips the CPU baseline")
    ap.add_argument("--mesh-m", type=int, default=16, help="cells per direction (16 = the benchmark)")
    ap.add_argument("--batch", action="store_true", help="64-mesh batched vs per-mesh comparison")
    ap.add_argument("--batch-small", action="store_true", help="with --batch: 64 small meshes instead")
    ap.add_argument("--no-autotune", action="store_true", help="keep the default launch shapes (profiling)")
    ap.add_argument("--diagnostics", action="store_true", help="conservation / entropy time series (EC and LF)")
    ap.add_argument("--directions", action="store_true", help="the residual kernel with stored pair tables "
                    "against pair directions formed on the fly from per-node metric terms")
    ap.add_argument("--skew", action="store_true", help="the skew-symmetric form (esd_rhs_skew) against "
                    "esd_rhs on the tetrahedron and triangle workloads at p = 4")
    ap.add_argument("--sweep", action="store_true", help="per-degree throughput of the triangle and "
                    "tetrahedron workloads and the differentiation workload (one line each)")
    ap.add_argument("--partition", action="store_true", help="the benchmark mesh split into element "
                    "partitions with the facet-trace exchange, against the whole mesh (one GPU)")
    args = ap.parse_args()
    WORKLOAD["M"] = args.mesh_m
    if args.batch:
        run_batch(args)
        return
    if args.sweep:
        run_sweep(args)
        return
    if args.diagnostics:
        run_diagnostics_series(args)
        return
    if args.skew:
        run_skew(args)
        return
    if args.directions:
        run_directions(args)
        return
    if args.partition:
        run_partition(args)
        return
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
