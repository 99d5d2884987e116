"""Formats the parity records that the GPU tests append to $ESD_PARITY_LOG (one JSON object
per checked case; tests/gpu_common.py) as a markdown table: per case, the largest relative
error over the conserved variables of the CUDA path and of the FP64 oracle against the
oracle in long double, their ratio, the CUDA path against the FP64 oracle, and the error
relative to the sums of |terms|.

    ESD_PARITY_LOG=parity.jsonl python -m pytest tests -m gpu
    python tests/parity_report.py parity.jsonl
"""
import json
import sys


def fmt(x):
    return "—" if x is None else f"{x:.1e}"


def main(path):
    rows = [json.loads(line) for line in open(path) if line.strip()]
    print("| case | elements (long double) | CUDA vs exact | FP64 oracle vs exact | ratio | CUDA vs FP64 oracle "
          "| vs sum of abs(terms) | flat 1e-12 applies |")
    print("|---|---|---|---|---|---|---|---|")
    for r in rows:
        gx = max(r["e_gpu_exact"]) if r.get("n_exact", 1) else None
        ox = max(r["e_oracle64_exact"]) if r.get("n_exact", 1) else None
        ratio = max((g / max(o, 4 * 2.0 ** -53)) for g, o in zip(r["e_gpu_exact"], r["e_oracle64_exact"])) \
            if gx is not None else None
        go = max(r["e_gpu_oracle64"])
        sc = max(r["e_term_scale"]) if r.get("e_term_scale") and gx is not None else None
        flat = r.get("flat")
        nflat = f"{sum(flat)}/{len(flat)}" if isinstance(flat, list) else "—"
        ne = f"{r.get('n_elems', '')} ({r.get('n_exact', '—')})"
        print(f"| {r['case']} | {ne} | {fmt(gx)} | {fmt(ox)} | {fmt(ratio) if ratio is not None else '—'} "
              f"| {fmt(go)} | {fmt(sc)} | {nflat} |")


if __name__ == "__main__":
    main(sys.argv[1])
