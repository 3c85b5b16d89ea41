"""Recomputes the tables of section 5.4 with the discrete Fourier analysis tool (oracle/lfa.py) and
prints each cell as "tool (paper)" in markdown.  TEST INFRASTRUCTURE ONLY: calls nothing but the
oracle; its output documents the readings of the analysis beside the paper's numbers.

    python -m oracle.lfa_tables [--ar 1 100] [--tables erk,ark_stab,ark_rates,aw_stab,aw_rates,aw_eta]
"""
from __future__ import annotations

import argparse
import json
import os
import time

from . import lfa

GOLD = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "tests", "golden",
                    "paper_lfa_tables.json")


def _c(x):
    if x is None:
        return "A"
    if x >= 1e6:
        return ">1e6"
    return f"{x:g}"


def _cell(ours, paper, fmt="{:.4f}"):
    o = "A" if ours is None else (fmt.format(ours) if isinstance(ours, float) and fmt else _c(ours))
    p = "A" if paper is None else (fmt.format(paper) if fmt and isinstance(paper, float) else _c(paper))
    return f"{o} ({p})"


def table_erk(T, ars):
    rows = ["| scheme | quantity | " + " | ".join(f"AR {a}" for a in ars) + " |",
            "|---|---|" + "---|" * len(ars)]
    idx = [T["AR"].index(a) for a in ars]
    for sch in ("ERK3J", "ARK3J"):
        res = []
        for a in ars:
            m, nx, ny = lfa.table_model(0.8, 0.0, a, 0.5)
            res.append(lfa.factors(m, sch, nx, ny, 0.9, 200.0, precond="none"))
        for q, name in ((0, "rho"), (1, "sm")):
            rows.append(f"| {sch} | {name} | " + " | ".join(
                _cell(r[q], T["erk_ark"][sch][name][k]) for r, k in zip(res, idx)) + " |")
    return "\n".join(rows)


def table_stability(T, key, scheme, ars):
    t = T[key]
    idx = [T["AR"].index(a) for a in ars]
    rows = ["| d | " + " | ".join(f"{pc} AR {a}" for pc in ("sgs", "exact") for a in ars) + " |",
            "|---|" + "---|" * (2 * len(ars))]
    for i, d in enumerate(t["d"]):
        cells = []
        for pc in ("sgs", "exact"):
            for a, k in zip(ars, idx):
                m, nx, ny = lfa.table_model(0.8, 0.0, a, d)
                lim = lfa.max_stable_cstar(m, scheme, nx, ny, 200.0, 0.8, pc)
                cells.append(f"{_c(lim)} ({_c(t[pc][i][k])})")
        rows.append(f"| {d} | " + " | ".join(cells) + " |")
    return "\n".join(rows)


def table_rates(T, key, scheme, ars):
    t = T[key]
    idx = [T["AR"].index(a) for a in ars]
    rows = ["| d | quantity | " + " | ".join(f"{pc} AR {a}" for pc in ("sgs", "exact") for a in ars) + " |",
            "|---|---|" + "---|" * (2 * len(ars))]
    for i, d in enumerate(t["d"]):
        res = {}
        for pc in ("sgs", "exact"):
            for a in ars:
                m, nx, ny = lfa.table_model(0.8, 0.0, a, d)
                res[pc, a] = lfa.optimal_cstar(m, scheme, nx, ny, 200.0, 0.8, pc)
        for q, name in ((0, "cstar"), (1, "rho"), (2, "sm")):
            cells = []
            for pc in ("sgs", "exact"):
                for a, k in zip(ars, idx):
                    r = res[pc, a]
                    ours = None if r is None else r[q]
                    paper = t[pc][name][i][k]
                    cells.append(_cell(ours, paper, None if q == 0 else "{:.4f}"))
            rows.append(f"| {d} | {name} | " + " | ".join(cells) + " |")
    return "\n".join(rows)


def table_eta(T, ars, alpha_key, alpha):
    t = T["aw_opt_eta"]
    idx = [T["AR"].index(a) for a in ars]
    rows = ["| scheme | d | quantity | " + " | ".join(f"AR {a}" for a in ars) + " |",
            "|---|---|---|" + "---|" * len(ars)]
    for sch in ("AW3", "AW51", "AW52", "AW5J"):
        for i, d in enumerate(t["d"]):
            res = []
            for a in ars:
                m, nx, ny = lfa.table_model(0.8, alpha, a, d)
                res.append(lfa.optimal_eta_cstar(m, sch, nx, ny, 200.0, "sgs"))
            for q, name in ((0, "eta"), (1, "cstar"), (2, "rho"), (3, "sm")):
                cells = []
                for r, k in zip(res, idx):
                    ours = None if r is None else r[q]
                    paper = t[alpha_key][sch][name][i][k]
                    cells.append(_cell(ours, paper, None if q == 1 else ("{:.1f}" if q == 0 else "{:.4f}")))
                rows.append(f"| {sch} | {d} | {name} | " + " | ".join(cells) + " |")
    return "\n".join(rows)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--ar", type=int, nargs="+", default=[1, 100])
    ap.add_argument("--tables", default="erk,ark_stab,ark_rates,aw_stab,aw_rates,aw_eta")
    a = ap.parse_args()
    T = json.load(open(GOLD))
    want = a.tables.split(",")
    jobs = [("erk", "Table ERK-ARK (c* = 0.9, no preconditioner)", lambda: table_erk(T, a.ar)),
            ("ark_stab", "Table Prec-ARK-stability (maximal c*, ARK3J)",
             lambda: table_stability(T, "prec_ark_stability", "ARK3J", a.ar)),
            ("ark_rates", "Table Prec-ARK-rates (ARK3J at the optimal c*)",
             lambda: table_rates(T, "prec_ark_rates", "ARK3J", a.ar)),
            ("aw_stab", "Table AW-stability (maximal c*, AW3, eta 0.8)",
             lambda: table_stability(T, "aw_stability", "AW3", a.ar)),
            ("aw_rates", "Table AW (AW3 at the optimal c*, eta 0.8)",
             lambda: table_rates(T, "aw_rates", "AW3", a.ar)),
            ("aw_eta", "Table AWa0 (optimal eta and c*, alpha 0)", lambda: table_eta(T, a.ar, "alpha0", 0.0)),
            ("aw_eta", "Table AWa45 (optimal eta and c*, alpha 45)", lambda: table_eta(T, a.ar, "alpha45", 45.0))]
    for key, title, fn in jobs:
        if key not in want:
            continue
        t0 = time.time()
        body = fn()
        print(f"\n**{title}** — tool (paper); {time.time() - t0:.0f} s\n\n{body}", flush=True)


if __name__ == "__main__":
    main()
