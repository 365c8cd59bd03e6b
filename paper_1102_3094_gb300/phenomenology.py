"""Lamellar ordering behind cold fronts at the parameters of arXiv:1102.3094
(Sec. 3): the 2D runs of its Figs. 1 (no hydrodynamics) and 2 (with
hydrodynamics, tau = 5) and the 3D runs of its Fig. 3 (no hydrodynamics),
repeated with this library and summarised by the orientation order
parameter s (+1: lamellae parallel to the walls, -1: perpendicular),
globally, near the walls and in the bulk, and by the S(k) peak.  The paper
reports these runs as snapshots only, so the comparison is qualitative:
which fronts give parallel and which perpendicular lamellae.

    python -m paper_1102_3094_gb300.phenomenology [--quick] [--stencil compact|isotropic]
                                                  [--figures fig1,fig2,fig3]

Parameters (Sec. 3): b = 0.1, kappa = -c = -0.03, Tc = 0.005, Gamma = 0.1,
T_w = 0.9 Tc, phi uniform in [-0.01, 0.01]; 256 x 256 with cold walls at
y = 0 and 255 in 2D, 32 x 32 x 256 with cold walls at z = 0 and 255 in 3D.
The initial temperature is only said to be above Tc; 1.1 Tc is used.  With
the compact 7-point Laplacian the explicit phi update of the 3D runs is
unstable at these parameters (Gamma lam (a + kappa lam + c lam^2) > 2 near
lam = 12), which lf_create reports as LF_EUNSTABLE; the isotropic 19-point
stencils (largest lam 16/3) run them.
"""
from __future__ import annotations

import argparse
import json
import math
import sys

import numpy as np

# (figure, hydro, tau, xi, snapshot time of the paper's figure)
CASES = [
    ("fig1", 0, 1.0, 1e-2, 55_700),
    ("fig1", 0, 1.0, 1e-1, 11_700),
    ("fig1", 0, 1.0, 1.0, 11_700),
    ("fig1", 0, 1.0, math.inf, 1_950),
    ("fig2", 1, 5.0, 1e-4, 1_440_000),
    ("fig2", 1, 5.0, 1e-3, 356_000),
    ("fig2", 1, 5.0, 5e-3, 356_000),
    ("fig2", 1, 5.0, math.inf, 21_000),
    ("fig3", 0, 1.0, 1e-2, 7_800),
    ("fig3", 0, 1.0, 1.0, 1_500),
    ("fig3", 0, 1.0, 1e2, 110),
]


def run_case(fig, hydro, tau, xi, t_end, n_reports=10, precision="fp32", seed=3, stencil="compact"):
    from paper_1102_3094_gb300 import lf

    Tc = 0.005
    shape = dict(d=3, nx=32, ny=32, nz=256) if fig == "fig3" else dict(d=2, nx=256, ny=256)
    base = {"figure": fig, "hydro": hydro, "tau": tau, "xi": xi, "t_end": t_end, "stencil": stencil}
    try:
        sim = lf.Lattice(b=0.1, kappa=-0.03, c=0.03, Gamma=0.1, Tc=Tc, T0=1.1 * Tc, T_w=0.9 * Tc, xi=xi,
                         tau=tau, hydro=hydro, phi_amp=0.01, seed=seed, precision=precision, stencil=stencil,
                         **shape)
    except lf.LFError as ex:                  # refused at creation (LF_EUNSTABLE)
        return dict(base, series=[], diverged=None, refused=str(ex))
    rows = []
    done = 0
    diverged = None
    for r in range(1, n_reports + 1):
        target = round(t_end * r / n_reports)
        try:
            sim.step(target - done)
        except lf.LFError as ex:              # the state went non-finite inside this stretch
            diverged = {"after": done, "before": target, "error": str(ex)}
            break
        done = target
        d = sim.diag()
        if d["rc"] != 0:                       # a NaN/Inf reached the state during this stretch
            diverged = {"after": rows[-1]["t"] if rows else 0, "before": done, "error": lf.strerror(d["rc"])}
            break
        prof = sim.layers()
        near = float(np.mean(np.concatenate([prof[:20], prof[-20:]])))
        bulk = float(np.mean(prof[96:160]))
        rows.append({"t": done, "s": d["orient_s"], "s_walls": near, "s_bulk": bulk, "k_peak": d["k_peak"],
                     "mach": d["mach"], "rc": d["rc"]})
    sim.close()
    return dict(base, series=rows, diverged=diverged, refused=None)


def main(argv=None) -> int:
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--quick", action="store_true", help="a tenth of every run length")
    ap.add_argument("--out", default=None, help="write the JSON lines here as well")
    ap.add_argument("--stencil", choices=["compact", "isotropic"], default="compact")
    ap.add_argument("--figures", default="fig1,fig2,fig3", help="comma-separated subset of fig1,fig2,fig3")
    args = ap.parse_args(argv)
    figs = set(args.figures.split(","))
    results = []
    for fig, hydro, tau, xi, t_end in CASES:
        if fig not in figs:
            continue
        res = run_case(fig, hydro, tau, xi, max(100, t_end // 10) if args.quick else t_end, stencil=args.stencil)
        results.append(res)
        print(json.dumps(res), flush=True)
    print(f"\nstencil: {args.stencil}")
    print("| figure | hydro | xi | t | s | s near walls | s bulk | k_peak |")
    print("|---|---|---|---|---|---|---|---|")
    for r in results:
        if r["refused"]:
            print(f"| {r['figure']} | {r['hydro']} | {r['xi']:g} | refused: {r['refused']} | | | | |")
            continue
        if not r["series"]:
            print(f"| {r['figure']} | {r['hydro']} | {r['xi']:g} | diverged before {r['diverged']['before']} | | | | |")
            continue
        last = r["series"][-1]
        note = f" (diverged before {r['diverged']['before']})" if r["diverged"] else ""
        print(f"| {r['figure']} | {r['hydro']} | {r['xi']:g} | {last['t']}{note} | {last['s']:+.3f} | "
              f"{last['s_walls']:+.3f} | {last['s_bulk']:+.3f} | {last['k_peak']:.3f} |")
    if args.out:
        with open(args.out, "w") as fh:
            for r in results:
                fh.write(json.dumps(r) + "\n")
    return 0


if __name__ == "__main__":
    sys.exit(main())
