"""Runs of the synthetic lamellar-quench configurations to their stated
lengths, with either stencil, reporting the structure-factor peak, the
orientation order parameter and the Mach number along the way (Sec. 2 asks for
Ma < 0.1) and where a run goes non-finite.

    python -m paper_1102_3094_gb300.config_runs [--cube 384] [--square 1024]
                                                [--quick] [--out FILE]

Configurations (b = 1, kappa = -0.025, c = 0.02, Gamma = 0.05, Tc = 1,
T0 = 1.1, T_w = 0.5, phi uniform in [-0.05, 0.05]):
  * 3D, cube^3 D3Q19, FP32, periodic in x and y, cold walls normal to z,
    xi in {1e-3, 1e-2}, tau in {0.6, 3}, 20k steps;
  * 2D, square^2 D2Q9, FP32, cold walls normal to y, xi in {1e-3, 1e-1},
    tau = 1, 50k steps.
"""
from __future__ import annotations

import argparse
import json
import sys


def run(d, n, xi, tau, stencil, steps, reports, seed=1):
    from paper_1102_3094_gb300 import lf

    shape = dict(d=3, nx=n, ny=n, nz=n) if d == 3 else dict(d=2, nx=n, ny=n)
    sim = lf.Lattice(precision="fp32", xi=xi, tau=tau, seed=seed, stencil=stencil, **shape)
    rows, done, diverged = [], 0, None
    for r in range(1, reports + 1):
        target = steps * r // reports
        try:
            sim.step(target - done)
        except lf.LFError as ex:              # the state went non-finite inside this stretch
            diverged = {"after": done, "before": target, "error": str(ex)}
            break
        done = target
        dg = sim.diag()
        if dg["rc"] != 0:
            diverged = {"after": rows[-1]["t"] if rows else 0, "before": done, "error": lf.strerror(dg["rc"])}
            break
        rows.append({"t": done, "k_peak": dg["k_peak"], "s_peak": dg["s_peak"], "s": dg["orient_s"],
                     "mach": dg["mach"], "mass": dg["mass"]})
    sim.close()
    return {"d": d, "n": n, "xi": xi, "tau": tau, "stencil": stencil, "steps": steps, "series": rows,
            "diverged": diverged, "finite_to": rows[-1]["t"] if rows else 0}


def precision_pair(n, xi, stencil, seeds, steps, reports, d=2, tau=1.0):
    """The precision form against FP64 on the GPU: the same run (lattice,
    physics, seed) in FP32 (deviation populations) and in FP64, S(k) peak
    position and height and s at every report time; per report time the seed
    means of both and their relative (k, S) or absolute (s) differences."""
    from paper_1102_3094_gb300 import lf

    shape = dict(d=3, nx=n, ny=n, nz=n) if d == 3 else dict(d=2, nx=n, ny=n)
    per = {"fp32": {}, "fp64": {}}
    for seed in seeds:
        for prec in ("fp32", "fp64"):
            sim = lf.Lattice(precision=prec, xi=xi, tau=tau, seed=seed, stencil=stencil, **shape)
            rows, done = [], 0
            for r in range(1, reports + 1):
                target = steps * r // reports
                try:
                    sim.step(target - done)
                except lf.LFError:               # the run went non-finite in this stretch
                    break
                done = target
                dg = sim.diag()
                if dg["rc"] != 0:
                    break
                rows.append({"t": done, "k_peak": dg["k_peak"], "s_peak": dg["s_peak"], "s": dg["orient_s"]})
            sim.close()
            per[prec][seed] = rows
    table = []
    for i in range(reports):
        # seeds whose runs are finite at this report time in both precisions
        ok = [sd for sd in seeds if len(per["fp32"][sd]) > i and len(per["fp64"][sd]) > i]
        if not ok:
            break
        m = {p_: {k: sum(per[p_][sd][i][k] for sd in ok) / len(ok) for k in ("k_peak", "s_peak", "s")} for p_ in per}
        table.append({"t": per["fp32"][ok[0]][i]["t"], "seeds": len(ok), "fp32": m["fp32"], "fp64": m["fp64"],
                      "d_k_peak": abs(m["fp32"]["k_peak"] / m["fp64"]["k_peak"] - 1),
                      "d_s_peak": abs(m["fp32"]["s_peak"] / m["fp64"]["s_peak"] - 1),
                      "d_s": abs(m["fp32"]["s"] - m["fp64"]["s"])})
    return {"d": d, "n": n, "xi": xi, "tau": tau, "stencil": stencil, "seeds": list(seeds), "steps": steps,
            "table": table,
            "runs": {p_: {str(k): v for k, v in d.items()} for p_, d in per.items()}}


def main(argv=None) -> int:
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--cube", type=int, default=384, help="3D lattice side (0: skip the 3D runs)")
    ap.add_argument("--square", type=int, default=1024, help="2D lattice side (0: skip the 2D runs)")
    ap.add_argument("--quick", action="store_true", help="a tenth of every run length")
    ap.add_argument("--reports", type=int, default=10)
    ap.add_argument("--out", default=None)
    ap.add_argument("--precision", action="store_true",
                    help="instead: FP32 against FP64 over 8 seeds at square^2, 50k steps (isotropic stencils "
                         "at xi = 1e-3 and 0.1, compact at xi = 1e-3)")
    ap.add_argument("--precision3d", type=int, default=0, metavar="N",
                    help="instead: FP32 against FP64 over 8 seeds at N^3, 20k steps (isotropic stencils, "
                         "tau = 3, xi = 1e-3: the 3D configuration that runs its length)")
    args = ap.parse_args(argv)
    if args.precision or args.precision3d:
        import torch

        torch.cuda.init()
        div = 10 if args.quick else 1
        if args.precision3d:
            out = [precision_pair(args.precision3d, 1e-3, "isotropic", range(1, 9), 20_000 // div, args.reports,
                                  d=3, tau=3.0)]
        else:
            out = [precision_pair(args.square, xi, st, range(1, 9), 50_000 // div, args.reports)
                   for xi, st in ((1e-3, "isotropic"), (1e-1, "isotropic"), (1e-3, "compact"))]
        for res in out:
            lat = f"{res['n']}^{res['d']}"
            print(f"\n{lat} {res['stencil']} xi = {res['xi']:g}, tau = {res['tau']:g}, 8 seeds: seed means, "
                  "FP32 against FP64")
            print("| t | seeds | k_peak fp32 / fp64 | S_peak fp32 / fp64 | s fp32 / fp64 | dk | dS | ds |")
            print("|---|---|---|---|---|---|---|---|")
            for r in res["table"]:
                a, b = r["fp32"], r["fp64"]
                print(f"| {r['t']} | {r['seeds']} | {a['k_peak']:.4f} / {b['k_peak']:.4f} | "
                      f"{a['s_peak']:.4g} / {b['s_peak']:.4g} | "
                      f"{a['s']:+.3f} / {b['s']:+.3f} | {100 * r['d_k_peak']:.2f} % | {100 * r['d_s_peak']:.2f} % | "
                      f"{r['d_s']:.3f} |")
        if args.out:
            with open(args.out, "w") as fh:
                for r in out:
                    fh.write(json.dumps(r) + "\n")
        return 0
    import torch

    torch.cuda.init()
    div = 10 if args.quick else 1
    cases = []
    if args.cube:
        for stencil in ("compact", "isotropic"):
            for tau in (0.6, 3.0):
                for xi in (1e-3, 1e-2):
                    cases.append((3, args.cube, xi, tau, stencil, 20_000 // div))
    if args.square:
        for stencil in ("compact", "isotropic"):
            for xi in (1e-3, 1e-1):
                cases.append((2, args.square, xi, 1.0, stencil, 50_000 // div))
    results = []
    for c in cases:
        res = run(*c, reports=args.reports)
        results.append(res)
        print(json.dumps(res), flush=True)
    print("\n| lattice | stencil | tau | xi | finite to (of) | k_peak | S_peak | s | max Ma |")
    print("|---|---|---|---|---|---|---|---|---|")
    for r in results:
        last = r["series"][-1] if r["series"] else None
        ma = max((x["mach"] for x in r["series"]), default=float("nan"))
        lat = f"{r['n']}^{r['d']}"
        if last:
            print(f"| {lat} | {r['stencil']} | {r['tau']:g} | {r['xi']:g} | {r['finite_to']} ({r['steps']}) | "
                  f"{last['k_peak']:.4f} | {last['s_peak']:.4g} | {last['s']:+.3f} | {ma:.3f} |")
        else:
            print(f"| {lat} | {r['stencil']} | {r['tau']:g} | {r['xi']:g} | non-finite before "
                  f"{r['diverged']['before']} ({r['steps']}) | | | | |")
    if args.out:
        with open(args.out, "w") as fh:
            for r in results:
                fh.write(json.dumps(r) + "\n")
    return 0


if __name__ == "__main__":
    sys.exit(main())
