"""Writes tests/golden/oracle_long3d_48.json: statistics of long FP64 oracle
runs of the 3D configuration's physics at 48^3, for the GPU test that compares
the FP32 GPU path with them at the stated report times.

Physics: D3Q19, b = 1, kappa = -0.025, c = 0.02, Gamma = 0.05, Tc = 1,
T0 = 1.1, T_w = 0.5, tau = 3, xi = 1e-3, walls at z = 0 and 47, isotropic
19-point stencils (the 3D configuration that runs its length finite), phi
uniform in [-0.05, 0.05] from SplitMix64(seed), seeds 1..8; 6,000 steps,
reported every 1,000: the structure-factor peak position and height and the
orientation order parameter (definitions in oracle/diag.py).

Only the oracle is called.  One process per seed (spawned), one OpenMP thread
each; about 100 minutes on 8 cores.  The file is rewritten after every report
time, so a partial run leaves the report times it reached.

    python tests/golden/make_oracle_long3d_stats.py [--n 48] [--steps 6000] [--every 1000] [--seeds 8]
"""
from __future__ import annotations

import argparse
import json
import multiprocessing as mp
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))


def run_seed(args):
    seed, n, steps, every, q = args
    os.environ["OMP_NUM_THREADS"] = "1"
    sys.path.insert(0, ROOT)
    from oracle import diag as D
    from oracle import oracle as O

    cfg = O.make_cfg(d=3, nx=n, ny=n, nz=n, xi=1e-3, tau=3.0, stencil=1, seed=seed)
    st = O.init(cfg)
    for t in range(every, steps + 1, every):
        st = O.run(st, every)
        _, _, k_peak, s_peak = D.structure_factor(st.phi)
        s, _ = D.orientation(st.phi, True)
        q.put((seed, {"t": t, "k_peak": k_peak, "s_peak": s_peak, "s": s}))
    q.put((seed, None))
    return seed


def main() -> int:
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=48)
    ap.add_argument("--steps", type=int, default=6_000)
    ap.add_argument("--every", type=int, default=1_000)
    ap.add_argument("--seeds", type=int, default=8)
    ap.add_argument("--out", default=os.path.join(HERE, "oracle_long3d_48.json"))
    a = ap.parse_args()
    ctx = mp.get_context("spawn")
    q = ctx.Manager().Queue()
    runs = {str(s): [] for s in range(1, a.seeds + 1)}
    cfg = {"d": 3, "nx": a.n, "ny": a.n, "nz": a.n, "xi": 1e-3, "tau": 3.0, "stencil": "isotropic",
           "precision": "fp64 oracle", "steps": a.steps, "every": a.every}
    with ctx.Pool(a.seeds) as pool:
        res = pool.map_async(run_seed, [(s, a.n, a.steps, a.every, q) for s in range(1, a.seeds + 1)])
        done = 0
        while done < a.seeds:
            seed, row = q.get()
            if row is None:
                done += 1
                continue
            runs[str(seed)].append(row)
            with open(a.out + ".tmp", "w") as fh:
                json.dump({"config": cfg, "runs": runs}, fh, indent=1)
            os.replace(a.out + ".tmp", a.out)
        res.get()
    print(a.out)
    return 0


if __name__ == "__main__":
    sys.exit(main())
