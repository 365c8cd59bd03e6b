"""The precision form over the 2D configuration's stated length: FP32 GPU runs
at 256 x 256 (the size of the configuration's oracle cross-check), 50,000
steps, 8 seeds, against the FP64 oracle's runs of the same seeds
(tests/golden/oracle_long_256.json, written by make_oracle_long_stats.py
beside it).

What the runs show, and what is asserted:
  * every FP32 trajectory follows its FP64 trajectory through 35,000 steps:
    the S(k) peak height of each seed within 1 % at every report time up to
    35,000 (measured: 0.8 % at most).  Later, single trajectories part ways
    (rounding differences grow in the coarsening dynamics: seed 1's peak height
    is 7 % off at 40,000 steps and 21 % at 50,000), so single runs are not
    compared after that;
  * the seed means at every report time: the S(k) peak position within 2 %
    and the orientation order parameter s within 0.02 absolute (measured:
    0.9 % and 0.0003 at most); the peak height within 2 % through 40,000 steps
    (measured 1.4 %), and after that within the standard error of the oracle's
    8-seed mean of the peak height (12 % there; measured 4.1 % and 4.7 %),
    the resolution 8 seeds give once trajectories have parted."""
import json
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1102_3094_gb300 import lf  # noqa: E402

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "oracle_long_256.json")
TRACK_UNTIL = 35_000          # report times at which every single trajectory is compared
MEAN_2PCT_UNTIL = 40_000      # report times at which the seed mean of the peak height is held to 2 %


def _gpu_series(seed, steps, every):
    sim = lf.Lattice(nx=256, ny=256, precision="fp32", xi=1e-3, tau=1.0, seed=seed)
    rows, done = [], 0
    for t in range(every, steps + 1, every):
        sim.step(t - done)
        done = t
        d = sim.diag()
        assert d["rc"] == 0, (seed, t)
        rows.append({"t": t, "k_peak": d["k_peak"], "s_peak": d["s_peak"], "s": d["orient_s"]})
    sim.close()
    return rows


def test_fp32_runs_against_oracle_over_50k_steps():
    gold = json.load(open(GOLDEN))
    cfg = gold["config"]
    seeds = sorted(int(k) for k in gold["runs"])
    runs = {s: gold["runs"][str(s)] for s in seeds}
    gpu = {s: _gpu_series(s, cfg["steps"], cfg["every"]) for s in seeds}
    nrep = min(len(r) for r in runs.values())
    assert nrep == cfg["steps"] // cfg["every"]
    for i in range(nrep):
        t = runs[seeds[0]][i]["t"]
        assert all(gpu[s][i]["t"] == t and runs[s][i]["t"] == t for s in seeds)
        if t <= TRACK_UNTIL:
            for s in seeds:
                d = abs(gpu[s][i]["s_peak"] / runs[s][i]["s_peak"] - 1)
                assert d < 0.01, ("trajectory", s, t, d)
        want = {k: np.mean([runs[s][i][k] for s in seeds]) for k in ("k_peak", "s_peak", "s")}
        got = {k: np.mean([gpu[s][i][k] for s in seeds]) for k in ("k_peak", "s_peak", "s")}
        assert abs(got["k_peak"] / want["k_peak"] - 1) < 0.02, (t, got, want)
        assert abs(got["s"] - want["s"]) < 0.02, (t, got, want)
        d_s = abs(got["s_peak"] / want["s_peak"] - 1)
        if t <= MEAN_2PCT_UNTIL:
            assert d_s < 0.02, (t, got, want)
        else:
            sem = np.std([runs[s][i]["s_peak"] for s in seeds], ddof=1) / np.sqrt(len(seeds)) / want["s_peak"]
            assert d_s < sem, (t, d_s, sem)
