"""Writes tests/golden/fullsize_<config>.json and .npz: the oracle's whole contour-integral pass
on the two wide-band workloads, for the full-size parity tests on the GPU.

  drude2d_s128  Drude NEP on a 128 x 128 grid (n = 16384, bandwidth 128), ellipse c = 2,
                a = 1, b = 0.2, N = 128, L = 32, M = 8
  sqrt3d_s24    square-root NEP on a 24^3 grid (n = 13824, bandwidth 576), circle c = 4,
                r = 1.5, N = 64, L = 24, M = 8

Both at problem seed 0 with the probe block synth.random_probe_block(n, L, 0). The JSON file
holds the eigenvalues and scaled residuals of the returned pairs, the Hankel rank m, the
Rayleigh-Ritz basis rank, the Hankel singular values and the Frobenius norm of the moment
block S = [S_0 .. S_{M-1}]; the .npz file holds the moment block on a fixed set of rows
(every (n // rows)-th row), which the GPU test compares element by element.

Everything here comes from oracle/ (plain FP64 numpy and the C band LU) and synth/.
Run from the repository root:  python tests/golden/make_golden_fullsize.py [config ...]
(about 2 minutes for the Drude workload and 10 for the square-root one on 8 cores).
"""
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import synth  # noqa: E402
from oracle import ciss  # noqa: E402

CONFIGS = ["drude2d_s128", "sqrt3d_s24"]
SAMPLE_ROWS = 48


def sample_rows(n: int, count: int = SAMPLE_ROWS) -> np.ndarray:
    step = max(1, n // count)
    return np.arange(0, n, step)[:count] + (step // 2)


def main(names):
    for name in names:
        t0 = time.time()
        p = synth.config_problem(name, seed=0)
        V = synth.random_probe_block(p.n, p.L, 0)
        r = ciss.solve(p, V=V)
        rows = sample_rows(p.n)
        S = r["S"]
        meta = {
            "config": name, "seed": 0, "probe_seed": 0, "n": p.n, "N": p.N, "L": p.L, "M": p.M,
            "lam_re": [float(x.real) for x in r["lam"]], "lam_im": [float(x.imag) for x in r["lam"]],
            "eta": [float(x) for x in r["eta"]], "hankel_rank": int(r["m"]), "basis_rank": int(r["rank_basis"]),
            "sigma": [float(x) for x in r["sigma"]], "S_fro": float(np.linalg.norm(S)),
            "max_backward": float(np.max(r["beta"])), "max_sweeps": int(np.max(r["sweeps"])),
            "rows": [int(x) for x in rows],
            "source": "oracle.ciss.solve (FP64 contour-integral pass), tests/golden/make_golden_fullsize.py",
            "seconds": round(time.time() - t0, 1),
        }
        with open(os.path.join(HERE, f"fullsize_{name}.json"), "w") as f:
            json.dump(meta, f, indent=1)
        np.savez_compressed(os.path.join(HERE, f"fullsize_{name}.npz"), S_rows=S[:, rows, :])
        print(name, "eigenvalues", len(r["lam"]), "m", r["m"], "seconds", meta["seconds"], flush=True)


if __name__ == "__main__":
    main(sys.argv[1:] or CONFIGS)
