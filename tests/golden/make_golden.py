"""Writes tests/golden/counts.json: eigenvalue counts inside the contour by the argument
principle (winding of det T(z), Sec. 2), computed with the oracle only.

Run from the repository root:  python tests/golden/make_golden.py
"""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import synth  # noqa: E402
from oracle import count  # noqa: E402


def main():
    out = {}
    for name in ["delay1d_n64", "delay2d_s64"]:
        p = synth.config_problem(name, seed=0)
        out[name] = {"count": count.count_inside(p), "seed": 0,
                     "source": "oracle.count.count_inside (argument principle, Sec. 2)"}
        print(name, out[name])
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "counts.json"), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
