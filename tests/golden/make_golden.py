"""Writes the oracle-only regression fixtures in this folder.

Every stored value comes from the oracle (oracle/) applied to the seeded synthetic inputs
(paper_2101_08563_gb300/synth.py); nothing here runs the CUDA path.

    python tests/golden/make_golden.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import fastfca as ff  # noqa: E402
from paper_2101_08563_gb300 import synth  # noqa: E402


def trajectory_m2n3():
    g = {"M": 2, "N": 3, "F": 5, "T": 48, "K": 4, "seed": 31, "iters": 12}
    mix = synth.generate_mixture(g["M"], g["N"], g["F"], g["T"], g["K"], seed=g["seed"])
    p = synth.random_init(mix.x, g["N"], seed=g["seed"])
    out = ff.run(mix.x, p.P, p.lam, p.v, iters=g["iters"])
    g["_source"] = "oracle.fastfca.run (Algorithm 1) on synth.generate_mixture, written by make_golden.py"
    g["ll"] = out["ll"].tolist()
    with open(os.path.join(HERE, "oracle_trajectory_m2n3.json"), "w") as fh:
        json.dump(g, fh, indent=1)


if __name__ == "__main__":
    trajectory_m2n3()
