"""Writes the stored oracle cases under tests/golden/.

Calls only the FP64 oracle and the seeded input generator.  The paper prints
no worked numerical example, so these files pin the oracle against its own
earlier output (regression) and serve as fixed expectations for smoke checks.
Run from the repository root:  python tests/golden/make_golden.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import oracle as O  # noqa: E402
from paper_1503_00330_b300 import workloads as W  # noqa: E402


def tiny():
    K, T, L, seed, n_obs = 8, 6, 3, 7, 2
    p = W.problem(K, T, L, seed=seed, n_obs=n_obs)
    u, c = O.pi_update(p.model, p.cost, p.x0, p.u_nom, K, T, p.lam, p.sigma_u, seed)
    return {"source": "oracle/pi_oracle.c via tests/golden/make_golden.py",
            "K": K, "T": T, "L": L, "seed": seed, "n_obs": n_obs,
            "u_out": u.tolist(), "costs_out": c.tolist()}


if __name__ == "__main__":
    with open(os.path.join(HERE, "tiny_update.json"), "w") as f:
        json.dump(tiny(), f, indent=1)
        f.write("\n")
