"""Writes the stored expected values under tests/golden/ by calling only the
CPU oracle (and the seeded input generator). Run from the repository root:
    python tests/golden/make_golden.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from paper_1708_00744_b300 import inputs  # noqa: E402


def sweep_case(n, seed, sigma, nsweeps, K):
    a = inputs.initial_matrix(seed, n)
    g = np.stack([inputs.proposal_gaussians(seed, s, n) for s in range(nsweeps)])
    u = np.stack([inputs.metropolis_uniforms(seed, s, n) for s in range(nsweeps)])
    method = oracle.SM if K == 1 else oracle.DELAYED
    out = oracle.sweeps(method, a, g, u, sigma, K=K)
    sg0, la0 = oracle.slogdet(a)
    return {
        "n": n, "seed": seed, "sigma": sigma, "nsweeps": nsweeps, "K": K,
        "method": "sherman-morrison (Eq. 2)" if K == 1 else "delayed rank-K (Eq. 3-4)",
        "initial_logabs": la0, "initial_sign": sg0,
        "accepted": ["".join("1" if x else "0" for x in row) for row in out["accepted"]],
        "ratios": [[float(x) for x in row] for row in out["ratios"]],
        "final_logabs": out["logabs"], "final_sign": out["sign"],
        "near_ties": out["near_ties"],
        "ainv_frobenius": float(np.linalg.norm(out["Ainv"])),
    }


def main():
    cases = [sweep_case(64, 0, 0.1, 1, 1), sweep_case(64, 0, 0.1, 1, 8)]
    doc = {
        "source": "CPU oracle (oracle/qmc_oracle.c) on seeded synthetic inputs; "
                  "one Metropolis sweep of a 64-electron walker, A_ij ~ N(0,1) from seed 0, "
                  "proposal v = a_j + 0.1 g (Sec. I move, Sec. II delayed scheme)",
        "cases": cases,
    }
    with open(os.path.join(HERE, "sweep_n64_seed0.json"), "w") as f:
        json.dump(doc, f, indent=1)
        f.write("\n")


if __name__ == "__main__":
    main()
