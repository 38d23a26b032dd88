"""Writes small2d_oracle.json beside this script: values the FP64 oracle computes for the
small2d workload (unit square, 32 x 32 right triangles, 1089 nodes, 50 observations, the
bilaplacian prior with gamma = 0.1, delta = 0.5; k = 20, p = 10).

The paper prints no worked numeric example, so the stored values are the oracle's own,
written by this script, which calls only ``oracle/`` and the seeded input generators of
``workloads.py``.  ``tests/test_golden.py`` recomputes them: the file records what the
oracle computed when its pins last passed, so any later change to the oracle's arithmetic
shows up as a difference and has to be made on purpose (re-run this script and name, in
the commit, the passage of the paper that justifies the change).

Stored (Section 2: cost, eq. (cost); gradient, eq. (firstcontrol); Algorithm 1: inexact
Newton-CG to a relative gradient of 1e-9; Algorithm 2 with Omega from the workload's
seeded normals):
  J and |g| at m = 0 (the prior mean);
  Newton iterations, J, |m|_2 and m at eight fixed nodes at the MAP point;
  the k = 20 leading eigenvalues of the prior-preconditioned misfit Hessian at the MAP.

Run from the repository root:  python tests/golden/make_golden.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import workloads as W  # noqa: E402
from oracle import algorithms as A  # noqa: E402
from oracle.inverse import make_problem  # noqa: E402

NODES = [0, 100, 300, 544, 545, 700, 900, 1088]


def compute():
    w = W.WORKLOADS["small2d"]
    orc, _, _ = make_problem(w, W.draws(w))
    m0 = orc.m_prior.copy()
    g0, J0, _, _ = orc.gradient(m0)
    res = A.newton_cg(orc, rel_tol=1e-9)
    u = orc.forward(res.m)
    J = orc.cost(res.m, u)[0]
    lam, _ = A.lowrank_eig(orc, res.m, W.omega(w), w.k)
    return {
        "workload": "small2d: 2D 32x32 P1 right triangles, n=1089, q=50, gamma=0.1, delta=0.5, k=20, p=10",
        "J_prior_mean": float(J0),
        "gradient_norm_prior_mean": float(np.linalg.norm(g0)),
        "newton_rel_tol": 1e-9,
        "newton_converged": bool(res.converged),
        "newton_iterations": int(res.iterations),
        "J_map": float(J),
        "m_map_norm": float(np.linalg.norm(res.m)),
        "m_map_nodes": NODES,
        "m_map_at_nodes": [float(res.m[i]) for i in NODES],
        "eigenvalues": [float(x) for x in lam],
    }


if __name__ == "__main__":
    out = os.path.join(HERE, "small2d_oracle.json")
    with open(out, "w") as f:
        json.dump(compute(), f, indent=1)
        f.write("\n")
    print("wrote", out)
