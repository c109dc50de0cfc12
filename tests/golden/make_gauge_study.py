"""Write tests/golden/gauge_study.json from the oracle only.

FP64 solutions for the gauge and modified-Newton studies of Section 4
(Fig. 3 and Fig. 2 analogues on the 35 statistics), on the velocity-space
rule over the paper's box (u_x, u_r) in [-30.7, 37.3] x [0, 34.0]: 16 x 12
blocks of 8-point Gauss-Legendre, 10 azimuths.

  beta64_hermite[m], beta64_trivial[m]: the upstream Maxwellian of Mach
      2 + m (n = 1, T = 1, v = sqrt(5/3) Mach) in its Hermite gauge
      (moments e_0) and in the trivial gauge (moments T(g0, gH) e_0);
  passes64_*: Newton passes of Algorithm 1 in FP64 from the uniform
      density at tol 1e-6 and 1e-9 (the same in both gauges up to rounding:
      Newton's method with a backtracking line search is invariant under the
      linear change of statistics that a gauge transformation is);
  beta64_m4_sweep[k]: equilibrium plus M_(3,0,0) = 0.5 k / 25 in the trivial
      gauge.

Run: python tests/golden/make_gauge_study.py
"""
import json
import math
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import oracle as O  # noqa: E402

RULE = dict(rule_id=214, ax=-30.7, bx=37.3, nbx=16, br=34.0, nbr=12, ng=8, K=10)
MACHS = list(range(2, 13))


def main():
    r = RULE
    O.set_velocity_rule(r["rule_id"], r["ax"], r["bx"], r["nbx"], r["br"], r["nbr"], r["ng"], r["K"])
    q = r["rule_id"]
    B = len(MACHS)
    g0 = np.tile([0.0, 0.0, 0.0, 1.0, 1.0, 1.0], (B, 1))
    gH = g0.copy()
    gH[:, 0] = [math.sqrt(5.0 / 3.0) * m for m in MACHS]
    e0 = np.zeros((B, 35))
    e0[:, 0] = 1.0
    Mt = np.array([O.transform_M(g0[i], gH[i], e0[i]) for i in range(B)])
    # FP64 solutions, started next to them (the Maxwellian's own parameters).
    bh0 = e0.copy()
    bt0 = e0.copy()
    bt0[:, O.index_of(1, 0, 0)] = gH[:, 0]
    bh, sth, _ = O.solve_batch(q, e0, beta0=bh0, tol=1e-13, g=gH, final_step=True)
    bt, stt, _ = O.solve_batch(q, Mt, beta0=bt0, tol=1e-13, g=g0, final_step=True)
    assert all(s & 1 for s in sth) and all(s & 1 for s in stt)
    out = {"_source": "oracle/mem_oracle.c (or_solve, or_transform_M), Section 4 Fig. 2 and Fig. 3 setups",
           "rule": RULE, "mach": MACHS, "beta64_hermite": bh.tolist(), "beta64_trivial": bt.tolist()}
    uni = e0.copy()
    for a, b, c in ((2, 0, 0), (0, 2, 0), (0, 0, 2)):
        uni[:, O.index_of(a, b, c)] = math.sqrt(0.5)
    for tol in (1e-6, 1e-9):
        _, sh_, ih = O.solve_batch(q, e0, beta0=uni, tol=tol, g=gH)
        _, st_, it_ = O.solve_batch(q, Mt, beta0=uni, tol=tol, g=g0)
        out["passes64_hermite_tol_%g" % tol] = ih.tolist()
        out["passes64_trivial_tol_%g" % tol] = it_.tolist()
        out["status64_hermite_tol_%g" % tol] = sh_.tolist()
        out["status64_trivial_tol_%g" % tol] = st_.tolist()
    n = 26
    Ms = np.zeros((n, 35))
    Ms[:, 0] = 1.0
    Ms[:, O.index_of(3, 0, 0)] = np.linspace(0.0, 0.5, n)
    b0 = np.zeros((n, 35))
    b0[:, 0] = 1.0
    bs, sts, its = O.solve_batch(q, Ms, beta0=b0, tol=1e-13, g=g0[:1].repeat(n, 0), final_step=True)
    assert all(s & 1 for s in sts)
    out["m4"] = np.linspace(0.0, 0.5, n).tolist()
    out["beta64_m4_sweep"] = bs.tolist()
    out["passes64_m4_sweep"] = its.tolist()
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "gauge_study.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=0)
    print(path)


if __name__ == "__main__":
    main()
