"""Write tests/golden/mach10_paper_mesh.json from the oracle only.

The paper's Mach-10 setup (Section 4): 150 cells on [-47.1, 47.1], tanh
start with thickness 15.7, the velocity-space rule on the Rankine-Hugoniot
box of Appendix D (n = 5; 6 x 4 blocks of 8-point Gauss-Legendre in
(u_x, u_r), 12 azimuths), FP64 Algorithm 1 (tol 1e-8, maxI 500, the paper's
order), CFL 0.5.  Stored: rho, u_x, T and the simulated time after 100 local
Lax-Friedrichs steps and after 60 FLIC steps (the FLIC oracle solves every
interface from a cold start, twice, so its steps are expensive).

Run: python tests/golden/make_mach10_paper_mesh.py   (about 30 min on 8 cores)
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import oracle as O  # noqa: E402

RULE_ID = 200
STEPS = {"lf": 100, "flic": 60}


def main():
    d = O.shock_domain(10.0)
    O.set_velocity_rule(RULE_ID, d[0], d[1], 6, d[2], 4, 8, 12)
    out = {"_source": "oracle/mem_oracle.c (or_shock_step), Section 4 Mach-10 setup", "mach": 10.0, "ncells": 150,
           "domain": [-47.1, 47.1], "thickness": 15.7, "rule": {"nbx": 6, "nbr": 4, "ng": 8, "K": 12,
                                                                  "box": list(map(float, d))}}
    for scheme, n in STEPS.items():
        so = O.Shock(10.0, 150, -47.1, 47.1, order=RULE_ID, ic="tanh", thickness=15.7, scheme=scheme)
        for _ in range(n):
            so.step()
        rho, ux, T = so.profile()
        assert np.isfinite(rho).all() and np.isfinite(T).all()
        out[scheme] = {"steps": n, "t": so.t, "rho": rho.tolist(), "ux": ux.tolist(), "T": T.tolist(),
                       "up": [so.n_up, so.v_up, so.T_up], "down": [so.n_dn, so.v_dn, so.T_dn]}
        print(scheme, n, so.t, flush=True)
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "mach10_paper_mesh.json"), "w") as f:
        json.dump(out, f)


if __name__ == "__main__":
    main()
