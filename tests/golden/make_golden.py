"""Write tests/golden/rh_and_speed.json from the oracle only.

The stored values are Rankine-Hugoniot states (Appendix D, Eq. "RH
condition") and equilibrium characteristic speeds, used by the GPU tests on
boxes where re-deriving them is not wanted.  Run: python tests/golden/make_golden.py
"""
import json
import math
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import oracle as O  # noqa: E402


def main():
    out = {"_source": "oracle/mem_oracle.c (or_rh, or_flux at beta = 0); Appendix D RH condition, Eq. 'The lax F'"}
    for mach in (1.2, 1.5, 4.0, 10.0):
        r, t = O.rh(mach)
        v1 = math.sqrt(5.0 / 3.0) * mach
        r2 = math.sqrt(5 + math.sqrt(10))
        out["mach_%g" % mach] = {"rho_ratio": r, "T_ratio": t, "v_up": v1, "v_dn": v1 / r,
                                 "speed_up": v1 + r2, "speed_dn": v1 / r + r2 * math.sqrt(t)}
        _, sp, _, _ = O.flux(8, [0.0] * 35, [v1 / r, 0, 0, math.sqrt(t), math.sqrt(t), math.sqrt(t)], r)
        out["mach_%g" % mach]["speed_dn_oracle_q8"] = sp
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "rh_and_speed.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print(path)


if __name__ == "__main__":
    main()
