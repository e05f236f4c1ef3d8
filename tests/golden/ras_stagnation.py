"""Writes ras_stagnation.json: the oracle's Krylov solves of scaled-down
space-time heat problems (the operator, overlap ratio 1.4, weight range and
rank rule of the configured 8 x 8 x 4 workload; fewer subdomains, points and
neurons so that the oracle finishes), with the four Schwarz/Krylov pairs of
Sec. 3 and Sec. 5: AS-CG, AS-GMRES(50), SAS-GMRES(50) and RAS-GMRES(50)
(Boolean D_i), all to a relative residual of 1e-10 from W = 0, at most 1500
iterations.  Record per pair: iterations, the final stopping quantity, the
float64 normal-equation residual, and the stopping quantity after 50 and 500
iterations.  It shows that the stagnation of RAS-GMRES on the full workload
is a property of the method with the Boolean D_i, not of the GPU's
double-float factors.  Uses only the oracle; run: python ras_stagnation.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import rann_inputs as ri  # noqa: E402
from oracle import solver as sv  # noqa: E402

CASES = [dict(sub=(3, 3, 2), pts=(6, 6, 4), neurons=40), dict(sub=(4, 4, 2), pts=(6, 6, 4), neurons=60)]


def main():
    out = []
    for kw in CASES:
        p = ri.heat3d(**kw)
        S = sv.build_system(p)
        rec = {"problem": {"sub": list(kw["sub"]), "pts": list(kw["pts"]), "neurons": kw["neurons"]},
               "J": p.J, "dof": S.dof}
        for kind, solver in (("as", "cg"), ("as", "gmres"), ("sas", "gmres"), ("ras", "gmres")):
            sol = sv.solve(S, solver, sv.schwarz(S, kind), 1e-10, 50, 1500)
            h = sol.history
            rec[f"{kind}-{solver}"] = {"iters": sol.iters, "final": float(h[-1]),
                                       "normal_residual": float(sol.rel_res_normal),
                                       "after_50": float(h[min(50, len(h) - 1)]),
                                       "after_500": float(h[min(500, len(h) - 1)])}
        out.append(rec)
        print(json.dumps(rec), flush=True)
    json.dump({"source": "oracle (this script)", "cases": out}, open(os.path.join(HERE, "ras_stagnation.json"), "w"),
              indent=1)


if __name__ == "__main__":
    main()
