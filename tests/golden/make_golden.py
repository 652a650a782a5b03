"""Write the golden values of the paper's worked example (oracle only).

The example of the paper's section "Definition of Dirac operators": a 4^4
lattice, cold start (all links 1), Wilson operator with kappa = 0.141139 and
eps_CG = 1.0e-8, applied to and solved on a Gaussian pseudofermion.  The
paper prints the commands but no output, so the stored numbers are this
oracle's: D x, and the solution y of D y = x by CG on D^dag D (tol 1e-12, to
leave room below the paper's 1e-8), on the seeded Gaussian source of
paper_2409_03030_gb300.synth (seed 123, the paper's Random.seed!(123)).  The
time direction is antiperiodic, as everywhere in this project.

Run:  python tests/golden/make_golden.py   (rewrites paper_example_4x4x4x4.json)
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2409_03030_gb300 import synth  # noqa: E402

DIMS = (4, 4, 4, 4)
KAPPA = 0.141139
SEED = 123
TOL = 1e-12
# sampled components (alpha, t, z, y, x, colour); the first is the paper's y[1,1,1,1,1,1]
SAMPLES = [(0, 0, 0, 0, 0, 0), (3, 3, 3, 3, 3, 2), (1, 2, 0, 3, 1, 1), (2, 1, 3, 0, 2, 0),
           (0, 3, 1, 2, 0, 2), (3, 0, 2, 1, 3, 1), (1, 1, 1, 1, 1, 0), (2, 2, 2, 2, 2, 2)]


def compute():
    U = synth.gauge(DIMS, "unit")
    x = synth.gaussian_spinor(DIMS, seed=SEED)
    dx = oracle.dirac(DIMS, U, x, KAPPA)
    y, iters, sys_rel, full_rel, ok = oracle.solve(DIMS, U, x, KAPPA, eo=False, tol=TOL,
                                                   maxiter=100000)
    assert ok, "oracle CG did not converge"
    cplx = lambda v: [float(v.real), float(v.imag)]  # noqa: E731
    return {
        "source": "paper, section 'Definition of Dirac operators': 4^4 cold start, "
                  "kappa = 0.141139, eps_CG = 1.0e-8; values from oracle/ via "
                  "tests/golden/make_golden.py",
        "dims": list(DIMS), "kappa": KAPPA, "links": "unit (cold start)",
        "t_antiperiodic": True, "source_seed": SEED, "cg_tol": TOL,
        "layout": "spinor index (alpha, t, z, y, x, colour)",
        "norm_x": float(np.linalg.norm(x)),
        "norm_Dx": float(np.linalg.norm(dx)),
        "norm_y": float(np.linalg.norm(y)),
        "cg_iters": int(iters),
        "system_true_rel_resid": float(sys_rel),
        "full_rel_resid": float(full_rel),
        "samples": [list(s) for s in SAMPLES],
        "Dx": [cplx(dx[s]) for s in SAMPLES],
        "y": [cplx(y[s]) for s in SAMPLES],
    }


if __name__ == "__main__":
    out = os.path.join(HERE, "paper_example_4x4x4x4.json")
    with open(out, "w") as fh:
        json.dump(compute(), fh, indent=1)
        fh.write("\n")
    print(out)
