"""TEST INFRASTRUCTURE (an input generator run by hand, never by the product).

Relax the endpoints of a vacancy hop in Tersoff carbon diamond with the
oracle, in a 4 x 4 x 4 conventional cell (511 atoms), at the fixed lattice
constant of the diamond workloads.

Writes cfneb_inputs/data/tersoff_c_diamond_vacancy_4x4x4.json: for every atom
its ideal site as an integer offset from the vacant site in units of a/4, and
its relaxed displacement from that site in the initial state (vacancy at
site 0) and in the final state (the hopping atom on site 0).  Larger
supercells embed this field around the vacancy
(cfneb_inputs.diamond_vacancy_hop_relaxed).  Runs the FP64 CPU reference
only: single-image FIRE at a fixed cell until the largest force is below
1e-6 eV/A.  Usage: python -m oracle.make_diamond_vacancy_endpoints
"""
import json
import os

import numpy as np

import cfneb_inputs
from oracle import Tersoff, AtomicImage, to_generalized, relax_single, Fire

REPS = (4, 4, 4)


def relax_fixed_cell(R, h, fmax=1e-6):
    n = len(R)
    img = AtomicImage(Tersoff(), h, c=n, cell_filter=False)
    X = to_generalized(R, h, h, n)
    X, E, steps, ok = relax_single(img, X, fmax, 20000, Fire(dt=0.05, maxstep=0.05))
    if not ok:
        raise RuntimeError("endpoint relaxation did not converge")
    return X[:n].copy(), E, steps


def main():
    a = cfneb_inputs.DIAMOND_A
    R0, h, R1, _ = cfneb_inputs.diamond_vacancy_hop(a, REPS)
    Rf, _ = cfneb_inputs.diamond(a, *REPS)
    site = Rf[0]
    hop = int(np.flatnonzero(np.any(R1 != R0, axis=1))[0])
    # ideal site of every atom relative to the vacancy, minimum image
    s = (R0 - site) @ np.linalg.inv(h)
    s -= np.round(s)
    off = np.rint(s @ h / (a / 4.0)).astype(int)
    assert np.allclose(off * (a / 4.0), s @ h, atol=1e-9)
    X0, E0, n0 = relax_fixed_cell(R0, h)
    X1, E1, n1 = relax_fixed_cell(R1, h)
    # R0 and R1 are ideal sites (R1[hop] is the vacant site itself)
    d0 = X0 - R0
    d1 = X1 - R1
    out = dict(
        description="Tersoff 1988 C diamond (a = %.4f A): vacancy hop in a 4 x 4 x 4 "
                    "conventional cell (511 atoms), both endpoints relaxed at fixed cell "
                    "with the FP64 CPU reference (FIRE, fmax < 1e-6 eV/A).  offset: ideal "
                    "site minus the vacant site in units of a/4 (minimum image); d0, d1: "
                    "relaxed displacement from the ideal site in the initial and final "
                    "state; the hopping atom's d1 is measured from the vacant site." % a,
        a=a, reps=list(REPS), hop=hop, E_initial=E0, E_final=E1,
        offset=off.tolist(), d0=np.round(d0, 15).tolist(), d1=np.round(d1, 15).tolist())
    path = os.path.join(os.path.dirname(cfneb_inputs.__file__), "data",
                        "tersoff_c_diamond_vacancy_4x4x4.json")
    with open(path, "w") as f:
        json.dump(out, f, separators=(",", ":"))
    print("initial E %.9f (%d steps), final E %.9f (%d steps), hop atom %d"
          % (E0, n0, E1, n1, hop))


if __name__ == "__main__":
    main()
