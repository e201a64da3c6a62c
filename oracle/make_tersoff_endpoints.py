"""TEST INFRASTRUCTURE (an input generator run by hand, never by the product).

Relax the 8-atom graphite and hexagonal-diamond cells with the oracle.

Writes cfneb_inputs/data/tersoff_c_endpoints_8atom.json, the endpoints every
Tersoff workload is tiled from.  Runs the FP64 CPU reference only:
single-image FIRE in the rotation-free cell-filter coordinates (so both the
atoms and the cell relax) until the largest generalised-force row is below
1e-6 eV/A.  Usage: python -m oracle.make_tersoff_endpoints
"""
import json
import os

import numpy as np

import cfneb_inputs
from oracle import Tersoff, AtomicImage, to_generalized, from_generalized, relax_single, Fire


def relax_cell(R, h, fmax=1e-6):
    pot = Tersoff()
    n = len(R)
    img = AtomicImage(pot, h, c=n, cell_filter=True)
    X = to_generalized(R, h, h, n)
    X, E, steps, ok = relax_single(img, X, fmax, 20000, Fire(dt=0.05, maxstep=0.05))
    if not ok:
        raise RuntimeError("endpoint relaxation did not converge")
    R1, h1, _ = from_generalized(X, h, n)
    return R1, h1, E, steps


def main():
    s_g, h_g, s_d, h_d = cfneb_inputs.graphite_hexdiamond_cells()
    Rg, hg, Eg, ng = relax_cell(s_g @ h_g, h_g)
    Rd, hd, Ed, nd = relax_cell(s_d @ h_d, h_d)
    out = dict(
        description="Tersoff 1988 C: AB graphite and hexagonal diamond, 8-atom "
                    "orthohexagonal cells with matched atom order, relaxed with the "
                    "FP64 CPU reference (cell filter + FIRE, fmax < 1e-6 eV/A).",
        R_graphite=Rg.tolist(), h_graphite=hg.tolist(), E_graphite=Eg,
        R_hexdiamond=Rd.tolist(), h_hexdiamond=hd.tolist(), E_hexdiamond=Ed)
    path = os.path.join(os.path.dirname(cfneb_inputs.__file__), "data",
                        "tersoff_c_endpoints_8atom.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print("graphite E/atom %.6f (%d steps), h diag %s" % (Eg / 8, ng, np.diag(hg)))
    print("hexdiamond E/atom %.6f (%d steps), h diag %s" % (Ed / 8, nd, np.diag(hd)))


if __name__ == "__main__":
    main()
