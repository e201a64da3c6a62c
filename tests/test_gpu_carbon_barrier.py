"""Barrier parity on converged Tersoff carbon bands (Sec. II.A climbing
image, Sec. II.C cell filter).

1. Diamond vacancy hop between endpoints relaxed by the oracle
   (cfneb_inputs.diamond_vacancy_hop_relaxed), k = 0.1 eV/A^2, FIRE dt 0.05,
   dt_max 0.2, maxstep 0.1, climbing image on.  A continuous band whose
   climbing image sits on the hop's saddle (the energy along each segment
   rises monotonically to it).
   * 511 atoms, fixed cell, 5 images, fmax 1e-3: the FP64 oracle's barrier
     against the GPU's, mixed within 1 meV and FP64 within 1e-6 eV.
   * 98,303 atoms (16 x 24 x 32 cells), cell filter on, 11 images (and
     adaptive refinement between 8 and 24 images), fmax 0.05 eV/A: mixed
     within 1 meV of the FP64 path, both within 0.01 eV of the 511-atom
     oracle barrier (the finite-size and cell-relaxation effect is ~2 meV).
   Symmetric hops use an odd image count so that one image starts on the
   saddle: with an even count the climbing image is one of the two images
   flanking it, which the mixed path's step energies cannot order, and from
   the other one its climb can end on another stationary point of Tersoff's
   rough surface (FP64 bands converge either way).

2. Graphite -> hexagonal diamond, the 2 x 2 x 2 tiling of the 8-atom cells
   (64 atoms), 9 images, interior jitter N(0, 0.01 A) from seed 2510,
   k = 0.1 eV/A^2, FIRE dt 0.1: the FP64 oracle relaxes it to fmax < 1e-3
   eV/A, the GPU the same inputs in mixed precision and in FP64; the
   barriers must agree within 1 meV (mixed) and 1e-6 eV (FP64) and all
   three climb on the same image.  This is a parity check of a converged
   stationary point, not the graphite -> diamond barrier: Tersoff's 2.1 A
   cutoff leaves graphite layers 3.35 A apart interaction-free, the
   relaxed images 1-6 are flat graphite at different layer spacings, and
   the climbing image (0.085 eV/atom) sits just outside the interacting
   region while the energy along the last segment to diamond rises to
   ~0.9 eV/atom: the whole transformation lies in one segment.
"""
import numpy as np
import pytest

import cfneb_inputs as ci
from _cases import gpu_band, oracle_band

pytestmark = pytest.mark.gpu

FTOL = 1e-3


@pytest.fixture(scope="module")
def g():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2510_16721_gb300 as g
    g.build()
    return g


@pytest.fixture(scope="module")
def oracle_result(oracle_mod):
    cfg = ci.tersoff_graphite_hexdiamond(reps=(2, 2, 2))
    R0, h0, R1, h1 = cfg["endpoints"]
    ob = oracle_band(oracle_mod, oracle_mod.Tersoff(), R0, h0, R1, h1, 9, k=0.1, dt=0.1,
                     cell_filter=True, noise=cfg["noise"])
    steps, conv = ob.relax(FTOL, 40000)
    assert conv
    return dict(barrier=ob.barrier(), ci=ob.ci, steps=steps, E=np.array(ob.E))


@pytest.mark.parametrize("precision, tol", [(1, 1e-3), (0, 1e-6)])
def test_converged_carbon_barrier_matches_oracle(g, oracle_result, precision, tol):
    cfg = ci.tersoff_graphite_hexdiamond(reps=(2, 2, 2))
    R0, h0, R1, h1 = cfg["endpoints"]
    b = gpu_band(g, R0, h0, R1, h1, 9, g.tersoff_potential(), k=0.1, dt=0.1,
                 cell_filter=True, noise=cfg["noise"], precision=precision)
    steps, conv = b.relax(FTOL, 40000)
    assert conv
    path = b.get_path()
    E = path["energies"]
    barrier = E.max() - E[0]
    assert path["fmax"] < FTOL
    assert abs(barrier - oracle_result["barrier"]) <= tol, (barrier, oracle_result["barrier"])
    assert int(np.argmax(E[1:-1])) + 1 == oracle_result["ci"]
    # the endpoints are the oracle's (the FP64 energy pass of the stored X)
    assert abs((E[-1] - E[0]) - (oracle_result["E"][-1] - oracle_result["E"][0])) <= 1e-6
    print("precision %d: barrier %.9f eV in %d steps (oracle %.9f eV in %d steps)"
          % (precision, barrier, steps, oracle_result["barrier"], oracle_result["steps"]))


# ---- diamond vacancy hop between relaxed endpoints ---------------------------

VAC = dict(k=0.1, dt=0.05, dt_max=0.2, maxstep=0.1)
VAC_SMALL, VAC_LARGE = (4, 4, 4), (16, 24, 32)


@pytest.fixture(scope="module")
def oracle_vacancy(oracle_mod):
    R0, h0, R1, h1 = ci.diamond_vacancy_hop_relaxed(VAC_SMALL)
    ob = oracle_band(oracle_mod, oracle_mod.Tersoff(), R0, h0, R1, h1, 5, cell_filter=False,
                     **VAC)
    steps, conv = ob.relax(FTOL, 20000)
    assert conv
    return dict(barrier=ob.barrier(), ci=ob.ci, steps=steps)


@pytest.mark.parametrize("precision, tol", [(1, 1e-3), (0, 1e-6)])
def test_vacancy_hop_barrier_matches_oracle(g, oracle_vacancy, precision, tol):
    R0, h0, R1, h1 = ci.diamond_vacancy_hop_relaxed(VAC_SMALL)
    b = gpu_band(g, R0, h0, R1, h1, 5, g.tersoff_potential(), cell_filter=False,
                 precision=precision, **VAC)
    steps, conv = b.relax(FTOL, 20000)
    assert conv
    E = b.get_path()["energies"]
    barrier = E.max() - E[0]
    assert abs(barrier - oracle_vacancy["barrier"]) <= tol, (barrier, oracle_vacancy)
    assert int(np.argmax(E[1:-1])) + 1 == oracle_vacancy["ci"] == 2
    print("precision %d: barrier %.9f eV in %d steps (oracle %.9f eV in %d steps)"
          % (precision, barrier, steps, oracle_vacancy["barrier"], oracle_vacancy["steps"]))


@pytest.fixture(scope="module")
def large_vacancy():
    return ci.diamond_vacancy_hop_relaxed(VAC_LARGE)


@pytest.mark.parametrize("adaptive", [False, True])
def test_large_vacancy_hop_mixed_barrier_matches_fp64(g, oracle_vacancy, large_vacancy,
                                                      adaptive):
    """98,303 atoms, cell filter on, 11 images (adaptive: 8..24), fmax 0.05:
    the mixed path's converged barrier within 1 meV of the FP64 path's."""
    R0, h0, R1, h1 = large_vacancy
    out = {}
    for precision in (1, 0):
        b = gpu_band(g, R0, h0, R1, h1, 11, g.tersoff_potential(), cell_filter=True,
                     precision=precision, adaptive=adaptive, n_min=8, n_max=24, **VAC)
        steps, conv = b.relax(0.05, 6000)
        assert conv, (precision, steps)
        path = b.get_path()
        E = path["energies"]
        assert path["fmax"] < 0.05
        out[precision] = (E.max() - E[0], steps, b.n_images)
        b.destroy()
    (bm, sm, nm), (bd, sd, nd) = out[1], out[0]
    assert abs(bm - bd) <= 1e-3, out
    # the saddle the 511-atom oracle band climbs to, up to the finite-size
    # and cell-relaxation effect
    assert abs(bd - oracle_vacancy["barrier"]) <= 1e-2, (bd, oracle_vacancy)
    print("98,303 atoms: mixed %.6f eV (%d steps, %d images), FP64 %.6f eV (%d steps, %d "
          "images), oracle 511 atoms %.6f eV" % (bm, sm, nm, bd, sd, nd,
                                                 oracle_vacancy["barrier"]))
