"""Pins of the oracle's NEB, climbing image, FIRE and refinement.

The Mueller-Brown surface (published stationary points and an independent
Newton solve) pins the tangent/projection/CI/FIRE chain; the LJ vacancy hop
and the Tersoff carbon vacancy hop pin symmetry and the saddle energy
(constrained minimisation of the midpoint image with scipy); rotating both
endpoints must leave the
converged path unchanged; insertion/deletion must keep the endpoints.
"""
import json
import math
import os

import numpy as np
import pytest
from scipy.optimize import minimize, root

import cfneb_inputs as ci

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_upwind_tangent_cases(oracle_mod):
    Xm, X0, Xp = np.array([0.0, 0.0]), np.array([1.0, 0.0]), np.array([1.0, 2.0])
    tp, tm = Xp - X0, X0 - Xm
    t = oracle_mod.upwind_tangent
    np.testing.assert_array_equal(t(Xm, X0, Xp, 0.0, 1.0, 2.0), tp)      # uphill to the right
    np.testing.assert_array_equal(t(Xm, X0, Xp, 2.0, 1.0, 0.0), tm)      # uphill to the left
    # maximum: weighted, the higher neighbour gets the larger weight
    np.testing.assert_allclose(t(Xm, X0, Xp, 0.5, 1.0, 0.0), tp * 0.5 + tm * 1.0)
    np.testing.assert_allclose(t(Xm, X0, Xp, 0.0, 1.0, 0.5), tp * 1.0 + tm * 0.5)
    # minimum
    np.testing.assert_allclose(t(Xm, X0, Xp, 3.0, 1.0, 2.0), tp * 1.0 + tm * 2.0)
    # exact tie falls to the weighted branch; all equal -> tp + tm
    np.testing.assert_allclose(t(Xm, X0, Xp, 1.0, 1.0, 2.0), tp * 1.0 + tm * 0.0)
    np.testing.assert_allclose(t(Xm, X0, Xp, 1.0, 1.0, 1.0), tp + tm)


def test_neb_projection_algebra(oracle_mod):
    """f_NEB is perpendicular-plus-spring: its tangential part is the spring."""
    rng = np.random.default_rng(0)
    X = np.cumsum(rng.normal(size=(6, 5)), axis=0)
    E = np.array([0.0, 1.0, 3.0, 2.5, 1.0, -1.0])
    F = rng.normal(size=(6, 5))
    k = 0.7
    out, ci_ = oracle_mod.neb_forces(X, E, F, k, climb=True)
    assert ci_ == 2
    for i in range(1, 5):
        tau = oracle_mod.upwind_tangent(X[i - 1], X[i], X[i + 1], E[i - 1], E[i], E[i + 1])
        th = tau / np.linalg.norm(tau)
        perp = F[i] - np.dot(F[i], th) * th
        np.testing.assert_allclose(out[i] - np.dot(out[i], th) * th, perp, atol=1e-12)
        if i == ci_:
            assert abs(np.dot(out[i], th) + np.dot(F[i], th)) < 1e-12
        else:
            spring = k * (np.linalg.norm(X[i + 1] - X[i]) - np.linalg.norm(X[i] - X[i - 1]))
            assert abs(np.dot(out[i], th) - spring) < 1e-12


def test_fire_on_quadratic(oracle_mod):
    """FIRE reaches the minimum of an anisotropic quadratic bowl."""
    K = np.diag([1.0, 10.0, 50.0])
    x = np.array([1.0, -0.5, 0.2])
    fire = oracle_mod.Fire(dt=0.02, maxstep=0.1, row_dim=3)
    for _ in range(3000):
        f = -K @ x
        if np.linalg.norm(f) < 1e-10:
            break
        x = x + fire.step(f)
    assert np.linalg.norm(x) < 1e-10


def test_fire_resets_on_uphill(oracle_mod):
    fire = oracle_mod.Fire(dt=0.1, maxstep=10.0, row_dim=1)
    f = np.array([1.0])
    fire.step(f)                  # fresh: no power check
    assert fire.dt == 0.1 and fire.n_pos == 0
    fire.step(f)                  # P > 0
    assert fire.n_pos == 1
    fire.step(-f)                 # P < 0: velocity zeroed, dt halved
    assert fire.n_pos == 0 and fire.dt == pytest.approx(0.05) and fire.alpha == 0.1
    np.testing.assert_allclose(fire.v, 0.05 * -f)


def test_fire_row_clamp(oracle_mod):
    fire = oracle_mod.Fire(dt=1.0, maxstep=0.2, row_dim=3)
    dx = fire.step(np.array([3.0, 4.0, 0.0, 0.01, 0.0, 0.0]))
    np.testing.assert_allclose(dx[:3], [0.12, 0.16, 0.0])
    np.testing.assert_allclose(dx[3:], [0.01, 0.0, 0.0])


def _mb_minima():
    from oracle import muller_brown as mb
    A = minimize(mb.energy, [-0.558, 1.442], jac=mb.gradient, tol=1e-14).x
    B = minimize(mb.energy, [0.623, 0.028], jac=mb.gradient, tol=1e-14).x
    return A, B


def test_muller_brown_climbing_image_finds_saddle(oracle_mod):
    from oracle import muller_brown as mb
    with open(os.path.join(GOLDEN, "muller_brown.json")) as f:
        g = json.load(f)
    A, B = _mb_minima()
    for m, ref in zip((A, B), g["minima"][:2]):
        assert np.max(np.abs(m - ref[:2])) < 1e-3
    # independent Newton solve of grad V = 0 from the published saddle
    sol = root(mb.gradient, g["saddles"][0][:2], tol=1e-14)
    saddle = sol.x
    assert np.max(np.abs(saddle - g["saddles"][0][:2])) < 1e-3
    X = oracle_mod.interpolate(A, B, 9)
    band = oracle_mod.Band(X, mb.image, k=1.0, climb=True,
                           fire=oracle_mod.Fire(dt=0.002, maxstep=0.02, row_dim=2), row_dim=2)
    steps, conv = band.relax(1e-6, 20000)
    assert conv
    assert np.max(np.abs(band.X[band.ci] - saddle)) < 1e-6
    assert abs(band.E[band.ci] - g["saddles"][0][2]) < 5e-3
    # the path passes the intermediate minimum region: some image below the
    # second saddle energy between the two saddles
    assert min(band.E[1:-1]) < g["saddles"][1][2]


def test_lj_vacancy_hop_symmetric_and_saddle(oracle_mod):
    cfg = ci.lj_vacancy_31()
    R0, h0, R1, h1 = cfg["endpoints"]
    band = oracle_mod.make_band(oracle_mod.LJ(), R0, h0, R1, h1, 7, k=1.0, climb=True,
                                cell_filter=False, fire=oracle_mod.Fire(dt=0.01))
    steps, conv = band.relax(1e-4, 20000)
    assert conv
    E = np.array(band.E)
    assert E[0] == pytest.approx(E[-1], abs=1e-12)
    np.testing.assert_allclose(E, E[::-1], atol=1e-6)
    assert band.ci == 3
    hop = int(np.argmax(np.linalg.norm(R1 - R0, axis=1)))
    np.testing.assert_allclose(band.info[3]["R"][hop], 0.5 * (R0[hop] + R1[hop]), atol=1e-5)
    # saddle energy: minimise all other atoms with the hopping atom held at
    # the midpoint (scipy L-BFGS on the oracle energy)
    pot = oracle_mod.LJ()
    Rm = R0.copy()
    Rm[hop] = 0.5 * (R0[hop] + R1[hop])
    others = [i for i in range(len(R0)) if i != hop]

    def f(x):
        R = Rm.copy()
        R[others] = x.reshape(-1, 3)
        e, F, _ = pot.evaluate(R, h0)
        return np.sum(e), -F[others].ravel()

    res = minimize(f, Rm[others].ravel(), jac=True, method="L-BFGS-B",
                   options=dict(gtol=1e-11, ftol=1e-15, maxiter=5000))
    e0 = np.sum(pot.evaluate(R0, h0)[0])
    assert abs((res.fun - e0) - band.barrier()) < 1e-6


def test_tersoff_vacancy_hop_symmetric_and_saddle(oracle_mod):
    """Tersoff carbon diamond vacancy hop between relaxed endpoints (511
    atoms, fixed cell, 5 images, k = 0.1 eV/A^2, FIRE dt 0.05 / dt_max 0.2 /
    maxstep 0.1): the converged profile is symmetric, the climbing image is
    the centre image with the hopping atom at the midpoint of its two sites,
    and the barrier equals the constrained minimum of the energy with the
    hopping atom held at that midpoint (scipy L-BFGS from the symmetric
    midpoint configuration, on the oracle energy): the split-vacancy saddle."""
    R0, h0, R1, h1 = ci.diamond_vacancy_hop_relaxed((4, 4, 4))
    pot = oracle_mod.Tersoff()
    band = oracle_mod.make_band(pot, R0, h0, R1, h1, 5, k=0.1, climb=True, cell_filter=False,
                                fire=oracle_mod.Fire(dt=0.05, dt_max=0.2, maxstep=0.1))
    steps, conv = band.relax(1e-3, 20000)
    assert conv
    E = np.array(band.E)
    np.testing.assert_allclose(E, E[::-1], atol=1e-6)
    assert band.ci == 2
    hop = int(np.argmax(np.linalg.norm(R1 - R0, axis=1)))
    mid = 0.5 * (R0[hop] + R1[hop])
    np.testing.assert_allclose(band.info[2]["R"][hop], mid, atol=1e-5)
    base = 0.5 * (R0 + R1)
    others = [i for i in range(len(R0)) if i != hop]

    def f(x):
        R = base.copy()
        R[others] = x.reshape(-1, 3)
        e, F, _ = pot.evaluate(R, h0)
        return np.sum(e), -F[others].ravel()

    res = minimize(f, base[others].ravel(), jac=True, method="L-BFGS-B",
                   options=dict(gtol=1e-9, ftol=1e-15, maxiter=5000))
    e0 = np.sum(pot.evaluate(R0, h0)[0])
    assert abs((res.fun - e0) - band.barrier()) < 1e-6
    assert 5.0 < band.barrier() < 15.0


def _rot(a, b):
    Rz = np.array([[math.cos(a), -math.sin(a), 0], [math.sin(a), math.cos(a), 0], [0, 0, 1]])
    Rx = np.array([[1, 0, 0], [0, math.cos(b), -math.sin(b)], [0, math.sin(b), math.cos(b)]])
    return Rz @ Rx


def test_path_invariant_under_rotation(oracle_mod):
    """Rotating both end cells by Q leaves the CFNEB trajectory unchanged.

    With the reference cell rotated too, h0 -> h0 Q, the generalised
    coordinates transform as R~ -> R~ Q and B -> Q^T B Q; every dot product
    the band uses is invariant, so energies agree step by step and the images
    agree after undoing the rotation (checked after 300 FIRE steps)."""
    R0, h0, R1, h1 = ci.lj_vacancy_hop()
    h1 = ci.strained_cell(h1, 11, 0.02)
    R1 = ci.affine(R1, h0, h1)
    Q = _rot(0.8, -0.4)
    res = []
    for (a0, g0, a1, g1) in [(R0, h0, R1, h1), (R0 @ Q, h0 @ Q, R1 @ Q, h1 @ Q)]:
        band = oracle_mod.make_band(oracle_mod.LJ(), a0, g0, a1, g1, 5, k=1.0, climb=True,
                                    cell_filter=True, fire=oracle_mod.Fire(dt=0.01))
        band.step(300)
        band.compute()
        res.append((np.array(band.E), band, band.fmax))
    (E1, b1, f1), (E2, b2, f2) = res
    np.testing.assert_allclose(E2, E1, rtol=1e-9)
    for x1, x2 in zip(b1.X, b2.X):
        n = x1.shape[0] - 3
        np.testing.assert_allclose(x2[:n] @ Q.T, x1[:n], atol=1e-8)
        np.testing.assert_allclose(Q @ x2[n:] @ Q.T, x1[n:], atol=1e-8)


def test_insert_delete_keep_endpoints(oracle_mod):
    R0, h0, R1, h1 = ci.lj_vacancy_hop()
    band = oracle_mod.make_band(oracle_mod.LJ(), R0, h0, R1, h1, 5, k=1.0, climb=True,
                                cell_filter=False, fire=oracle_mod.Fire(dt=0.01))
    band.step(3)
    X0, XN, E0, EN = band.X[0].copy(), band.X[-1].copy(), band.E[0], band.E[-1]
    mid = 0.5 * (band.X[1] + band.X[2])
    band.insert_image(1)
    assert band.N == 6
    np.testing.assert_array_equal(band.X[2], mid)
    band.delete_image(4)
    assert band.N == 5
    with pytest.raises(IndexError):
        band.delete_image(0)
    with pytest.raises(IndexError):
        band.delete_image(band.N - 1)
    band.step(2)
    np.testing.assert_array_equal(band.X[0], X0)
    np.testing.assert_array_equal(band.X[-1], XN)
    assert band.E[0] == E0 and band.E[-1] == EN


def test_refine_rules(oracle_mod):
    """Spacing-driven insertion and deletion on a 1-D chain."""
    def flat(X):
        return 0.0, np.zeros_like(X), {}
    pts = [np.array([x]) for x in (0.0, 0.1, 0.2, 1.0, 1.1)]
    band = oracle_mod.Band(pts, flat, climb=False, row_dim=1, n_max=8)
    assert band.refine() == "insert"          # longest segment 0.8 > 1.5 * 0.275
    np.testing.assert_allclose([x[0] for x in band.X], [0, .1, .2, .6, 1.0, 1.1])
    pts = [np.array([x]) for x in (0.0, 1.0, 2.0, 2.01, 2.02, 3.0, 4.0)]
    band = oracle_mod.Band(pts, flat, climb=False, row_dim=1, n_min=3)
    assert band.refine() == "delete"          # 1 <= 1.5 * 0.67; 0.02 < 0.5 * 0.67
    np.testing.assert_allclose([x[0] for x in band.X], [0, 1, 2, 2.02, 3, 4])
    band = oracle_mod.Band(pts, flat, climb=False, row_dim=1, n_min=7)
    assert band.refine() is None              # already at the lower bound
    pts = [np.array([x]) for x in (0.0, 0.2, 0.4, 0.6)]
    band = oracle_mod.Band(pts, flat, climb=False, row_dim=1)
    assert band.refine() is None


def test_adaptive_band_runs_and_keeps_bounds(oracle_mod):
    A, B = _mb_minima()
    from oracle import muller_brown as mb
    X = [A + t * (B - A) for t in (0.0, 0.1, 0.2, 0.3)] + [B]   # one long segment
    band = oracle_mod.Band(X, mb.image, k=1.0, climb=True, row_dim=2, adaptive=True,
                           n_min=4, n_max=9, k_ref=10, cooldown=20,
                           fire=oracle_mod.Fire(dt=0.002, maxstep=0.02, row_dim=2))
    band.relax(1e-4, 4000)
    assert 4 <= band.N <= 9
    assert band.events and band.events[0][:2] == ("insert", 20)
    assert all(e[1] % 10 == 0 for e in band.events)
    gaps = np.diff([ev[1] for ev in band.events])
    assert np.all(gaps >= 20)
    np.testing.assert_array_equal(band.X[0], A)
    np.testing.assert_array_equal(band.X[-1], B)
