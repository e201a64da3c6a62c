"""Pins of the oracle's cell filter (paper Sec. II.C).

The generalised force must be minus the gradient of E with respect to the
generalised coordinates X = (R~, c B) (or (R~, c D)); the rotation-free
coordinate B must not change under a rigid rotation of the lattice; the
filter off reduces to plain fixed-cell forces.
"""
import math

import numpy as np
import pytest

import cfneb_inputs as ci


def _lj_case(seed=0):
    R0, h0, R1, h1 = ci.lj_vacancy_hop()
    h1 = ci.strained_cell(h1, seed, 0.03)
    R1 = ci.affine(R1, h0, h1)
    rng = np.random.default_rng(seed)
    return R0, h0, R1 + rng.normal(0, 0.03, R1.shape), h1


def _tersoff_case(seed=1):
    Rg, hg, Rd, hd = ci.tersoff_endpoint_cells()
    h = 0.5 * (hg + hd)
    h[0, 1] = 0.05
    s = 0.5 * (Rg @ np.linalg.inv(hg) + Rd @ np.linalg.inv(hd))
    rng = np.random.default_rng(seed)
    return Rg, hg, s @ h + rng.normal(0, 0.03, Rg.shape), h


def _fd_generalized(img, X, delta):
    G = np.zeros_like(X)
    for i in range(X.shape[0]):
        for c in range(3):
            Xp = X.copy(); Xp[i, c] += delta
            Xm = X.copy(); Xm[i, c] -= delta
            G[i, c] = -(img(Xp)[0] - img(Xm)[0]) / (2 * delta)
    return G


@pytest.mark.parametrize("case", ["lj", "tersoff"])
@pytest.mark.parametrize("variant", [0, 1])
@pytest.mark.parametrize("pressure", [0.0, 0.3])
def test_generalized_force_is_minus_gradient(oracle_mod, case, variant, pressure):
    if case == "lj":
        R0, h0, R, h = _lj_case()
        pot = oracle_mod.LJ()
    else:
        R0, h0, R, h = _tersoff_case()
        pot = oracle_mod.Tersoff()
    n = len(R)
    c = float(n)
    img = oracle_mod.AtomicImage(pot, h0, c, True, variant, pressure)
    X = oracle_mod.to_generalized(R, h, h0, c, variant)
    E, Fg, _ = img(X)
    G = _fd_generalized(img, X, 1e-6)
    scale = max(1.0, np.max(np.abs(Fg)))
    assert np.max(np.abs(Fg[:n] - G[:n])) < 2e-6 * scale
    assert np.max(np.abs(Fg[n:] - G[n:])) < 2e-6 * scale


def test_paper_factor_is_twice_the_gradient(oracle_mod):
    """Without the 1/2 the lattice force is exactly twice -dE/dX_lat."""
    R0, h0, R, h = _lj_case(3)
    pot = oracle_mod.LJ()
    n = len(R)
    img = oracle_mod.AtomicImage(pot, h0, n, True, 0, 0.0, paper_factor=True)
    X = oracle_mod.to_generalized(R, h, h0, n)
    _, Fg, _ = img(X)
    G = _fd_generalized(img, X, 1e-6)
    np.testing.assert_allclose(Fg[n:], 2.0 * G[n:], rtol=1e-5, atol=1e-8)


def _rotation(a, b, c):
    Rz = np.array([[math.cos(a), -math.sin(a), 0], [math.sin(a), math.cos(a), 0], [0, 0, 1]])
    Rx = np.array([[1, 0, 0], [0, math.cos(b), -math.sin(b)], [0, math.sin(b), math.cos(b)]])
    Ry = np.array([[math.cos(c), 0, math.sin(c)], [0, 1, 0], [-math.sin(c), 0, math.cos(c)]])
    return Rz @ Rx @ Ry


def test_B_invariant_under_rotation(oracle_mod):
    """B = D D^T does not change when the cell is rotated, h -> h Q."""
    R0, h0, R, h = _lj_case(4)
    Q = _rotation(0.4, -0.9, 1.3)
    n = len(R)
    X = oracle_mod.to_generalized(R, h, h0, n)
    Xq = oracle_mod.to_generalized(R @ Q, h @ Q, h0, n)
    np.testing.assert_allclose(Xq, X, atol=1e-12)
    # the deformation-gradient variant does see the rotation
    Xd = oracle_mod.to_generalized(R, h, h0, n, 1)
    Xdq = oracle_mod.to_generalized(R @ Q, h @ Q, h0, n, 1)
    assert np.max(np.abs(Xdq[n:] - Xd[n:])) > 0.1


def test_map_back_round_trip(oracle_mod):
    """from_generalized(to_generalized(R, h)) is R, h up to a rigid rotation:
    same fractional coordinates and the same metric h h^T."""
    R0, h0, R, h = _tersoff_case(5)
    Q = _rotation(0.2, 0.5, -0.3)
    h = h @ Q
    R = R @ Q
    n = len(R)
    X = oracle_mod.to_generalized(R, h, h0, n)
    R2, h2, D = oracle_mod.from_generalized(X, h0, n)
    np.testing.assert_allclose(R2 @ np.linalg.inv(h2), R @ np.linalg.inv(h), atol=1e-12)
    np.testing.assert_allclose(h2 @ h2.T, h @ h.T, atol=1e-12)
    np.testing.assert_allclose(D, D.T, atol=1e-14)
    assert np.all(np.linalg.eigvalsh(D) > 0)
    # energies agree: the filter only removes a rotation
    pot = oracle_mod.Tersoff()
    assert abs(np.sum(pot.evaluate(R2, h2)[0]) - np.sum(pot.evaluate(R, h)[0])) < 1e-10


def test_sym_sqrt_rejects_non_spd(oracle_mod):
    with pytest.raises(oracle_mod.NotSPD):
        oracle_mod.sym_sqrt(np.diag([1.0, -0.1, 2.0]))
    B = np.array([[2.0, 0.3, 0.1], [0.3, 1.5, -0.2], [0.1, -0.2, 1.1]])
    S = oracle_mod.sym_sqrt(B)
    np.testing.assert_allclose(S @ S, B, atol=1e-14)


def test_filter_off_is_plain_forces(oracle_mod):
    R0, h0, _, _ = _lj_case(6)
    rng = np.random.default_rng(6)
    R = R0 + rng.normal(0, 0.05, R0.shape)
    n = len(R)
    pot = oracle_mod.LJ()
    img = oracle_mod.AtomicImage(pot, h0, n, cell_filter=False)
    X = oracle_mod.to_generalized(R, h0, h0, n)
    E, Fg, info = img(X)
    _, F, _ = pot.evaluate(R, h0)
    np.testing.assert_allclose(X[:n], R, atol=1e-13)
    np.testing.assert_allclose(Fg[:n], F, atol=1e-12)
    assert np.all(Fg[n:] == 0.0)
