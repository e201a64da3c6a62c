"""Pins of the oracle's NEP-style potential (descriptors + neural network
site energy with synthetic weights).

Each check uses something other than the oracle's own formulas: central
finite differences of the energy (forces, strain derivative), invariance
under rotation and atom relabelling, extensivity under tiling (periodic
images), numpy's Chebyshev series for the radial basis, scipy's spherical
harmonics for the angular descriptors (the Legendre double sum equals
4 pi / (2l + 1) sum_m |sum_j g_j Y_lm(r^_j)|^2), and continuity at the
cutoff.
"""
import math

import numpy as np
import pytest

import cfneb_inputs as ci

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def nep():
    from oracle import nep as m
    return m


def _pot(nep, seed=3, rc=2.1):
    return nep.NEP(ci.nep_weights(seed), rc=rc)


def _energy(pot, R, h):
    e, _, _ = pot.evaluate(R, h)
    return float(np.sum(e))


def _cases():
    Rg, hg, Rd, hd = ci.tersoff_endpoint_cells()
    hm = 0.5 * (hg + hd)
    hm[2, 2] = 0.5 * (hg[2, 2] + hd[2, 2]) * 0.72
    sm = 0.5 * (Rg @ np.linalg.inv(hg) + Rd @ np.linalg.inv(hd))
    out = {"graphite8": (Rg, hg), "midpath8": (sm @ hm, hm)}
    rng = np.random.default_rng(6)
    return {k: (R + rng.normal(0.0, 0.05, R.shape), h) for k, (R, h) in out.items()}


@pytest.mark.parametrize("name", ["graphite8", "midpath8"])
def test_nep_forces_finite_difference(nep, name):
    R, h = _cases()[name]
    pot = _pot(nep)
    _, F, _ = pot.evaluate(R, h)
    d = 1e-5
    Ffd = np.zeros_like(R)
    for i in range(len(R)):
        for c in range(3):
            Rp = R.copy(); Rp[i, c] += d
            Rm = R.copy(); Rm[i, c] -= d
            Ffd[i, c] = -(_energy(pot, Rp, h) - _energy(pot, Rm, h)) / (2 * d)
    assert np.max(np.abs(F)) > 1e-2
    assert np.max(np.abs(F - Ffd)) <= 1e-6 * max(1.0, np.max(np.abs(F)))


def test_nep_virial_strain_derivative(nep):
    R, h = _cases()["midpath8"]
    pot = _pot(nep)
    _, _, V = pot.evaluate(R, h)
    d = 1e-6
    Vfd = np.zeros((3, 3))
    for m in range(3):
        for n in range(3):
            e = np.zeros((3, 3)); e[m, n] = d
            Ep = _energy(pot, R @ (np.eye(3) + e), h @ (np.eye(3) + e))
            Em = _energy(pot, R @ (np.eye(3) - e), h @ (np.eye(3) - e))
            Vfd[m, n] = -(Ep - Em) / (2 * d)
    assert np.max(np.abs(V - Vfd)) <= 1e-6 * max(1.0, np.max(np.abs(V)))


def test_nep_rotation_and_relabelling(nep):
    R, h = _cases()["midpath8"]
    pot = _pot(nep)
    e, F, V = pot.evaluate(R, h)
    th = 0.7
    Q = np.array([[math.cos(th), -math.sin(th), 0], [math.sin(th), math.cos(th), 0], [0, 0, 1]])
    Q = Q @ np.array([[1, 0, 0], [0, math.cos(0.3), math.sin(0.3)], [0, -math.sin(0.3), math.cos(0.3)]])
    e2, F2, V2 = pot.evaluate(R @ Q, h @ Q)
    np.testing.assert_allclose(e2, e, atol=1e-12)
    np.testing.assert_allclose(F2, F @ Q, atol=1e-11)
    np.testing.assert_allclose(V2, Q.T @ V @ Q, atol=1e-10)
    perm = np.random.default_rng(2).permutation(len(R))
    e3, F3, _ = pot.evaluate(R[perm], h)
    np.testing.assert_allclose(e3, e[perm], atol=1e-12)
    np.testing.assert_allclose(F3, F[perm], atol=1e-11)


def test_nep_extensive_under_tiling(nep):
    """rc exceeds half of the 8-atom cell's widths: images of the same atom
    are separate neighbours; a 2x2x2 tiling gives the same per-atom terms."""
    R, h = _cases()["midpath8"]
    pot = _pot(nep)
    e1, F1, V1 = pot.evaluate(R, h)
    R8, h8 = ci.tile(R, h, (2, 2, 2))
    e8, F8, V8 = pot.evaluate(R8, h8)
    np.testing.assert_allclose(np.sum(e8), 8 * np.sum(e1), rtol=1e-12)
    np.testing.assert_allclose(F8, np.tile(F1, (8, 1)), atol=1e-10)
    np.testing.assert_allclose(V8, 8 * V1, rtol=1e-10, atol=1e-10)


def test_nep_radial_basis_is_a_chebyshev_series(nep):
    x = np.linspace(-1.0, 1.0, 41)
    B = nep.chebyshev_basis(torch, torch.tensor(x)).numpy()
    np.testing.assert_allclose(B, np.polynomial.chebyshev.chebvander(x, nep.K - 1), atol=1e-13)


def test_nep_angular_descriptors_from_spherical_harmonics(nep):
    """q_nl of every atom against 4 pi / (2l + 1) sum_m |sum_j g_j Y_lm|^2
    with scipy's spherical harmonics and numpy's Chebyshev series."""
    from scipy.special import sph_harm_y
    R, h = _cases()["midpath8"]
    rc = 2.1
    pot = _pot(nep, rc=rc)
    q = pot.descriptors(R, h)
    I, J, d = nep.periodic_pairs(R, h, rc)
    r = np.linalg.norm(d, axis=1)
    x = 2.0 * (r / rc - 1.0) ** 2 - 1.0
    fk = 0.5 * (np.polynomial.chebyshev.chebvander(x, nep.K - 1) + 1.0) * \
        (0.5 * (1.0 + np.cos(np.pi * r / rc)))[:, None]
    gA = fk @ pot.w["cA"].T
    polar = np.arccos(np.clip(d[:, 2] / r, -1.0, 1.0))
    azim = np.arctan2(d[:, 1], d[:, 0])
    for i in range(len(R)):
        sel = I == i
        for n in range(nep.NA):
            for l in range(1, nep.L + 1):
                s = 0.0
                for m in range(-l, l + 1):
                    Y = sph_harm_y(l, m, polar[sel], azim[sel])
                    s += abs(np.sum(gA[sel, n] * Y)) ** 2
                ref = 4.0 * np.pi / (2 * l + 1) * s
                assert abs(q[i, nep.NR + n * nep.L + l - 1] - ref) <= 1e-10 * max(1.0, abs(ref))


def test_nep_continuous_at_the_cutoff(nep):
    """A dimer in a large box: as the distance reaches rc the energy tends to
    the isolated-atom value like (rc - r)^2 and the force to zero like
    (rc - r) (f_c and f_c' vanish there)."""
    rc = 2.1
    pot = _pot(nep, rc=rc)
    h = np.eye(3) * 20.0

    def dimer(r):
        return np.array([[5.0, 5.0, 5.0], [5.0 + r, 5.0, 5.0]])
    e_far = np.sum(pot.evaluate(dimer(2.5), h)[0])
    de, df = [], []
    for delta in (1e-3, 1e-4):
        e, F, _ = pot.evaluate(dimer(rc - delta), h)
        de.append((np.sum(e) - e_far) / delta ** 2)
        df.append(np.max(np.abs(F)) / delta)
    assert abs(de[0]) > 0 and abs(de[1] - de[0]) <= 0.01 * abs(de[0])
    assert df[0] > 0 and abs(df[1] - df[0]) <= 0.01 * df[0]
