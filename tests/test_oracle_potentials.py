"""Pins of the oracle's potentials (energy, force, virial; paper Sec. II.B).

Each check uses something other than the oracle itself: central finite
differences of the energy, strain derivatives, FCC coordination shells, the
published LJ lattice sums and Tersoff's fitted diamond/graphite values,
extensivity under tiling, and rotation covariance.
"""
import itertools
import json
import math
import os

import numpy as np
import pytest

import cfneb_inputs as ci

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _load(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


def _energy(pot, R, h):
    e, _, _ = pot.evaluate(R, h)
    return float(np.sum(e))


def _perturbed(R, h, seed, amp, shear=0.0):
    rng = np.random.default_rng(seed)
    R = R + rng.normal(0.0, amp, R.shape)
    if shear:
        e = np.eye(3)
        e[0, 1] += shear
        e[2, 0] -= 0.5 * shear
        s = R @ np.linalg.inv(h)
        h = h @ e
        R = s @ h
    return R, h


def _fd_forces(pot, R, h, delta=1e-5):
    F = np.zeros_like(R)
    for i in range(R.shape[0]):
        for c in range(3):
            Rp = R.copy(); Rp[i, c] += delta
            Rm = R.copy(); Rm[i, c] -= delta
            F[i, c] = -(_energy(pot, Rp, h) - _energy(pot, Rm, h)) / (2 * delta)
    return F


def _fd_virial(pot, R, h, delta=1e-6):
    """V_mn = -dU/d eps_mn with h' = h (I + eps), R' = R (I + eps)."""
    V = np.zeros((3, 3))
    for m in range(3):
        for n in range(3):
            e = np.zeros((3, 3)); e[m, n] = delta
            Ep = _energy(pot, R @ (np.eye(3) + e), h @ (np.eye(3) + e))
            Em = _energy(pot, R @ (np.eye(3) - e), h @ (np.eye(3) - e))
            V[m, n] = -(Ep - Em) / (2 * delta)
    return V


# ---------------------------------------------------------------------------
# Lennard-Jones
# ---------------------------------------------------------------------------

def _fcc_shells(a, rc):
    """Distances and multiplicities of the FCC neighbour shells inside rc,
    from the lattice vectors (not a supercell sum)."""
    vecs = []
    m = int(math.ceil(rc / a)) + 1
    for i, j, k in itertools.product(range(-m, m + 1), repeat=3):
        for b in ci.FCC_BASIS:
            v = (np.array([i, j, k]) + b) * a
            r = np.linalg.norm(v)
            if 1e-9 < r < rc:
                vecs.append(r)
    r = np.array(vecs)
    key, inv, count = np.unique(np.round(r, 8), return_inverse=True, return_counts=True)
    dist = np.array([r[inv == k][0] for k in range(len(key))])
    return dist, count


@pytest.mark.parametrize("reps", [(2, 2, 2), (3, 3, 3), (2, 3, 4)])
@pytest.mark.parametrize("shift", [False, True])
def test_lj_fcc_matches_shell_sum(oracle_mod, reps, shift):
    a, rc = ci.LJ_A, 2.5
    R, h = ci.fcc(a, *reps)
    pot = oracle_mod.LJ(rc=rc, shift=shift)
    e, F, V = pot.evaluate(R, h)
    dist, count = _fcc_shells(a, rc)
    assert count.sum() == 78  # 12 + 6 + 24 + 12 + 24 within 2.5 sigma
    phi = lambda r: 4 * (r ** -12 - r ** -6)
    dphi = lambda r: 4 * (-12 * r ** -13 + 6 * r ** -7)
    e_shell = 0.5 * np.sum(count * (phi(dist) - (phi(rc) if shift else 0.0)))
    np.testing.assert_allclose(e, e_shell, rtol=1e-12, atol=1e-12)
    assert np.max(np.abs(F)) < 1e-10
    v_shell = -0.5 * len(R) * np.sum(count * dphi(dist) * dist) / 3.0
    np.testing.assert_allclose(V, v_shell * np.eye(3), atol=1e-9)


def test_lj_published_lattice_sums(oracle_mod):
    """Long-cutoff FCC energy approaches 2 eps [A12 (s/r0)^12 - A6 (s/r0)^6]."""
    g = _load("lj_fcc_lattice_sums.json")
    r0 = (2 * g["A12"] / g["A6"]) ** (1 / 6)
    a = r0 * math.sqrt(2)
    R, h = ci.fcc(a, 2, 2, 2)
    rc = 12.0
    e, _, _ = oracle_mod.LJ(rc=rc, shift=False).evaluate(R, h)
    textbook = 2 * (g["A12"] * r0 ** -12 - g["A6"] * r0 ** -6)
    # r^-6 tail beyond rc: 1/2 * int 4 pi r^2 rho (-4 r^-6) dr
    rho = 4 / a ** 3
    tail = -8 * math.pi * rho / (3 * rc ** 3)
    assert abs(np.mean(e) - (textbook - tail)) < 2e-4
    assert abs(textbook - (-8.6102)) < 1e-3


@pytest.mark.parametrize("case", ["vacancy31", "triclinic", "tiny"])
def test_lj_forces_finite_difference(oracle_mod, case):
    pot = oracle_mod.LJ(rc=2.5, shift=True)
    if case == "vacancy31":
        R, h, _, _ = ci.lj_vacancy_hop()
        R, h = _perturbed(R, h, 1, 0.03)
    elif case == "triclinic":
        R, h = ci.fcc(ci.LJ_A, 2, 2, 3)
        R, h = _perturbed(R, h, 2, 0.05, shear=0.07)
    else:  # one conventional cell: rc exceeds the whole cell width
        R, h = ci.fcc(ci.LJ_A, 1, 1, 1)
        R, h = _perturbed(R, h, 3, 0.04, shear=0.05)
    _, F, _ = pot.evaluate(R, h)
    Ffd = _fd_forces(pot, R, h)
    assert np.max(np.abs(F - Ffd)) <= 1e-6 * max(1.0, np.max(np.abs(F)))


@pytest.mark.parametrize("case", ["vacancy31", "tiny"])
def test_lj_virial_strain_derivative(oracle_mod, case):
    pot = oracle_mod.LJ(rc=2.5, shift=True)
    if case == "vacancy31":
        R, h, _, _ = ci.lj_vacancy_hop()
        R, h = _perturbed(R, h, 4, 0.03, shear=0.04)
    else:
        R, h = ci.fcc(ci.LJ_A, 1, 1, 1)
        R, h = _perturbed(R, h, 5, 0.04, shear=0.05)
    _, _, V = pot.evaluate(R, h)
    Vfd = _fd_virial(pot, R, h)
    assert np.max(np.abs(V - Vfd)) <= 1e-6 * max(1.0, np.max(np.abs(V)))


def test_lj_pair_closed_form(oracle_mod):
    """Two atoms in a box much larger than rc: E = phi(r) - phi(rc)."""
    h = np.eye(3) * 20.0
    R = np.array([[1.0, 1.0, 1.0], [2.3, 1.4, 0.9]])
    r = np.linalg.norm(R[1] - R[0])
    e, F, V = oracle_mod.LJ(rc=2.5, shift=True).evaluate(R, h)
    phi = lambda x: 4 * (x ** -12 - x ** -6)
    assert abs(np.sum(e) - (phi(r) - phi(2.5))) < 1e-14
    dphi = 4 * (-12 * r ** -13 + 6 * r ** -7)
    rij = R[1] - R[0]
    np.testing.assert_allclose(F[0], dphi * rij / r, rtol=1e-13)
    np.testing.assert_allclose(F[1], -dphi * rij / r, rtol=1e-13)
    np.testing.assert_allclose(V, -dphi * np.outer(rij, rij) / r, rtol=1e-12)


# ---------------------------------------------------------------------------
# Tersoff
# ---------------------------------------------------------------------------

def _tersoff_terms(r, p):
    """Tersoff's published pieces, used for closed-form cluster energies."""
    if r < p["R"] - p["D"]:
        fc = 1.0
    elif r > p["R"] + p["D"]:
        fc = 0.0
    else:
        fc = 0.5 - 0.5 * math.sin(math.pi / 2 * (r - p["R"]) / p["D"])
    return fc, p["A"] * math.exp(-p["lambda1"] * r), -p["B"] * math.exp(-p["lambda2"] * r)


@pytest.mark.parametrize("r", [1.4, 1.9, 2.05])
def test_tersoff_dimer_closed_form(oracle_mod, r):
    """Isolated dimer: zeta = 0, b = 1, E = f_C (f_R + f_A)."""
    pot = oracle_mod.Tersoff()
    h = np.eye(3) * 30.0
    R = np.array([[5.0, 5.0, 5.0], [5.0 + r, 5.0, 5.0]])
    fc, fr, fa = _tersoff_terms(r, pot.params)
    assert abs(_energy(pot, R, h) - fc * (fr + fa)) < 1e-12


def test_tersoff_triangle_closed_form(oracle_mod):
    """Equilateral triangle of side r: zeta_ij = f_C(r) g(60 deg) for every bond."""
    pot = oracle_mod.Tersoff()
    p = pot.params
    r = 1.45
    h = np.eye(3) * 30.0
    R = np.array([[5, 5, 5], [5 + r, 5, 5], [5 + r / 2, 5 + r * math.sqrt(3) / 2, 5]], float)
    fc, fr, fa = _tersoff_terms(r, p)
    cs = 0.5
    g = 1 + p["c"] ** 2 / p["d"] ** 2 - p["c"] ** 2 / (p["d"] ** 2 + (p["h"] - cs) ** 2)
    zeta = fc * g
    b = (1 + (p["beta"] * zeta) ** p["n"]) ** (-1 / (2 * p["n"]))
    expected = 3 * fc * (fr + b * fa)  # 6 directed bonds, 1/2 each
    assert abs(_energy(pot, R, h) - expected) < 1e-11


def _cubic_diamond(a):
    basis = np.array([[0, 0, 0], [0, .5, .5], [.5, 0, .5], [.5, .5, 0],
                      [.25, .25, .25], [.25, .75, .75], [.75, .25, .75], [.75, .75, .25]])
    return basis * a, np.eye(3) * a


def test_tersoff_diamond_published(oracle_mod):
    """Equilibrium lattice constant and cohesive energy of diamond agree with
    Tersoff's fitted values; the virial vanishes at the minimum."""
    from scipy.optimize import minimize_scalar
    g = _load("tersoff_1988_carbon.json")
    pot = oracle_mod.Tersoff()
    f = lambda a: _energy(pot, *_cubic_diamond(a)) / 8.0
    res = minimize_scalar(f, bracket=(3.5, 3.56, 3.62), tol=1e-12)
    assert abs(res.x - g["diamond_lattice_constant_A"]) < g["tolerance_lattice_A"]
    assert abs(res.fun - g["diamond_cohesive_energy_eV"]) < g["tolerance_energy_eV"]
    _, F, V = pot.evaluate(*_cubic_diamond(res.x))
    assert np.max(np.abs(F)) < 1e-10
    assert np.max(np.abs(V)) < 1e-5


def test_tersoff_graphene_bond(oracle_mod):
    from scipy.optimize import minimize_scalar
    g = _load("tersoff_1988_carbon.json")
    pot = oracle_mod.Tersoff()
    s_g, h_g, _, _ = ci.graphite_hexdiamond_cells()

    def f(bond):
        h = h_g.copy()
        h[0, 0] = bond * math.sqrt(3)
        h[1, 1] = 3 * bond
        return _energy(pot, s_g @ h, h) / 8.0

    res = minimize_scalar(f, bracket=(1.40, 1.45, 1.50), tol=1e-12)
    assert abs(res.x - g["graphite_bond_length_A"]) < g["tolerance_bond_A"]


def _carbon_cases():
    Rg, hg, Rd, hd = ci.tersoff_endpoint_cells()
    out = {"graphite8": (Rg, hg), "hexdiamond8": (Rd, hd)}
    s_g, h_g, s_d, h_d = ci.graphite_hexdiamond_cells()
    # a compressed, mid-path structure where interlayer bonds are forming
    hm = 0.5 * (hg + hd)
    hm[2, 2] = 0.5 * (hg[2, 2] + hd[2, 2]) * 0.72
    sm = 0.5 * (Rg @ np.linalg.inv(hg) + Rd @ np.linalg.inv(hd))
    out["midpath8"] = (sm @ hm, hm)
    R2, h2 = ci.tile(Rd, hd, (2, 1, 1))
    out["hexdiamond16"] = (R2, h2)
    return out


@pytest.mark.parametrize("name", ["graphite8", "hexdiamond8", "midpath8", "hexdiamond16"])
def test_tersoff_forces_finite_difference(oracle_mod, name):
    R, h = _carbon_cases()[name]
    R, h = _perturbed(R, h, 7, 0.05, shear=0.03)
    pot = oracle_mod.Tersoff()
    _, F, _ = pot.evaluate(R, h)
    Ffd = _fd_forces(pot, R, h)
    assert np.max(np.abs(F - Ffd)) <= 2e-6 * max(1.0, np.max(np.abs(F)))


@pytest.mark.parametrize("name", ["graphite8", "midpath8", "hexdiamond16"])
def test_tersoff_virial_strain_derivative(oracle_mod, name):
    R, h = _carbon_cases()[name]
    R, h = _perturbed(R, h, 8, 0.05, shear=0.03)
    pot = oracle_mod.Tersoff()
    _, _, V = pot.evaluate(R, h)
    Vfd = _fd_virial(pot, R, h)
    assert np.max(np.abs(V - Vfd)) <= 2e-6 * max(1.0, np.max(np.abs(V)))


def test_extensive_under_tiling(oracle_mod):
    """A periodic structure and its 2x2x2 tiling: same energy per atom, same
    forces, virial x 8 (checks the periodic-image enumeration when rc exceeds
    half the cell width)."""
    for pot, (R, h) in [(oracle_mod.Tersoff(), _carbon_cases()["midpath8"]),
                        (oracle_mod.LJ(), ci.fcc(ci.LJ_A, 1, 1, 1))]:
        R, h = _perturbed(R, h, 9, 0.03, shear=0.02)
        e1, F1, V1 = pot.evaluate(R, h)
        R8, h8 = ci.tile(R, h, (2, 2, 2))
        e8, F8, V8 = pot.evaluate(R8, h8)
        np.testing.assert_allclose(np.sum(e8), 8 * np.sum(e1), rtol=1e-12)
        np.testing.assert_allclose(F8, np.tile(F1, (8, 1)), atol=1e-10)
        np.testing.assert_allclose(V8, 8 * V1, rtol=1e-10, atol=1e-10)


def test_rotation_covariance(oracle_mod):
    """R -> R Q, h -> h Q: E unchanged, F -> F Q, V -> Q^T V Q."""
    th = 0.7
    Q = np.array([[math.cos(th), -math.sin(th), 0], [math.sin(th), math.cos(th), 0], [0, 0, 1]])
    Q = Q @ np.array([[1, 0, 0], [0, math.cos(0.3), math.sin(0.3)], [0, -math.sin(0.3), math.cos(0.3)]])
    for pot, (R, h) in [(oracle_mod.Tersoff(), _carbon_cases()["midpath8"]),
                        (oracle_mod.LJ(), ci.fcc(ci.LJ_A, 2, 2, 2))]:
        R, h = _perturbed(R, h, 10, 0.04, shear=0.02)
        e, F, V = pot.evaluate(R, h)
        e2, F2, V2 = pot.evaluate(R @ Q, h @ Q)
        assert abs(np.sum(e) - np.sum(e2)) < 1e-10 * abs(np.sum(e))
        np.testing.assert_allclose(F2, F @ Q, atol=1e-9)
        np.testing.assert_allclose(V2, Q.T @ V @ Q, atol=1e-9)


def test_sampled_forces_match_full(oracle_mod):
    R, h = ci.tile(*ci.tersoff_endpoint_cells()[2:], (2, 2, 2))
    R, h = _perturbed(R, h, 11, 0.05, shear=0.01)
    pot = oracle_mod.Tersoff()
    _, F, _ = pot.evaluate(R, h)
    idx = np.array([0, 5, 17, 63])
    np.testing.assert_allclose(pot.forces_sampled(R, h, idx), F[idx], atol=1e-12)
    lj = oracle_mod.LJ()
    R, h = ci.fcc(ci.LJ_A, 2, 2, 2)
    R, h = _perturbed(R, h, 12, 0.03)
    _, F, _ = lj.evaluate(R, h)
    np.testing.assert_allclose(lj.forces_sampled(R, h, idx[:3]), F[idx[:3]], atol=1e-12)
