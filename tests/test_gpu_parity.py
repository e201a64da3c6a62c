"""GPU parity: the CUDA library (through its C ABI) against the FP64 oracle.

Tolerances (stated per result):
  FP64 path   forces: max |dF| <= 1e-10 * max(1, max |F|) (the floor covers
              forces that vanish by symmetry); energies and virials 1e-10
              relative; band states after several FIRE steps 1e-9.
  mixed path  forces: max |dF| <= 1e-4 (eV/A for Tersoff, eps/sigma for LJ)
              at the same configuration, for configurations whose forces stay
              below 100 eV/A; beyond that (close contacts of unrelaxed or
              randomly displaced structures, |F| up to ~400 eV/A) the FP32
              arithmetic bound is relative, max |dF| <= 1e-6 max |F| (2e-6
              for LJ, whose forces sum ~78 neighbour terms); barriers within
              1 meV (1e-3 eps).
"""
import numpy as np
import pytest

import cfneb_inputs as ci
from _cases import (f32_structure, gpu_band, lj_band_case, lj_structures, oracle_band,
                    tersoff_structures)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def g():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2510_16721_gb300 as g
    g.build()
    return g


def _rel(a, b, floor=1.0):
    """max |a - b| relative to max(floor, max |b|)."""
    return np.max(np.abs(np.asarray(a) - np.asarray(b))) / max(floor, np.max(np.abs(b)))


# ---------------------------------------------------------------------------
# single-point energies, forces, virials
# ---------------------------------------------------------------------------

def _single_atom():
    # one atom in a cell narrower than rc: it only sees its own images
    h = np.array([[1.6, 0.1, 0.0], [0.0, 1.7, 0.2], [0.1, 0.0, 1.8]])
    return np.array([[0.3, 0.2, 0.1]]), h


@pytest.mark.parametrize("name", ["vacancy31", "one_cell", "triclinic240", "fcc2916", "single"])
def test_lj_single_point_fp64(g, oracle_mod, name):
    R, h = _single_atom() if name == "single" else lj_structures()[name]
    E, F, V = g.evaluate([(R, h)], g.lj_potential(), g.FP64)
    e, Fo, Vo = oracle_mod.LJ().evaluate(R, h)
    assert abs(E[0] - np.sum(e)) <= 1e-10 * abs(np.sum(e))
    assert _rel(F[0], Fo) <= 1e-10
    assert np.max(np.abs(V[0] - Vo)) <= 1e-10 * max(1.0, np.max(np.abs(Vo)))


@pytest.mark.parametrize("name", ["vacancy31", "one_cell", "triclinic240", "fcc2916"])
def test_lj_single_point_mixed(g, oracle_mod, name):
    """Randomly displaced structures (0.02-0.05 sigma) with pair forces up to
    ~100 eps/sigma: FP32 pair arithmetic over ~78 neighbours keeps the force
    error within 2e-6 of the largest force (1e-4 eps/sigma floor)."""
    R, h = f32_structure(*lj_structures()[name])
    E, F, V = g.evaluate([(R, h)], g.lj_potential(), g.MIXED)
    e, Fo, Vo = oracle_mod.LJ().evaluate(R, h)
    assert np.max(np.abs(F[0] - Fo)) <= max(1e-4, 2e-6 * np.max(np.abs(Fo)))
    # reported energies come from the FP64 energy pass on either precision
    assert abs(E[0] - np.sum(e)) <= 1e-10 * abs(np.sum(e))
    assert np.max(np.abs(V[0] - Vo)) <= 1e-4 * len(R)


@pytest.mark.parametrize("name", ["graphite8", "midpath8", "midpath576", "hexdiamond480"])
def test_tersoff_single_point_fp64(g, oracle_mod, name):
    R, h = tersoff_structures()[name]
    E, F, V = g.evaluate([(R, h)], g.tersoff_potential(), g.FP64)
    e, Fo, Vo = oracle_mod.Tersoff().evaluate(R, h)
    assert abs(E[0] - np.sum(e)) <= 1e-10 * abs(np.sum(e))
    assert _rel(F[0], Fo) <= 1e-10
    assert np.max(np.abs(V[0] - Vo)) <= 1e-10 * np.max(np.abs(Vo))


@pytest.mark.parametrize("name", ["graphite8", "midpath8", "midpath576", "hexdiamond480"])
def test_tersoff_single_point_mixed(g, oracle_mod, name):
    R, h = f32_structure(*tersoff_structures()[name])
    E, F, V = g.evaluate([(R, h)], g.tersoff_potential(), g.MIXED)
    e, Fo, Vo = oracle_mod.Tersoff().evaluate(R, h)
    assert np.max(np.abs(F[0] - Fo)) <= max(1e-4, 1e-6 * np.max(np.abs(Fo)))
    assert abs(E[0] - np.sum(e)) <= 1e-10 * abs(np.sum(e))
    assert np.max(np.abs(V[0] - Vo)) <= 1e-4 * len(R)


def test_several_structures_in_one_call(g, oracle_mod):
    s = lj_structures()
    items = [s["vacancy31"], s["one_cell"], s["triclinic240"]]
    E, F, V = g.evaluate(items, g.lj_potential(), g.FP64)
    for k, (R, h) in enumerate(items):
        e, Fo, _ = oracle_mod.LJ().evaluate(R, h)
        assert abs(E[k] - np.sum(e)) <= 1e-10 * abs(np.sum(e))
        assert _rel(F[k], Fo) <= 1e-10


# ---------------------------------------------------------------------------
# band steps: FP64 path against the oracle, step by step
# ---------------------------------------------------------------------------

def _compare_state(st, ob, tol):
    N = ob.N
    assert st["X"].shape[0] == N
    for i in range(N):
        assert _rel(st["X"][i], ob.X[i]) <= tol, ("X", i)
    for i in range(1, N - 1):
        assert _rel(st["F"][i], ob.F[i]) <= tol, ("F", i)
        assert _rel(st["Fneb"][i], ob.fneb[i - 1].reshape(st["Fneb"][i].shape)) <= tol, ("Fneb", i)


@pytest.mark.parametrize("nsteps", [1, 5, 40])
def test_lj_band_steps_fp64(g, oracle_mod, nsteps):
    R0, h0, R1, h1 = lj_band_case()
    gb = gpu_band(g, R0, h0, R1, h1, 7, g.lj_potential(), k=1.0, dt=0.01, cell_filter=False)
    ob = oracle_band(oracle_mod, oracle_mod.LJ(), R0, h0, R1, h1, 7, k=1.0, dt=0.01,
                     cell_filter=False)
    gb.step(nsteps)
    ob.step(nsteps)
    st = gb.get_state()
    _compare_state(st, ob, 1e-9)
    path = gb.get_path()
    # reported energies are those of the current (moved) images
    Eo = [ob.image_fn(x)[0] for x in ob.X]
    np.testing.assert_allclose(path["energies"], Eo, rtol=1e-10)
    assert st["ci"] == ob.ci
    assert st["steps"] == nsteps


@pytest.mark.parametrize("nsteps", [1, 8])
def test_lj_band_steps_cell_filter_fp64(g, oracle_mod, nsteps):
    R0, h0, R1, h1 = lj_band_case(strain_seed=3)
    gb = gpu_band(g, R0, h0, R1, h1, 5, g.lj_potential(), k=1.0, dt=0.01, cell_filter=True)
    ob = oracle_band(oracle_mod, oracle_mod.LJ(), R0, h0, R1, h1, 5, k=1.0, dt=0.01,
                     cell_filter=True)
    gb.step(nsteps)
    ob.step(nsteps)
    _compare_state(gb.get_state(), ob, 1e-9)
    path = gb.get_path()
    # the cell metric h h^T of every image (the rotation-free filter fixes h
    # only up to a rotation), after the oracle's last move
    for i in range(5):
        _, ho, _ = oracle_mod.from_generalized(ob.X[i], h0, ob.image_fn.c)
        np.testing.assert_allclose(path["cells"][i] @ path["cells"][i].T, ho @ ho.T,
                                   rtol=1e-9, atol=1e-12)


def test_lj_band_steps_cell_factor_j_fp64(g, oracle_mod):
    """Lattice scale J = Omega0^(1/3) n^(1/6) (CFNEB_CELL_FACTOR_J) against
    the oracle's c = "J": the band state after 8 steps at 1e-9."""
    R0, h0, R1, h1 = lj_band_case(strain_seed=3)
    gb = gpu_band(g, R0, h0, R1, h1, 5, g.lj_potential(), k=1.0, dt=0.01, cell_filter=True,
                  cell_factor=g.CELL_FACTOR_J)
    ob = oracle_band(oracle_mod, oracle_mod.LJ(), R0, h0, R1, h1, 5, k=1.0, dt=0.01,
                     cell_filter=True, c="J")
    assert ob.image_fn.c == pytest.approx(abs(np.linalg.det(h0)) ** (1 / 3) * len(R0) ** (1 / 6))
    gb.step(8)
    ob.step(8)
    _compare_state(gb.get_state(), ob, 1e-9)


@pytest.mark.parametrize("nsteps", [1, 6])
def test_tersoff_band_steps_fp64(g, oracle_mod, nsteps):
    cfg = ci.tersoff_graphite_hexdiamond()
    R0, h0, R1, h1 = cfg["endpoints"]
    gb = gpu_band(g, R0, h0, R1, h1, 9, g.tersoff_potential(), k=0.1, dt=0.1,
                  cell_filter=True, noise=cfg["noise"])
    ob = oracle_band(oracle_mod, oracle_mod.Tersoff(), R0, h0, R1, h1, 9, k=0.1, dt=0.1,
                     cell_filter=True, noise=cfg["noise"])
    gb.step(nsteps)
    ob.step(nsteps)
    st = gb.get_state()
    _compare_state(st, ob, 1e-9)
    for i in range(1, 8):
        assert _rel(st["virials"][i], ob.info[i]["V"]) <= 1e-10


def test_three_image_band(g, oracle_mod):
    """One moving image: it is the climbing image and feels no spring."""
    R0, h0, R1, h1 = lj_band_case()
    gb = gpu_band(g, R0, h0, R1, h1, 3, g.lj_potential(), k=1.0, dt=0.01, cell_filter=False)
    ob = oracle_band(oracle_mod, oracle_mod.LJ(), R0, h0, R1, h1, 3, k=1.0, dt=0.01,
                     cell_filter=False)
    gb.step(12)
    ob.step(12)
    _compare_state(gb.get_state(), ob, 1e-9)


def test_lj_vacancy_relax_matches_oracle(g, oracle_mod):
    R0, h0, R1, h1 = lj_band_case()
    gb = gpu_band(g, R0, h0, R1, h1, 7, g.lj_potential(), k=1.0, dt=0.01, cell_filter=False)
    done, conv = gb.relax(1e-4, 20000)
    assert conv
    ob = oracle_band(oracle_mod, oracle_mod.LJ(), R0, h0, R1, h1, 7, k=1.0, dt=0.01,
                     cell_filter=False)
    od, oconv = ob.relax(1e-4, 20000)
    assert oconv
    E = gb.get_path()["energies"]
    assert abs((E.max() - E[0]) - ob.barrier()) <= 1e-8
    np.testing.assert_allclose(E, E[::-1], atol=1e-6)
    # the mirror-symmetric hop relaxes in a step count that rounding-level
    # differences shift (which side breaks the symmetry first); the barrier
    # above is the parity result
    assert abs(done - od) <= max(5, 0.10 * od)


# ---------------------------------------------------------------------------
# mixed precision band
# ---------------------------------------------------------------------------

def test_tersoff_band_mixed_forces_at_same_configuration(g, oracle_mod):
    cfg = ci.tersoff_graphite_hexdiamond()
    R0, h0, R1, h1 = cfg["endpoints"]
    gb = gpu_band(g, R0, h0, R1, h1, 9, g.tersoff_potential(), k=0.1, dt=0.1,
                  cell_filter=True, noise=cfg["noise"], precision=g.MIXED)
    gb.step(20)
    st = gb.get_state()
    img = oracle_mod.AtomicImage(oracle_mod.Tersoff(), h0, len(R0), True)
    E = gb.get_path()["energies"]   # FP64 energies of the stored X
    # forces of the stored X come from the next step's evaluation
    gb.step(1)
    st2 = gb.get_state()
    for i in range(1, 8):
        Eo, Fo, _ = img(st["X"][i])
        assert np.max(np.abs(st2["F"][i] - Fo)) <= 1e-4, i
        assert abs(E[i] - Eo) <= 1e-10 * abs(Eo), i


def test_lj_band_mixed_forces_at_same_configuration(g, oracle_mod):
    """A strained vacancy-hop band (cell filter on, 4x4x4 cells, 255 atoms):
    mixed forces at the stored FP32 configuration within 1e-4 eps/sigma."""
    R0, h0, R1, h1 = ci.lj_vacancy_hop(ci.LJ_A, (4, 4, 4))
    h1s = ci.strained_cell(h1, 9, 0.02)
    R1 = ci.affine(R1, h1, h1s)
    gb = gpu_band(g, R0, h0, R1, h1s, 7, g.lj_potential(), k=1.0, dt=0.01, cell_filter=True,
                  precision=g.MIXED)
    gb.step(15)
    st = gb.get_state()
    gb.step(1)
    st2 = gb.get_state()
    img = oracle_mod.AtomicImage(oracle_mod.LJ(), h0, len(R0), True)
    for i in range(1, 6):
        Eo, Fo, _ = img(st["X"][i])
        assert np.max(np.abs(st2["F"][i] - Fo)) <= 1e-4, i


def test_lj_mixed_barrier_matches_fp64(g, oracle_mod):
    R0, h0, R1, h1 = lj_band_case()
    ob = oracle_band(oracle_mod, oracle_mod.LJ(), R0, h0, R1, h1, 7, k=1.0, dt=0.01,
                     cell_filter=False)
    ob.relax(1e-4, 20000)
    gb = gpu_band(g, R0, h0, R1, h1, 7, g.lj_potential(), k=1.0, dt=0.01, cell_filter=False,
                  precision=g.MIXED)
    done, conv = gb.relax(1e-3, 20000)
    E = gb.get_path()["energies"]
    assert abs((E.max() - E[0]) - ob.barrier()) <= 1e-3


# ---------------------------------------------------------------------------
# refinement
# ---------------------------------------------------------------------------

def test_insert_delete_keep_endpoints(g):
    R0, h0, R1, h1 = lj_band_case()
    gb = gpu_band(g, R0, h0, R1, h1, 5, g.lj_potential(), k=1.0, dt=0.01, cell_filter=False,
                  n_max=8)
    gb.step(3)
    s0 = gb.get_state()
    E0 = gb.get_path()["energies"]
    gb.insert_image(1)
    s1 = gb.get_state()
    assert s1["X"].shape[0] == 6
    np.testing.assert_array_equal(s1["X"][0], s0["X"][0])
    np.testing.assert_array_equal(s1["X"][-1], s0["X"][-1])
    np.testing.assert_array_equal(s1["X"][2], 0.5 * (s0["X"][1] + s0["X"][2]))
    np.testing.assert_array_equal(s1["X"][3], s0["X"][2])
    assert s1["n_pos"] == 0
    gb.delete_image(4)
    s2 = gb.get_state()
    assert s2["X"].shape[0] == 5
    np.testing.assert_array_equal(s2["X"][3], s1["X"][3])
    np.testing.assert_array_equal(s2["X"][4], s0["X"][4])
    with pytest.raises(g.CfnebError):
        gb.delete_image(0)
    with pytest.raises(g.CfnebError):
        gb.delete_image(4)
    gb.step(2)
    E1 = gb.get_path()["energies"]
    assert E1[0] == E0[0] and E1[-1] == E0[-1]


@pytest.mark.parametrize("kind", ["insert", "delete"])
def test_adaptive_refinement_matches_oracle(g, oracle_mod, kind):
    """Same refinement events as the oracle.  alpha_ins = 1 inserts at every
    check (until n_max); alpha_del = 2.5 deletes at every check (until n_min).
    Image counts and states agree after every block of steps."""
    # strained end cell and the cell filter: no mirror symmetry, so no exact
    # ties between segment lengths
    R0, h0, R1, h1 = lj_band_case(strain_seed=3)
    kw = dict(k=1.0, dt=0.01, cell_filter=True, adaptive=True, n_min=4, n_max=8)
    kw.update(dict(alpha_ins=1.0) if kind == "insert" else dict(alpha_ins=9.0, alpha_del=2.5))
    gb = gpu_band(g, R0, h0, R1, h1, 6, g.lj_potential(), **kw)
    ob = oracle_band(oracle_mod, oracle_mod.LJ(), R0, h0, R1, h1, 6, **kw)
    for _ in range(4):
        ob.step(30)
        gb.step(30)
        st = gb.get_state()
        assert st["X"].shape[0] == ob.N
        # 120 FIRE steps: rounding-order differences (FP64 tile sums, the
        # matrix square root) grow with the dynamics to ~1e-8 by the end
        _compare_state(st, ob, 3e-8)
    assert [e[0] for e in ob.events] == [kind, kind]


# ---------------------------------------------------------------------------
# full size: 98,304-atom Tersoff band (sampled oracle forces)
# ---------------------------------------------------------------------------

def test_large_tersoff_sampled_forces_mixed(g, oracle_mod):
    """98,304 atoms: the middle image of the large band (linear interpolation
    of the relaxed endpoints plus the seeded 0.01 A jitter), sampled atoms
    against the brute-force oracle."""
    cfg = ci.tersoff_graphite_hexdiamond(reps=ci.TERSOFF_LARGE_REPS, n_images=12)
    R0, h0, R1, h1 = cfg["endpoints"]
    s0 = R0 @ np.linalg.inv(h0)
    s1 = R1 @ np.linalg.inv(h1)
    s1 = s1 - np.round(s1 - s0)
    t = 5.0 / 11.0
    h = h0 + t * (h1 - h0)
    R = (s0 + t * (s1 - s0)) @ h + cfg["noise"][4]
    R, h = f32_structure(R, h)
    rng = np.random.default_rng(5)
    E, F, V = g.evaluate([(R, h)], g.tersoff_potential(), g.MIXED)
    idx = rng.choice(len(R), 64, replace=False)
    Fo = oracle_mod.Tersoff().forces_sampled(R, h, idx)
    # the unrelaxed middle image has close contacts (|F| up to ~430 eV/A)
    assert np.max(np.abs(F[0][idx] - Fo)) <= max(1e-4, 1e-6 * np.max(np.abs(Fo)))
    # the same configuration in FP64: sampled forces at 1e-10
    E64, F64, _ = g.evaluate([(R, h)], g.tersoff_potential(), g.FP64)
    assert _rel(F64[0][idx], Fo) <= 1e-10
    # both precisions report the FP64 total of the same configuration
    assert abs(E[0] - E64[0]) <= 1e-10 * abs(E64[0])


def test_large_tersoff_band_runs(g):
    cfg = ci.tersoff_graphite_hexdiamond(reps=ci.TERSOFF_LARGE_REPS, n_images=12,
                                         precision="mixed")
    R0, h0, R1, h1 = cfg["endpoints"]
    gb = gpu_band(g, R0, h0, R1, h1, 12, g.tersoff_potential(), k=0.1, dt=0.1,
                  cell_filter=True, noise=cfg["noise"], precision=g.MIXED, n_max=24)
    gb.step(5)
    p = gb.get_path()
    assert np.all(np.isfinite(p["energies"]))
    assert np.isfinite(p["fmax"]) and p["fmax"] > 0
    assert abs(p["energies"][0] / len(R0) - (-7.3955)) < 1e-3


# ---------------------------------------------------------------------------
# deformation-gradient filter variant and external pressure (Sec. II.C; the
# enthalpy H = U + P Omega of the 40 GPa example)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("variant,pressure", [(1, 0.0), (0, 0.05), (1, 0.05)])
def test_lj_filter_variant_and_pressure_fp64(g, oracle_mod, variant, pressure):
    """Strained vacancy hop with the cell filter on: the deformation-gradient
    coordinate D and/or an external pressure (eps/sigma^3), 8 FP64 steps
    against the oracle, energies (H) and virials included."""
    R0, h0, R1, h1 = lj_band_case(strain_seed=3)
    kw = dict(k=1.0, dt=0.01, cell_filter=True, variant=variant, pressure=pressure)
    gb = gpu_band(g, R0, h0, R1, h1, 7, g.lj_potential(), **kw)
    ob = oracle_band(oracle_mod, oracle_mod.LJ(), R0, h0, R1, h1, 7, **kw)
    gb.step(8)
    ob.step(8)
    st = gb.get_state()
    _compare_state(st, ob, 1e-9)
    for i in range(1, 6):
        assert _rel(st["virials"][i], ob.info[i]["V"]) <= 1e-10
    E = gb.get_path()["energies"]
    ob.compute()
    for i in range(1, 6):
        assert abs(E[i] - ob.E[i]) <= 1e-10 * max(1.0, abs(ob.E[i])), i


def test_tersoff_filter_variant_and_pressure_fp64(g, oracle_mod):
    """Graphite -> hexagonal diamond with D as the lattice coordinate and a
    pressure of 0.25 eV/A^3 (40 GPa), 5 FP64 steps against the oracle."""
    cfg = ci.tersoff_graphite_hexdiamond()
    R0, h0, R1, h1 = cfg["endpoints"]
    kw = dict(k=0.1, dt=0.1, cell_filter=True, variant=1, pressure=0.25)
    gb = gpu_band(g, R0, h0, R1, h1, 9, g.tersoff_potential(), noise=cfg["noise"], **kw)
    ob = oracle_band(oracle_mod, oracle_mod.Tersoff(), R0, h0, R1, h1, 9, noise=cfg["noise"],
                     **kw)
    gb.step(5)
    ob.step(5)
    st = gb.get_state()
    _compare_state(st, ob, 1e-9)
    for i in range(1, 8):
        assert _rel(st["virials"][i], ob.info[i]["V"]) <= 1e-10


def test_diamond_vacancy_hop_fp64(g, oracle_mod):
    """The serving stream's Tersoff vacancy request (cubic diamond, 63 atoms,
    unrelaxed endpoints, cell filter on): 10 FP64 steps against the oracle.
    (Longer runs of this band are chaotic in both implementations: fmax
    jumps between ~0.5 and ~50 eV/A as atoms cross the narrow cutoff shell.)"""
    R0, h0, R1, h1 = ci.diamond_vacancy_hop(ci.DIAMOND_A, (2, 2, 2))
    kw = dict(k=0.1, dt=0.1, cell_filter=True)
    gb = gpu_band(g, R0, h0, R1, h1, 9, g.tersoff_potential(), **kw)
    ob = oracle_band(oracle_mod, oracle_mod.Tersoff(), R0, h0, R1, h1, 9, **kw)
    gb.step(10)
    ob.step(10)
    _compare_state(gb.get_state(), ob, 1e-9)
