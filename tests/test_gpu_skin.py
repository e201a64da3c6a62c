"""Cell-list (and neighbour-list) reuse with a skin.

With a skin the lists cover rc + skin and an image keeps them while no pair
can have moved into rc; a kept list only changes which rounding the pair
vectors get, never which pairs are summed.  So a band with a skin must
match the FP64 oracle at the same tolerances as one that rebuilds at every
step, must actually skip rebuilds, and must rebuild once atoms have moved
far enough (a tiny skin), after image insertion or deletion, and when its
cell changes.
"""
import math

import numpy as np
import pytest

import cfneb_inputs as ci
from _cases import gpu_band, lj_band_case, oracle_band

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
    return np.max(np.abs(np.asarray(a) - np.asarray(b))) / max(floor, np.max(np.abs(b)))


def _compare_state(st, ob, tol):
    assert st["X"].shape[0] == ob.N
    for i in range(ob.N):
        assert _rel(st["X"][i], ob.X[i]) <= tol, ("X", i)
    for i in range(1, ob.N - 1):
        assert _rel(st["F"][i], ob.F[i]) <= tol, ("F", i)
        assert _rel(st["Fneb"][i], ob.fneb[i - 1].reshape(st["Fneb"][i].shape)) <= tol, ("Fneb", i)


def _tersoff576(g, oracle_mod, skin, precision=0, with_oracle=True):
    cfg = ci.tersoff_graphite_hexdiamond()
    R0, h0, R1, h1 = cfg["endpoints"]
    gb = gpu_band(g, R0, h0, R1, h1, 9, g.tersoff_potential(), k=0.1, dt=0.1,
                  cell_filter=True, noise=cfg["noise"], precision=precision, skin=skin)
    ob = None
    if with_oracle:
        ob = oracle_band(oracle_mod, oracle_mod.Tersoff(), R0, h0, R1, h1, 9, k=0.1, dt=0.1,
                         cell_filter=True, noise=cfg["noise"])
    return gb, ob


def test_tersoff_skin_reuses_lists_and_matches_oracle(g, oracle_mod):
    """The default Tersoff skin (0.15 A): 25 FP64 steps, every block of 5
    against the oracle at the band-state tolerance of the parity tests."""
    gb, ob = _tersoff576(g, oracle_mod, None)
    for _ in range(5):
        gb.step(5)
        ob.step(5)
        _compare_state(gb.get_state(), ob, 1e-9)
    builds, evals, skin = gb.list_stats()
    assert skin == pytest.approx(0.15)
    # 7 interior images: evaluations of the steps plus the ad-hoc ones
    assert evals >= 7 * 25
    assert 7 <= builds < evals


def test_skin_zero_rebuilds_at_every_evaluation(g, oracle_mod):
    gb, ob = _tersoff576(g, oracle_mod, 0.0)
    gb.step(6)
    ob.step(6)
    _compare_state(gb.get_state(), ob, 1e-9)
    builds, evals, skin = gb.list_stats()
    assert skin == 0.0 and builds == evals >= 7 * 6


def test_tiny_skin_rebuilds_as_atoms_move(g, oracle_mod):
    """A 1e-4 A skin: the first FIRE moves already exceed it, so images
    rebuild while the band relaxes; results stay at oracle parity."""
    gb, ob = _tersoff576(g, oracle_mod, 1e-4)
    gb.step(12)
    ob.step(12)
    _compare_state(gb.get_state(), ob, 1e-9)
    builds, evals, _ = gb.list_stats()
    assert builds > 7 * 6


def test_mixed_forces_from_kept_lists_match_oracle(g, oracle_mod):
    """Mixed precision: forces evaluated from kept lists (no rebuild between
    the stored configuration and its evaluation) against the oracle at that
    configuration, at the mixed-path force tolerance."""
    gb, _ = _tersoff576(g, None, None, precision=1, with_oracle=False)
    cfg = ci.tersoff_graphite_hexdiamond()
    R0, h0 = cfg["endpoints"][0], cfg["endpoints"][1]
    gb.step(20)
    b0, e0, _ = gb.list_stats()
    st = gb.get_state()
    gb.step(1)
    st2 = gb.get_state()
    b1, e1, _ = gb.list_stats()
    assert b0 < e0
    img = oracle_mod.AtomicImage(oracle_mod.Tersoff(), h0, len(R0), True)
    for i in range(1, 8):
        _, Fo, _ = img(st["X"][i])
        assert np.max(np.abs(st2["F"][i] - Fo)) <= max(1e-4, 1e-6 * np.max(np.abs(Fo))), i
    assert b1 - b0 < e1 - e0          # some image kept its list for that step


def test_lj_skin_with_cell_filter_matches_oracle(g, oracle_mod):
    """LJ walks the cell list directly; with a skin it keeps the bins of the
    build (strained end cell: every image's cell changes as it relaxes)."""
    R0, h0, R1, h1 = lj_band_case(strain_seed=3)
    kw = dict(k=1.0, dt=0.01, cell_filter=True)
    gb = gpu_band(g, R0, h0, R1, h1, 7, g.lj_potential(), skin=0.3, **kw)
    ob = oracle_band(oracle_mod, oracle_mod.LJ(), R0, h0, R1, h1, 7, **kw)
    for _ in range(4):
        gb.step(10)
        ob.step(10)
        _compare_state(gb.get_state(), ob, 1e-9)
    builds, evals, _ = gb.list_stats()
    assert builds < evals


@pytest.mark.parametrize("kind", ["insert", "delete"])
def test_adaptive_refinement_with_skin(g, oracle_mod, kind):
    """Image insertion and deletion move images between slots; every slot
    rebuilds its lists after a change, and the events and states still
    follow the oracle."""
    R0, h0, R1, h1 = lj_band_case(strain_seed=3)
    kw = dict(k=1.0, dt=0.01, cell_filter=True, adaptive=True, n_min=4, n_max=8)
    kw.update(dict(alpha_ins=1.0) if kind == "insert" else dict(alpha_ins=9.0, alpha_del=2.5))
    gb = gpu_band(g, R0, h0, R1, h1, 6, g.lj_potential(), skin=0.3, **kw)
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


@pytest.mark.parametrize("skin", [2.2, math.nan])
def test_invalid_skin_is_rejected(g, skin):
    cfg = ci.tersoff_graphite_hexdiamond(reps=(2, 2, 2))
    R0, h0, R1, h1 = cfg["endpoints"]
    with pytest.raises(g.CfnebError):
        gpu_band(g, R0, h0, R1, h1, 5, g.tersoff_potential(), k=0.1, dt=0.1, skin=skin)


@pytest.mark.parametrize("precision", [0, 1])
def test_lj_neighbour_list_and_cell_walk_match(g, oracle_mod, precision):
    """LJ bands with a skin keep per-atom neighbour lists (entries inside rc
    first, the skin shell after them); with skin 0 the force kernel walks
    the cell list.  A strained 4x4x4 vacancy band (255 atoms, cell filter
    on) through 12 steps on both paths: FP64 states within 1e-9 of the
    oracle, mixed forces at the stored configuration within 1e-4 eps/sigma
    of it and within 1e-4 of each other (both paths form the same FP32 pair
    vectors; only the summation order differs)."""
    R0, h0, R1, h1 = ci.lj_vacancy_hop(ci.LJ_A, (4, 4, 4))
    h1s = ci.strained_cell(h1, 9, 0.02)
    R1 = ci.affine(R1, h1, h1s)
    kw = dict(k=1.0, dt=0.01, cell_filter=True, precision=precision)
    lists = gpu_band(g, R0, h0, R1, h1s, 7, g.lj_potential(), **kw)
    walk = gpu_band(g, R0, h0, R1, h1s, 7, g.lj_potential(), skin=0.0, **kw)
    assert lists.list_stats()[2] == pytest.approx(0.3)
    if precision == 0:
        ob = oracle_band(oracle_mod, oracle_mod.LJ(), R0, h0, R1, h1s, 7, k=1.0, dt=0.01,
                         cell_filter=True)
        for _ in range(3):
            lists.step(4)
            walk.step(4)
            ob.step(4)
            _compare_state(lists.get_state(), ob, 1e-9)
            _compare_state(walk.get_state(), ob, 1e-9)
    else:
        lists.step(12)
        walk.step(12)
        sl, sw = lists.get_state(), walk.get_state()
        lists.step(1)
        walk.step(1)
        fl, fw = lists.get_state()["F"], walk.get_state()["F"]
        img = oracle_mod.AtomicImage(oracle_mod.LJ(), h0, len(R0), True)
        for i in range(1, 6):
            _, Fo, _ = img(sl["X"][i])
            assert np.max(np.abs(fl[i] - Fo)) <= 1e-4, i
            _, Fo, _ = img(sw["X"][i])
            assert np.max(np.abs(fw[i] - Fo)) <= 1e-4, i
    b, e, _ = lists.list_stats()
    assert b < e                      # lists kept between builds
    b, e, _ = walk.list_stats()
    assert b == e


def test_lj_neighbour_list_overflow_is_reported(g):
    """The list capacity follows the endpoints' mean density.  256 atoms at
    FCC density packed into one corner of a 20 sigma box have ~86 entries
    within rc + skin but a capacity of 40: the list kernel caps its writes
    and the band reports the overflow."""
    R = ci.fcc(ci.LJ_A, 4, 4, 4)[0] + 1.0
    h = np.eye(3) * 20.0
    R1 = R.copy()
    R1[0] += 0.05
    with pytest.raises(g.CfnebError) as e:
        gb = gpu_band(g, R, h, R1, h, 5, g.lj_potential(), k=1.0, dt=0.01)
        gb.step(1)
    assert e.value.status == g.ERR_NBR_OVERFLOW


@pytest.mark.parametrize("reps,lists", [((20, 20, 20), True), ((33, 33, 33), False)])
def test_large_lj_band_sampled_forces(g, oracle_mod, reps, lists):
    """Full-size LJ vacancy bands: 31,999 atoms (the largest band of the
    64-band batch) keep neighbour lists; 143,747 atoms exceed what a list
    entry can index (2^17 slots) and walk the cell list.  After 6 mixed
    steps, forces of an interior image at its stored configuration against
    the brute-force oracle on 48 sampled atoms (1e-4 eps/sigma), and the
    FP64 band's first evaluation at 1e-10."""
    R0, h0, R1, h1 = ci.lj_vacancy_hop(ci.LJ_A, reps)
    for prec, tol, nstep in ((g.MIXED, 1e-4, 6), (g.FP64, 1e-10, 0)):
        gb = gpu_band(g, R0, h0, R1, h1, 5, g.lj_potential(), k=1.0, dt=0.01,
                      cell_filter=False, precision=prec)
        assert gb.launches_per_step() == (13 if lists else 12)
        gb.step(nstep)
        st = gb.get_state()
        gb.step(1)
        F = gb.get_state()["F"][2][: len(R0)]
        X = st["X"][2][: len(R0)]
        idx = np.random.default_rng(7).choice(len(R0), 48, replace=False)
        Fo = oracle_mod.LJ().forces_sampled(X, h0, idx)
        err = np.max(np.abs(F[idx] - Fo))
        assert err <= (tol if prec == g.MIXED else tol * max(1.0, np.max(np.abs(Fo)))), err
        gb.destroy()
