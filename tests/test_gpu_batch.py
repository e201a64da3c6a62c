"""Batched execution: many uneven bands (LJ and Tersoff mixed) stepped by one
launch per kernel under one CUDA graph.

Each band's result must not depend on the company it keeps: every reduction
of a band sums its own tile slots in a fixed order, so a band stepped inside
a batch is bitwise identical to the same band stepped alone.
"""
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


def _make(g, which, precision, **kw):
    if which == "lj31":
        R0, h0, R1, h1 = lj_band_case()
        return gpu_band(g, R0, h0, R1, h1, 7, g.lj_potential(), k=1.0, dt=0.01,
                        cell_filter=False, precision=precision, **kw)
    if which == "lj72":   # 3x3x2 cells, vacancy, 0.3% strained end cell
        R0, h0, R1, h1 = ci.lj_vacancy_hop(ci.LJ_A, (3, 3, 2))
        h1s = ci.strained_cell(h1, 3, 0.003)
        return gpu_band(g, R0, h0, ci.affine(R1, h1, h1s), h1s, 5, g.lj_potential(), k=1.0,
                        dt=0.01, cell_filter=True, precision=precision, **kw)
    if which == "lj255":
        R0, h0, R1, h1 = ci.lj_vacancy_hop(ci.LJ_A, (4, 4, 4), divacancy=True)
        h1s = ci.strained_cell(h1, 5, 0.02)
        return gpu_band(g, R0, h0, ci.affine(R1, h1, h1s), h1s, 5, g.lj_potential(), k=1.0,
                        dt=0.01, cell_filter=True, precision=precision, **kw)
    if which == "nep96":  # the NEP-style potential on a 96-atom carbon path
        R0, h0, R1, h1 = ci.graphite_hexdiamond_path((3, 2, 2))
        return gpu_band(g, R0, h0, R1, h1, 7, g.nep_potential(ci.nep_weights(3), 2.1), k=0.1,
                        dt=0.05, cell_filter=True, precision=precision, **kw)
    cfg = ci.tersoff_graphite_hexdiamond()
    R0, h0, R1, h1 = cfg["endpoints"]
    return gpu_band(g, R0, h0, R1, h1, 9, g.tersoff_potential(), k=0.1, dt=0.1,
                    cell_filter=True, noise=cfg["noise"], precision=precision, **kw)


def _same(a, b):
    sa, sb = a.get_state(), b.get_state()
    for key in ("X", "F", "Fneb", "virials"):
        np.testing.assert_array_equal(sa[key], sb[key], err_msg=key)
    assert sa["steps"] == sb["steps"] and sa["ci"] == sb["ci"]


@pytest.mark.parametrize("precision", [0, 1])
def test_batch_equals_alone_bitwise(g, precision):
    names = ["lj31", "lj255", "ters576", "nep96"]
    batched = [_make(g, w, precision) for w in names]
    alone = [_make(g, w, precision) for w in names]
    bt = g.Batch(precision)
    for b in batched:
        bt.add(b)
    bt.step(12)
    for b in alone:
        b.step(12)
    for a, b in zip(batched, alone):
        _same(a, b)
    st = bt.status()
    assert [s["steps"] for s in st] == [12, 12, 12, 12]
    bt.destroy()


def _oracle_of(o, which):
    if which == "lj31":
        R0, h0, R1, h1 = lj_band_case()
        return oracle_band(o, o.LJ(), R0, h0, R1, h1, 7, k=1.0, dt=0.01, cell_filter=False)
    if which == "lj72":
        R0, h0, R1, h1 = ci.lj_vacancy_hop(ci.LJ_A, (3, 3, 2))
        h1s = ci.strained_cell(h1, 3, 0.003)
        return oracle_band(o, o.LJ(), R0, h0, ci.affine(R1, h1, h1s), h1s, 5, k=1.0, dt=0.01,
                           cell_filter=True)
    if which == "lj255":
        R0, h0, R1, h1 = ci.lj_vacancy_hop(ci.LJ_A, (4, 4, 4), divacancy=True)
        h1s = ci.strained_cell(h1, 5, 0.02)
        return oracle_band(o, o.LJ(), R0, h0, ci.affine(R1, h1, h1s), h1s, 5, k=1.0, dt=0.01,
                           cell_filter=True)
    cfg = ci.tersoff_graphite_hexdiamond()
    R0, h0, R1, h1 = cfg["endpoints"]
    return oracle_band(o, o.Tersoff(), R0, h0, R1, h1, 9, k=0.1, dt=0.1, cell_filter=True,
                       noise=cfg["noise"])


def test_batch_matches_oracle_fp64(g, oracle_mod):
    """Uneven FP64 bands (31-atom fixed-cell and 72- and 255-atom cell-filter
    LJ hops, the 576-atom Tersoff carbon band) stepped together in one batch:
    each band's state after 10 steps is the oracle's at 1e-9."""
    names = ["lj31", "lj72", "lj255", "ters576"]
    batched = [_make(g, w, 0) for w in names]
    bt = g.Batch(0)
    for b in batched:
        bt.add(b)
    bt.step(10)
    for name, b in zip(names, batched):
        ob = _oracle_of(oracle_mod, name)
        ob.step(10)
        st = b.get_state()
        assert st["X"].shape[0] == ob.N
        for i in range(ob.N):
            d = np.max(np.abs(st["X"][i] - ob.X[i])) / max(1.0, np.max(np.abs(ob.X[i])))
            assert d <= 1e-9, (name, "X", i, d)
        for i in range(1, ob.N - 1):
            Fo = ob.fneb[i - 1].reshape(st["Fneb"][i].shape)
            d = np.max(np.abs(st["Fneb"][i] - Fo)) / max(1.0, np.max(np.abs(Fo)))
            assert d <= 1e-9, (name, "Fneb", i, d)
        assert st["ci"] == ob.ci, name
    bt.destroy()


def test_batch_relax_matches_alone(g):
    batched = [_make(g, w, 0) for w in ("lj31", "lj72")]
    alone = [_make(g, w, 0) for w in ("lj31", "lj72")]
    bt = g.Batch(0)
    for b in batched:
        bt.add(b)
    nconv = bt.relax(5e-2, 4000)
    assert nconv == 2
    for b in alone:
        done, conv = b.relax(5e-2, 4000)
        assert conv
    for a, b in zip(batched, alone):
        _same(a, b)
        np.testing.assert_array_equal(a.get_path()["energies"], b.get_path()["energies"])
    st = bt.status()
    assert all(s["converged"] for s in st)
    assert all(s["fmax"] < 5e-2 for s in st)


def test_budget_admission_and_removal(g):
    a, b, c = (_make(g, w, 0) for w in ("lj31", "lj255", "ters576"))
    budget = a.bytes() + max(b.bytes(), c.bytes())
    bt = g.Batch(0, budget_bytes=budget)
    assert bt.try_add(a) and bt.try_add(b)
    assert not bt.try_add(c)                 # over the memory budget
    assert bt.bytes() == (a.bytes() + b.bytes(), budget)
    ref = _make(g, "lj255", 0)
    bt.step(5)
    ref.step(5)
    bt.remove(b)                             # b continues on its own stream
    assert bt.try_add(c)
    bt.step(3)
    b.step(4)
    ref.step(4)
    _same(b, ref)
    bt.destroy()


def test_batch_rejects_mixed_precision(g):
    bt = g.Batch(0)
    with pytest.raises(g.CfnebError):
        bt.add(_make(g, "lj31", 1))


def test_adaptive_band_in_batch(g):
    kw = dict(adaptive=True, n_min=4, n_max=9, alpha_ins=1.0)
    a = _make(g, "lj31", 0, **kw)
    ref = _make(g, "lj31", 0, **kw)
    other = _make(g, "lj255", 0)
    bt = g.Batch(0)
    bt.add(a)
    bt.add(other)
    bt.step(45)
    ref.step(45)
    assert a.n_images == ref.n_images > 7
    _same(a, ref)


def test_autotune_leaves_state_and_forces(g, oracle_mod):
    """Autotuning evaluates without moving: X and the move count are left as
    they were, and the forces at the chosen bin width still match the
    oracle (FP64)."""
    b = _make(g, "lj255", 0, bin_scale=0.0)
    b.step(3)
    before = b.get_state()
    best = b.autotune(3)
    assert best in (0.5, 0.75, 1.0, 1.3)
    after = b.get_state()
    np.testing.assert_array_equal(after["X"], before["X"])
    assert after["steps"] == before["steps"]
    b.step(1)
    st = b.get_state()
    R0, h0, _, _ = ci.lj_vacancy_hop(ci.LJ_A, (4, 4, 4), divacancy=True)
    img = oracle_mod.AtomicImage(oracle_mod.LJ(), h0, len(R0), True)
    for i in (1, 2, 3):
        _, Fo, _ = img(after["X"][i])
        assert np.max(np.abs(st["F"][i] - Fo)) <= 1e-10 * max(1.0, np.max(np.abs(Fo)))


def test_autotune_picks_kernel_variant_mixed(g, oracle_mod):
    """Mixed LJ band with neighbour lists: the autotuner picks the bin width
    and then the force kernel's blocks per SM among its variants; X and the
    move count are left alone, and the forces of the chosen variant match
    the oracle within the mixed tolerance."""
    b = _make(g, "lj255", 1, bin_scale=0.0)
    b.step(3)
    before = b.get_state()
    best = b.autotune(3)
    scale, minb = b.tuning()
    assert best in (0.5, 0.75, 1.0, 1.3) and scale == pytest.approx(best)
    assert minb in (5, 6, 7, 8)
    after = b.get_state()
    np.testing.assert_array_equal(after["X"], before["X"])
    assert after["steps"] == before["steps"]
    b.step(1)
    st = b.get_state()
    R0, h0, _, _ = ci.lj_vacancy_hop(ci.LJ_A, (4, 4, 4), divacancy=True)
    img = oracle_mod.AtomicImage(oracle_mod.LJ(), h0, len(R0), True)
    for i in (1, 2, 3):
        _, Fo, _ = img(after["X"][i])
        # FP32 pair vectors at the close contacts of the moving divacancy
        # (|F| up to ~25 eps/sigma): the relative FP32 bound
        assert np.max(np.abs(st["F"][i] - Fo)) <= max(1e-4, 1e-5 * np.max(np.abs(Fo)))


def test_batch_autotune_sets_variants(g):
    bands = [_make(g, w, 1, bin_scale=0.0) for w in ("lj255", "ters576")]
    bt = g.Batch(1)
    for b in bands:
        bt.add(b)
    bt.autotune(2)
    assert bands[0].tuning()[1] in (5, 6, 7, 8)
    assert bands[1].tuning()[1] in (4, 5, 6, 7, 8)
    bt.step(3)
    assert all(s["status"] == 0 for s in bt.status())
    bt.destroy()


def test_full_lj_batch_sampled_forces_mixed(g, oracle_mod):
    """The 64-band LJ batch as the benchmark steps it (vacancy and divacancy
    hops of 270-30,346 atoms, 5-15 images, +-2% end-cell strain, cell filter
    with the lattice scale J, mixed precision, one batch): after three batch
    steps, the atom rows of the generalised force (F D^T) of the middle image
    of the smallest, a median and the largest band, at the stored
    configuration, against the brute-force oracle on 32 sampled atoms each
    (1e-4 eps/sigma, or 2e-6 of the largest force on close contacts)."""
    bcs = ci.lj_batch(seed=4)
    bands = []
    for bc in bcs:
        R0, h0, R1, h1 = bc["endpoints"]
        bands.append(gpu_band(g, R0, h0, R1, h1, bc["n_images"], g.lj_potential(), k=bc["k"],
                              dt=bc["dt"], cell_filter=True, precision=g.MIXED,
                              cell_factor=g.CELL_FACTOR_J))
    bt = g.Batch(g.MIXED)
    for b in bands:
        bt.add(b)
    bt.step(3)
    order = np.argsort([len(bc["endpoints"][0]) for bc in bcs])
    picks = [int(order[0]), int(order[len(order) // 2]), int(order[-1])]
    states = {q: bands[q].get_state() for q in picks}
    bt.step(1)  # forces of the stored configurations come from this evaluation
    rng = np.random.default_rng(11)
    for q in picks:
        R0, h0, _, _ = bcs[q]["endpoints"]
        n = len(R0)
        i = bcs[q]["n_images"] // 2
        c = abs(np.linalg.det(h0)) ** (1.0 / 3.0) * n ** (1.0 / 6.0)
        R, h, D = oracle_mod.from_generalized(states[q]["X"][i], h0, c)
        idx = rng.choice(n, 32, replace=False)
        Fo = oracle_mod.LJ().forces_sampled(R, h, idx) @ D.T
        F = bands[q].get_state()["F"][i][:n]
        err = np.max(np.abs(F[idx] - Fo))
        assert err <= max(1e-4, 2e-6 * np.max(np.abs(Fo))), (q, n, err)
    bt.destroy()
    for b in bands:
        b.destroy()
