"""GPU parity of the NEP-style potential (descriptors + neural-network site
energy, synthetic weights) against the oracle's autograd FP64 definition:
single points in FP64 (1e-10) and mixed precision (forces within 1e-4
eV/A at the stored configuration, FP64 reported energies), and NEB steps
with the cell filter on the carbon graphite -> hexagonal-diamond path."""
import numpy as np
import pytest

import cfneb_inputs as ci
from _cases import f32_structure, gpu_band, oracle_band

pytestmark = pytest.mark.gpu
RC = 2.1


@pytest.fixture(scope="module")
def g():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2510_16721_gb300 as g
    g.build()
    return g


def _weights(seed=3):
    return ci.nep_weights(seed)


def _structures():
    Rg, hg, Rd, hd = ci.tersoff_endpoint_cells()
    hm = 0.5 * (hg + hd)
    hm[2, 2] = 0.5 * (hg[2, 2] + hd[2, 2]) * 0.72
    sm = 0.5 * (Rg @ np.linalg.inv(hg) + Rd @ np.linalg.inv(hd))
    rng = np.random.default_rng(12)
    out = []
    for R, h in [(Rg, hg), (sm @ hm, hm), ci.tile(Rd, hd, (3, 2, 2))]:
        out.append((R + rng.normal(0.0, 0.05, R.shape), h))
    return out


def _rel(a, b):
    return np.max(np.abs(np.asarray(a) - np.asarray(b))) / max(1.0, np.max(np.abs(b)))


def test_nep_single_points_fp64(g, oracle_mod):
    pot = oracle_mod.NEP(_weights(), rc=RC)
    S = _structures()
    E, F, V = g.evaluate(S, g.nep_potential(_weights(), RC), g.FP64)
    for k, (R, h) in enumerate(S):
        e, Fo, Vo = pot.evaluate(R, h)
        assert abs(E[k] - np.sum(e)) <= 1e-10 * max(1.0, abs(np.sum(e))), k
        assert _rel(F[k], Fo) <= 1e-10, k
        assert _rel(V[k], Vo) <= 1e-10, k


def test_nep_single_points_mixed(g, oracle_mod):
    pot = oracle_mod.NEP(_weights(), rc=RC)
    S = [f32_structure(R, h) for R, h in _structures()]
    E, F, V = g.evaluate(S, g.nep_potential(_weights(), RC), g.MIXED)
    for k, (R, h) in enumerate(S):
        e, Fo, Vo = pot.evaluate(R, h)
        assert np.max(np.abs(F[k] - Fo)) <= 1e-4, k
        assert abs(E[k] - np.sum(e)) <= 1e-10 * max(1.0, abs(np.sum(e))), k
        assert _rel(V[k], Vo) <= 1e-5, k


def test_nep_band_steps_fp64(g, oracle_mod):
    """96-atom graphite -> hexagonal-diamond band, cell filter on, 9 images:
    12 NEB + FIRE steps against the oracle band at 1e-9."""
    R0, h0, R1, h1 = ci.graphite_hexdiamond_path((3, 2, 2))
    kw = dict(k=0.1, dt=0.05, cell_filter=True)
    gb = gpu_band(g, R0, h0, R1, h1, 9, g.nep_potential(_weights(), RC), **kw)
    ob = oracle_band(oracle_mod, oracle_mod.NEP(_weights(), rc=RC), R0, h0, R1, h1, 9, **kw)
    for _ in range(3):
        gb.step(4)
        ob.step(4)
        st = gb.get_state()
        for i in range(ob.N):
            assert _rel(st["X"][i], ob.X[i]) <= 1e-9, ("X", i)
        for i in range(1, ob.N - 1):
            assert _rel(st["F"][i], ob.F[i]) <= 1e-9, ("F", i)
    # reported energies (the FP64 energy pass) of the current images
    E = gb.get_path()["energies"]
    img = oracle_mod.AtomicImage(oracle_mod.NEP(_weights(), rc=RC), h0, len(R0), True)
    for i in range(ob.N):
        Eo = img(ob.X[i])[0]
        assert abs(E[i] - Eo) <= 1e-10 * max(1.0, abs(Eo)), i


def test_nep_band_mixed_forces_at_same_configuration(g, oracle_mod):
    R0, h0, R1, h1 = ci.graphite_hexdiamond_path((3, 2, 2))
    gb = gpu_band(g, R0, h0, R1, h1, 9, g.nep_potential(_weights(), RC), k=0.1, dt=0.05,
                  cell_filter=True, precision=g.MIXED)
    gb.step(6)
    st = gb.get_state()
    gb.step(1)
    st2 = gb.get_state()
    img = oracle_mod.AtomicImage(oracle_mod.NEP(_weights(), rc=RC), h0, len(R0), True)
    for i in range(1, 8):
        _, Fo, _ = img(st["X"][i])
        assert np.max(np.abs(st2["F"][i] - Fo)) <= 1e-4, i


def test_nep_invalid_weights_are_rejected(g):
    R0, h0, R1, h1 = ci.graphite_hexdiamond_path((2, 2, 1))
    w = _weights()
    w[7] = np.nan
    with pytest.raises(g.CfnebError) as e:
        gpu_band(g, R0, h0, R1, h1, 5, g.nep_potential(w, RC), k=0.1, dt=0.05)
    assert e.value.status == g.ERR_INVALID_ARG
    with pytest.raises(g.CfnebError):
        gpu_band(g, R0, h0, R1, h1, 5, g.nep_potential(_weights(), -1.0), k=0.1, dt=0.05)


def test_large_nep_band_image_properties(g):
    """Full size: a 98,304-atom image of the graphite -> hexagonal-diamond
    path (the middle of the linear interpolation in the 32 x 24 x 16 tiling,
    seeded 0.02 A jitter) under the NEP-style potential, where the oracle's
    whole-structure autograd does not reach.  Properties that hold at any
    size: the forces sum to zero (translation invariance); a central
    difference of the FP64 energy along a random direction of all atoms
    matches -F.d; the mixed forces match the FP64 ones on 64 sampled atoms
    at the FP32-rounded configuration (1e-4 eV/A)."""
    R0, h0, R1, h1 = ci.graphite_hexdiamond_path(ci.TERSOFF_LARGE_REPS)
    s0 = R0 @ np.linalg.inv(h0)
    s1 = R1 @ np.linalg.inv(h1)
    h = 0.5 * (h0 + h1)
    rng = np.random.default_rng(21)
    R = (0.5 * (s0 + s1)) @ h + rng.normal(0.0, 0.02, R0.shape)
    R, h = f32_structure(R, h)
    pot = g.nep_potential(_weights(), RC)
    E, F, _ = g.evaluate([(R, h)], pot, g.FP64)
    F = F[0]
    assert len(R) == 98304
    assert np.all(np.abs(F.sum(axis=0)) <= 1e-9 * len(R) * max(1.0, np.max(np.abs(F))))
    d = rng.normal(size=R.shape)
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    s = 1e-4
    Ep, _, _ = g.evaluate([(R + s * d, h)], pot, g.FP64)
    Em, _, _ = g.evaluate([(R - s * d, h)], pot, g.FP64)
    fd = -(Ep[0] - Em[0]) / (2.0 * s)
    fd_ref = np.sum(F * d)
    assert abs(fd - fd_ref) <= 1e-3 * max(1.0, np.sqrt(np.sum(F * F))), (fd, fd_ref)
    _, Fm, _ = g.evaluate([(R, h)], pot, g.MIXED)
    idx = rng.choice(len(R), 64, replace=False)
    assert np.max(np.abs(Fm[0][idx] - F[idx])) <= 1e-4
