"""Precision contract of the mixed path at the large graphite -> hexagonal
diamond band (98,304 atoms, 12 images, cell filter on).

The NEB reductions (Sec. II.A: the tangent norms, the spring distances, the
projection F.tau) and the FIRE sums are formed from ten per-image dot
products.  In the mixed path the vectors are FP32; each row's 3-term product
sum is rounded once and the rows are accumulated with a two-sum pair, then
in FP64, so each dot's error is bounded by 2^-23 sum |a_c b_c| over its
terms (plus 2^-24 of the same sum for the FP32 differences dX+-) and does
not grow with the row count.  Checked here against the dots written out in
numpy FP64 from the very FP32 values the kernels read.

The band is then put at the same X in the FP64 path (cfneb_set_state) and
one non-moving evaluation is compared: climbing image, upwind branch of
every image, the NEB coefficients, f_NEB and fmax.  The FP64 path is the
oracle's stand-in at this size (it matches the oracle at 1e-10 on the
smaller bands of test_gpu_parity.py; the brute-force oracle needs hours per
evaluation of 98,304 atoms).

Last, the mixed path's tangent rule (energy differences within the step
energies' error bound count as ties) on a 98,303-atom carbon vacancy band.
"""
import numpy as np
import pytest

import cfneb_inputs as ci
from _cases import gpu_band

pytestmark = pytest.mark.gpu

EPS32 = 2.0 ** -24


@pytest.fixture(scope="module")
def g():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2510_16721_gb300 as g
    g.build()
    return g


def _dots_fp64(X, F):
    """|dX+|^2, |dX-|^2, dX+.dX-, F.dX+, F.dX-, F.F of every interior image
    and the sums of the absolute terms, from the stored values in FP64."""
    N = X.shape[0]
    out = np.zeros((N, 6))
    mag = np.zeros((N, 6))
    for i in range(1, N - 1):
        dp = (X[i + 1] - X[i]).ravel()
        dm = (X[i] - X[i - 1]).ravel()
        f = F[i].ravel()
        terms = [(dp, dp), (dm, dm), (dp, dm), (f, dp), (f, dm), (f, f)]
        for k, (a, b) in enumerate(terms):
            out[i, k] = np.dot(a, b)
            mag[i, k] = np.dot(np.abs(a), np.abs(b))
    return out, mag


def _branch(E, i):
    """Upwind case of image i: +1 uphill forward, -1 uphill backward, 0 the
    energy-weighted mix (Henkelman-Jonsson)."""
    if E[i + 1] > E[i] > E[i - 1]:
        return 1
    if E[i + 1] < E[i] < E[i - 1]:
        return -1
    return 0


@pytest.fixture(scope="module")
def large_pair(g):
    cfg = ci.tersoff_graphite_hexdiamond(ci.TERSOFF_LARGE_REPS, n_images=12)
    R0, h0, R1, h1 = cfg["endpoints"]
    kw = dict(k=0.1, dt=0.1, cell_filter=True, noise=cfg["noise"])
    bm = gpu_band(g, R0, h0, R1, h1, 12, g.tersoff_potential(), precision=g.MIXED, **kw)
    bm.step(30)
    X = bm.get_state()["X"]
    bm.relax(1e30, 1)  # one evaluation at X, no move
    sm = bm.get_state()
    am = bm.image_scalars()
    bd = gpu_band(g, R0, h0, R1, h1, 12, g.tersoff_potential(), precision=g.FP64, **kw)
    bd.set_state(X)
    bd.relax(1e30, 1)
    sd = bd.get_state()
    ad = bd.image_scalars()
    pm, pd = bm.get_path(), bd.get_path()
    return dict(X=X, sm=sm, am=am, sd=sd, ad=ad, fmax_m=pm["fmax"], fmax_d=pd["fmax"])


def test_mixed_dots_within_bound(large_pair):
    sm, am = large_pair["sm"], large_pair["am"]
    assert np.array_equal(sm["X"], large_pair["X"])  # the evaluation did not move
    ref, mag = _dots_fp64(sm["X"], sm["F"])
    N = ref.shape[0]
    for i in range(1, N - 1):
        for k in range(6):
            bound = 4.0 * EPS32 * mag[i, k] + 1e-30
            err = abs(am["dots"][i, k] - ref[i, k])
            assert err <= bound, (i, k, err, bound)


def test_mixed_matches_fp64_at_same_x(large_pair):
    am, ad, sm, sd = large_pair["am"], large_pair["ad"], large_pair["sm"], large_pair["sd"]
    N = am["E"].shape[0]
    assert np.array_equal(sd["X"], large_pair["X"])
    # climbing image and upwind branches
    assert sm["ci"] == sd["ci"]
    for i in range(1, N - 1):
        assert _branch(am["E"], i) == _branch(ad["E"], i), i
    # dots of the coordinates alone: the same FP32-exact X on both sides
    for i in range(1, N - 1):
        for k in range(3):
            assert abs(am["dots"][i, k] - ad["dots"][i, k]) <= 4.0 * EPS32 * abs(ad["dots"][i, k])
    # forces: FP32 arithmetic against FP64 at the same configuration
    dF = np.max(np.abs(sm["F"][1:-1] - sd["F"][1:-1]))
    assert dF <= 1e-4, dF
    # NEB coefficients and forces
    for i in range(1, N - 1):
        np.testing.assert_allclose(am["coef"][i], ad["coef"][i], rtol=1e-4, atol=1e-7)
    dG = np.max(np.abs(sm["Fneb"][1:-1] - sd["Fneb"][1:-1]))
    assert dG <= 2e-4, dG
    assert abs(large_pair["fmax_m"] - large_pair["fmax_d"]) <= 2e-4
    # step energies: FP32 site energies summed in FP64 against FP64.  The
    # FP32 rounding of each site energy (f_R and b f_A cancel to a fifth of
    # their size) is systematic in a crystal: bounded per atom, and largely
    # the same in neighbouring images
    n = (sm["X"].shape[1] - 3)
    dE = am["E"] - ad["E"]
    dd = np.diff(dE)
    print("step-energy error: max |dE| %.3e eV (%.2e per atom), max |d(E_i+1 - E_i)| %.3e eV"
          % (np.max(np.abs(dE)), np.max(np.abs(dE)) / n, np.max(np.abs(dd))))
    assert np.max(np.abs(dE)) <= 4e-6 * n


def _coefs(E, dots, ci, k, etol):
    """The f_NEB coefficients (a, b) of every interior image from the step
    energies and the ten dots, by the tangent rule with ties up to etol
    (Sec. II.A, upwind tangent; equal-weight tangent when both energy
    differences are within etol)."""
    out = {}
    for i in range(1, len(E) - 1):
        Em, E0, Ep = E[i - 1], E[i], E[i + 1]
        if Ep - E0 > etol and E0 - Em > etol:
            wp, wm = 1.0, 0.0
        elif E0 - Ep > etol and Em - E0 > etol:
            wp, wm = 0.0, 1.0
        else:
            a, c = abs(Ep - E0), abs(Em - E0)
            dmax, dmin = max(a, c), min(a, c)
            if dmax <= etol:
                wp, wm = 1.0, 1.0
            elif Ep > Em:
                wp, wm = dmax, dmin
            else:
                wp, wm = dmin, dmax
        pp, mm, pm, fp, fm = dots[i][:5]
        itn = 1.0 / np.sqrt(wp * wp * pp + 2.0 * wp * wm * pm + wm * wm * mm)
        ft = (wp * fp + wm * fm) * itn
        gamma = -2.0 * ft if i == ci else k * (np.sqrt(pp) - np.sqrt(mm)) - ft
        out[i] = (gamma * wp * itn, gamma * wm * itn, wp, wm)
    return out


def test_mixed_tangent_ties_within_energy_error():
    """The mixed path's tangent rule on a 98,303-atom Tersoff vacancy-hop
    band (linear interpolation between relaxed endpoints, 11 images): energy
    differences up to 8e-6 eV per atom (twice the step energies' error
    bound) count as ties, so the nearly flat images beside the endpoints
    take the equal-weight tangent, the others their upwind branch.  The NEB
    coefficients the step used match the rule applied to the step's own
    energies and dots (1e-9 relative)."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2510_16721_gb300 as g
    g.build()
    R0, h0, R1, h1 = ci.diamond_vacancy_hop_relaxed((16, 24, 32))
    b = gpu_band(g, R0, h0, R1, h1, 11, g.tersoff_potential(), k=0.1, dt=0.05, dt_max=0.2,
                 maxstep=0.1, cell_filter=True, precision=g.MIXED)
    b.step(40)  # the images beside the endpoints have relaxed to nearly equal energies
    sc = b.image_scalars()
    ci_ = b.get_state()["ci"]
    etol = 8e-6 * len(R0)
    want = _coefs(sc["E"], sc["dots"], ci_, 0.1, etol)
    kinds = set()
    for i, (a, bb, wp, wm) in want.items():
        kinds.add((wp, wm) if wp in (0.0, 1.0) and wm in (0.0, 1.0) else "weighted")
        np.testing.assert_allclose(sc["coef"][i], [a, bb], rtol=1e-9, atol=1e-12, err_msg=str(i))
    # the flat ends tie, the slopes are upwind
    assert (1.0, 1.0) in kinds and ((1.0, 0.0) in kinds or (0.0, 1.0) in kinds), kinds
    b.destroy()
