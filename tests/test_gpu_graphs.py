"""Steps run as CUDA graphs of eight captured steps (with a one-step graph
for the remainder).  Every captured step is the same launch sequence --
including the conditional list-rebuild node and, for many-body bands, the
finalize forked beside the force gather -- so a band stepped 24 steps at a
time must end bitwise where the same band stepped one step at a time ends
(the one-step graph), and where a band stepped 5 + 11 + 8 steps ends (both
graphs mixed)."""
import numpy as np
import pytest

import cfneb_inputs as ci
from _cases import gpu_band, lj_band_case

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def g():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2510_16721_gb300 as g
    g.build()
    return g


def _bands(g, which, precision):
    if which == "lj":
        R0, h0, R1, h1 = lj_band_case(strain_seed=3)
        mk = lambda: gpu_band(g, R0, h0, R1, h1, 7, g.lj_potential(), k=1.0, dt=0.01,
                              cell_filter=True, precision=precision, skin=0.05)
    else:
        cfg = ci.tersoff_graphite_hexdiamond(reps=(2, 2, 2))
        R0, h0, R1, h1 = cfg["endpoints"]
        mk = lambda: gpu_band(g, R0, h0, R1, h1, 9, g.tersoff_potential(), k=0.1, dt=0.1,
                              cell_filter=True, noise=cfg["noise"], precision=precision,
                              skin=0.02)
    return mk(), mk(), mk()


@pytest.mark.parametrize("which", ["lj", "tersoff"])
@pytest.mark.parametrize("precision", [0, 1])
def test_eight_step_graphs_equal_single_steps(g, which, precision):
    a, b, c = _bands(g, which, g.MIXED if precision else g.FP64)
    a.step(1)
    first = a.list_stats()[0]
    for _ in range(23):
        a.step(1)
    b.step(24)
    for n in (5, 11, 8):
        c.step(n)
    sa, sb, sc = a.get_state(), b.get_state(), c.get_state()
    for key in ("X", "F", "Fneb"):
        assert np.array_equal(sa[key], sb[key]), key
        assert np.array_equal(sa[key], sc[key]), key
    assert sa["ci"] == sb["ci"] == sc["ci"]
    # the small skins make some lists rebuild in later steps, inside graphs
    builds = a.list_stats()[0]
    assert builds == b.list_stats()[0] == c.list_stats()[0]
    assert builds > first
