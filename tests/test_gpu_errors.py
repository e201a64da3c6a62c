"""Error paths of the C ABI that the parity tests do not reach: each is
detected (on the host, or by the kernels' own checks) and surfaces as its
status code; none depends on an out-of-range access."""
import math

import numpy as np
import pytest

import cfneb_inputs as ci
from _cases import gpu_band

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def g():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2510_16721_gb300 as g
    g.build()
    return g


def test_nonfinite_coordinates_are_rejected(g):
    R0, h0, R1, h1 = ci.lj_vacancy_hop()
    R1 = R1.copy()
    R1[3, 1] = math.nan
    with pytest.raises(g.CfnebError) as e:
        gpu_band(g, R0, h0, R1, h1, 5, g.lj_potential(), k=1.0, dt=0.01)
    assert e.value.status == g.ERR_INVALID_ARG
    h = h0.copy()
    h[2, 2] = math.inf
    with pytest.raises(g.CfnebError) as e:
        g.evaluate([(R0, h)], g.lj_potential(), g.FP64)
    assert e.value.status == g.ERR_INVALID_ARG


def test_neighbour_capacity_overflow(g):
    """A carbon cloud at 0.5 atoms/A^3 has ~24 atoms within R + D + skin of
    each atom: more than the list holds; the list kernel caps its writes and
    reports the overflow."""
    rng = np.random.default_rng(11)
    h = np.eye(3) * 5.0
    R = rng.uniform(0.0, 5.0, size=(64, 3))
    with pytest.raises(g.CfnebError) as e:
        g.evaluate([(R, h)], g.tersoff_potential(), g.MIXED)
    assert e.value.status == g.ERR_NBR_OVERFLOW


def test_reflected_end_cell_is_not_spd_for_the_deformation_gradient(g):
    """With D itself as the lattice coordinate, an end cell of the opposite
    handedness gives det D < 0: the map-back reports it."""
    R0, h0, R1, h1 = ci.lj_vacancy_hop()
    h1 = h1 @ np.diag([1.0, 1.0, -1.0])
    R1 = (R1 @ np.linalg.inv(h0)) @ h1
    with pytest.raises(g.CfnebError) as e:
        gpu_band(g, R0, h0, R1, h1, 5, g.lj_potential(), k=1.0, dt=0.01, variant=1)
    assert e.value.status == g.ERR_NOT_SPD
