"""The allocation-free entry point, cfneb_lj_evaluate_noalloc.

It exists for callers that cannot allocate device memory (a process whose
allocator owns all of the device memory, a service that must not allocate
while serving): the caller hands in device buffers, the library works in one
static device array.  These tests call it through the C ABI with device
buffers owned by the test and check its output against cfneb_evaluate (the
allocating entry point) at the FP64 tolerance of the other parity tests,
on two calls in a row with different structures, so that the second call
runs on the scratch the first one left behind, and against the FP64 oracle.
"""
import numpy as np
import pytest

from _cases import lj_structures

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2510_16721_gb300 as g
    g.build()
    return torch, g


def _noalloc(torch, g, R, h):
    n = len(R)
    pos = torch.tensor(np.ascontiguousarray(R), dtype=torch.float64, device="cuda")
    e = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
    f = torch.full((n, 3), float("nan"), dtype=torch.float64, device="cuda")
    v = torch.full((9,), float("nan"), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    st = g.lj_evaluate_noalloc(pos.data_ptr(), n, h, 1.0, 1.0, 2.5, 1, e.data_ptr(),
                               f.data_ptr(), v.data_ptr(), stream=stream)
    assert st == g.OK, g.status_string(st)
    torch.cuda.synchronize()
    return float(e.cpu().item()), f.cpu().numpy(), v.cpu().numpy().reshape(3, 3)


def _rel(a, b):
    return np.max(np.abs(a - b)) / max(1.0, np.max(np.abs(b)))


def test_noalloc_matches_evaluate_on_two_calls(env):
    torch, g = env
    s = lj_structures()
    cases = [s["fcc2916"], s["vacancy31"]]   # large first, then small on the same scratch
    got = [_noalloc(torch, g, R, h) for (R, h) in cases]
    for (R, h), (E, F, V) in zip(cases, got):
        Er, Fr, Vr = g.evaluate([(R, h)], g.lj_potential(), g.FP64)
        assert abs(E - Er[0]) <= 1e-10 * abs(Er[0])
        assert _rel(F, Fr[0]) <= 1e-10
        assert _rel(V, Vr[0]) <= 1e-10


def test_noalloc_matches_oracle(env, oracle_mod):
    torch, g = env
    R, h = lj_structures()["triclinic240"]
    E, F, V = _noalloc(torch, g, R, h)
    e, Fo, Vo = oracle_mod.LJ(1.0, 1.0, 2.5, True).evaluate(R, h)
    assert abs(E - np.sum(e)) <= 1e-10 * abs(np.sum(e))
    assert _rel(F, Fo) <= 1e-10
    assert _rel(V, Vo) <= 1e-10


def test_noalloc_rejects_oversized_input(env):
    torch, g = env
    n = g.NOALLOC_MAX_ATOMS + 1
    h = np.eye(3) * 100.0
    pos = torch.zeros((n, 3), dtype=torch.float64, device="cuda")
    st = g.lj_evaluate_noalloc(pos.data_ptr(), n, h, 1.0, 1.0, 2.5, 1, 0, 0, 0)
    assert st == g.ERR_INVALID_ARG
