"""Image-range shards of the library (cfneb_shard_*) on one GPU: a band split
into two ranges, each driven by paper_2510_16721_gb300.sharded.ShardedBand in
its own thread (a thread communicator stands in for the ranks; the ranges
exchange images and sums on the host, no kernel waits on another), against
the same band stepped whole.  FP64: the states agree step for step."""
import threading

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


class ThreadComm:
    """allgather / exchange between threads of one process."""

    def __init__(self, shared, rank, size):
        self.s, self.rank, self.size = shared, rank, size

    def allgather(self, obj):
        self.s["slot"][self.rank] = obj
        self.s["bar"].wait()
        out = list(self.s["slot"])
        self.s["bar"].wait()
        return out

    def exchange(self, sends):
        for peer, arr in sends.items():
            self.s["mail"][(self.rank, peer)] = np.array(arr)
        self.s["bar"].wait()
        got = {peer: self.s["mail"].pop((peer, self.rank)) for peer in sends}
        self.s["bar"].wait()
        return got


def _cases(g, which):
    if which == "lj":
        R0, h0, R1, h1 = lj_band_case(strain_seed=3)
        return (R0, h0, R1, h1), 9, g.lj_potential(), dict(k=1.0, dt=0.01), None
    cfg = ci.tersoff_graphite_hexdiamond(reps=(2, 2, 2))
    R0, h0, R1, h1 = cfg["endpoints"]
    return (R0, h0, R1, h1), 9, g.tersoff_potential(), dict(k=0.1, dt=0.1), cfg["noise"]


@pytest.mark.parametrize("which", ["lj", "tersoff"])
def test_two_shards_follow_the_whole_band(g, which):
    from paper_2510_16721_gb300.sharded import ShardedBand
    (R0, h0, R1, h1), N, pot, kw, noise = _cases(g, which)
    nsteps = 10
    whole = gpu_band(g, R0, h0, R1, h1, N, pot, cell_filter=True, noise=noise, **kw)
    size = 2
    shared = {"bar": threading.Barrier(size), "slot": [None] * size, "mail": {}}
    out = [None] * size
    errors = []

    def run(rank):
        try:
            opt = g.default_options()
            opt.k_spring, opt.dt, opt.dt_max, opt.precision = kw["k"], kw["dt"], 10 * kw["dt"], 0
            sb = ShardedBand(ThreadComm(shared, rank, size), (R0, h0), (R1, h1), N, pot,
                             g.CellFilter(1, g.ROTFREE_B, 0.0, 0.0), opt, noise=noise)
            hist = []
            for _ in range(nsteps):
                f = sb.compute()
                sb.update()
                idx, X = sb.images()
                hist.append((f, sb.ci, idx, X))
            out[rank] = hist
        except Exception as e:  # noqa: BLE001 - reported below
            errors.append(repr(e))
            shared["bar"].abort()

    threads = [threading.Thread(target=run, args=(r,)) for r in range(size)]
    for t in threads:
        t.start()
    for t in threads:
        t.join(timeout=300)
    assert not errors, errors
    for step in range(nsteps):
        whole.step(1)
        st = whole.get_state()
        fmax = whole.get_path()["fmax"]
        for rank in range(size):
            f, ci_s, idx, X = out[rank][step]
            assert abs(f - fmax) <= 1e-10 * max(1.0, fmax), (step, rank, f, fmax)
            assert ci_s == st["ci"], (step, rank)
            for k, i in enumerate(idx):
                d = np.max(np.abs(X[k] - st["X"][i])) / max(1.0, np.max(np.abs(st["X"][i])))
                assert d <= 1e-10, (step, rank, i, d)
