"""Image-range sharding (paper_2510_16721_gb300.sharded) over world-size-2
gloo ranks on the CPU.

Each rank drives its range through the shard interface; here the range is
computed by the oracle (no GPU in this test), so what is exercised is the
sharded step itself: the halo exchange of the boundary images, the global
climbing image from an all-gather of the energies, and the FIRE sums added
over the ranks before one FIRE decision.  The sharded band must follow the
oracle's one-rank band step for step.  (On GPUs the range is the library's
shard; tests/test_gpu_sharded.py runs two of them against the one-band
path.)"""
import os

import numpy as np
import pytest

from _cases import lj_band_case, oracle_band

K, DT = 1.0, 0.01
N_IMAGES = 7
NSTEPS = 12


class OracleRange:
    """Images lo-1 .. hi of the whole band on the oracle, with the shard
    methods of the library's band; lo-1 and hi are ghosts."""

    def __init__(self, o, X, lo, hi, image_fn):
        self.o, self.image_fn = o, image_fn
        self.X = [np.array(x) for x in X[lo - 1:hi + 1]]
        self.E = [None] * len(self.X)
        self.F = [None] * len(self.X)
        self.fire = o.Fire(dt=DT, dt_max=10 * DT, maxstep=0.2)
        self.fneb = None
        for i in (0, len(self.X) - 1):  # the end images' energies (endpoints stay)
            self.E[i] = float(image_fn(self.X[i])[0])

    def shard_evaluate(self):
        for i in range(1, len(self.X) - 1):
            E, F, _ = self.image_fn(self.X[i])
            self.E[i], self.F[i] = float(E), F
        return np.array([e if e is not None else 0.0 for e in self.E])

    def shard_get_image(self, i):
        return self.X[i], self.E[i]

    def shard_set_ghost(self, side, X, e):
        i = 0 if side == 0 else len(self.X) - 1
        self.X[i], self.E[i] = np.array(X), float(e)

    def shard_project(self, ci_local):
        Xs = np.array([x.ravel() for x in self.X])
        Fs = np.array([np.zeros(Xs.shape[1]) if f is None else f.ravel() for f in self.F])
        Fn, _ = self.o.neb_forces(Xs, np.array(self.E, dtype=float), Fs, K, True, ci=ci_local)
        self.fneb = Fn[1:-1]
        v = self.fire.v if self.fire.v is not None else np.zeros_like(self.fneb)
        rows = self.fneb.reshape(-1, 3)
        return np.array([np.sum(self.fneb * v), np.sum(self.fneb * self.fneb), np.sum(v * v),
                         float(np.max(np.sum(rows * rows, axis=1)))])

    def shard_move(self, sums):
        dX = self.fire.step(self.fneb, sums=sums[:3])
        for i in range(1, len(self.X) - 1):
            self.X[i] = self.X[i] + dX[i - 1].reshape(self.X[i].shape)


class GlooComm:
    """The shard communicator over a gloo process group (torch.distributed)."""

    def __init__(self):
        import torch.distributed as dist
        from paper_2510_16721_gb300.sharded import TorchComm
        self.inner = TorchComm(dist)
        self.rank, self.size = self.inner.rank, self.inner.size

    def allgather(self, obj):
        return self.inner.allgather(obj)

    def exchange(self, sends):
        return self.inner.exchange(sends)


def _rank_main(rank, size, port, out):
    import traceback
    try:
        _rank_body(rank, size, port, out)
    except Exception:  # report instead of leaving the other rank waiting
        out.put((rank, traceback.format_exc()))


def _rank_body(rank, size, port, out):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
    import torch.distributed as dist
    import oracle as o
    from paper_2510_16721_gb300.sharded import ShardedBand
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=size)
    o.build()
    R0, h0, R1, h1 = lj_band_case(strain_seed=3)
    ref = oracle_band(o, o.LJ(), R0, h0, R1, h1, N_IMAGES, k=K, dt=DT, cell_filter=True)
    X0 = [x.copy() for x in ref.X]
    img = ref.image_fn
    comm = GlooComm()
    sb = ShardedBand(comm, None, None, N_IMAGES, None,
                     engine=lambda lo, hi: OracleRange(o, X0, lo, hi, img))
    res = []
    for step in range(NSTEPS):
        f = sb.compute()
        fo = ref.compute()
        sb.update()
        ref.update()
        idx, X = sb.images()
        d = max(np.max(np.abs(X[k] - ref.X[i])) for k, i in enumerate(idx))
        res.append((step, f, fo, sb.ci, ref.ci, d))
    out.put((rank, res))
    dist.destroy_process_group()


def test_two_rank_shards_follow_one_rank_band():
    import multiprocessing as mp
    import socket
    pytest.importorskip("torch")
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
    for rank in (0, 1):
        assert not isinstance(got[rank], str), got[rank]
    assert all(p.exitcode == 0 for p in procs)
    for rank in (0, 1):
        for step, f, fo, ci, cio, d in got[rank]:
            assert abs(f - fo) <= 1e-12 * max(1.0, fo), (rank, step, f, fo)
            assert ci == cio, (rank, step)
            assert d <= 1e-12, (rank, step, d)
