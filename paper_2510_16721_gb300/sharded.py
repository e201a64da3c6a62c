"""Image-range sharding of one band over several processes (one GPU each).

The paper runs bands of ~100 images of 1e5 atoms (Sec. I, Sec. III); their
images split naturally into contiguous ranges, one per device.  Each rank
holds a band of its own (the C ABI's image-range shard): its interior images
are the rank's images of the whole band, its two end images are ghosts --
copies of the neighbouring ranks' boundary images, or the true endpoints at
the two ends of the band.  Per step:

  1. every rank evaluates its images (energies, forces, virials; the cell
     filter) -- cfneb_shard_evaluate;
  2. halo: each rank's first and last image go to its neighbours' ghosts
     (point-to-point, both directions);
  3. the climbing image is the argmax of all ranks' energies (lowest global
     index on ties), known to every rank after an all-gather;
  4. each rank forms f_NEB for its images (tangents and springs need the
     ghosts) and its FIRE sums -- cfneb_shard_project;
  5. the FIRE sums F_NEB.v, |F_NEB|^2, |v|^2 are added over the ranks in
     rank order, the largest row norm taken over them (all-gather, so every
     rank holds the same bits), and every rank takes the same FIRE decision
     and moves its images -- cfneb_shard_move.

The arithmetic of each step runs in the library's kernels; this module only
moves images, energies and four sums between ranks.  `comm` is any object
with `rank`, `size`, `allgather(obj) -> list` and `exchange(sends) ->
receives` (a dict {peer: array} in, the same out); TorchComm adapts
torch.distributed.
"""
import math

import numpy as np

from . import create_band, default_options


def image_ranges(n_images, size):
    """Contiguous ranges [lo, hi) of the interior images 1..n_images-2, one
    per rank, as even as possible (the first ranks take one more)."""
    m = n_images - 2
    if size < 1 or m < size:
        raise ValueError("need at least one interior image per rank")
    q, r = divmod(m, size)
    out, lo = [], 1
    for k in range(size):
        hi = lo + q + (1 if k < r else 0)
        out.append((lo, hi))
        lo = hi
    return out


class TorchComm:
    """torch.distributed as a shard communicator: host arrays over a gloo
    group (the shards' exchanges are host-side; on NCCL jobs a gloo group is
    made for them)."""

    def __init__(self, dist, group=None):
        import torch
        self.torch, self.dist = torch, dist
        if group is None and dist.get_backend() != "gloo":
            group = dist.new_group(backend="gloo")
        self.group = group
        self.rank = dist.get_rank()
        self.size = dist.get_world_size()

    def allgather(self, obj):
        out = [None] * self.size
        self.dist.all_gather_object(out, obj, group=self.group)
        return out

    def exchange(self, sends):
        """Send sends[peer] to each peer and receive an array of the same
        shape from each (point-to-point, posted together)."""
        t = self.torch
        ops, recv = [], {}
        for peer, arr in sends.items():
            a = t.from_numpy(np.ascontiguousarray(arr, dtype=np.float64))
            recv[peer] = t.empty_like(a)
            ops.append(self.dist.P2POp(self.dist.isend, a, peer, group=self.group))
            ops.append(self.dist.P2POp(self.dist.irecv, recv[peer], peer, group=self.group))
        if ops:
            for w in self.dist.batch_isend_irecv(ops):
                w.wait()
        return {p: v.numpy() for p, v in recv.items()}


class ShardedBand:
    """One band spread over comm.size ranks by contiguous image ranges.

    `engine` makes the rank's range: engine(X_range) -> an object with the
    Band shard methods (shard_evaluate, shard_get_image, shard_set_ghost,
    shard_project, shard_move).  The default builds it with the library:
    the whole band's initial path is made once (cfneb_create_band), the
    rank's slice of images [lo - 1, hi] is loaded into a band of its own
    (cfneb_set_state) and turned into a shard.
    """

    def __init__(self, comm, initial, final, n_images, potential, cell_filter=None,
                 options=None, noise=None, stream=None, engine=None):
        self.comm = comm
        self.n_images = n_images
        self.ranges = image_ranges(n_images, comm.size)
        self.lo, self.hi = self.ranges[comm.rank]
        self.steps = 0
        self.fmax = math.inf
        self.ci = -1
        if engine is None:
            opt = options if options is not None else default_options()
            full = create_band(initial, final, n_images, potential, cell_filter, opt,
                               stream=stream, noise=noise)
            X = full.get_state()["X"]
            full.destroy()
            m = self.hi - self.lo + 2
            keep_nmax = opt.n_max
            opt.n_max = m
            band = create_band(initial, final, m, potential, cell_filter, opt, stream=stream)
            opt.n_max = keep_nmax
            band.set_state(X[self.lo - 1:self.hi + 1])
            band.shard_enable()
            self.band = band
        else:
            self.band = engine(self.lo, self.hi)

    def _neighbours(self):
        r, s = self.comm.rank, self.comm.size
        return (r - 1 if r > 0 else None), (r + 1 if r < s - 1 else None)

    def compute(self):
        """Steps 1-4 of a step: evaluate, halo, climbing image, f_NEB and the
        global FIRE sums; returns the global fmax (before any move)."""
        b = self.band
        E = b.shard_evaluate()
        m = self.hi - self.lo
        left, right = self._neighbours()
        # halo: my first image to the left neighbour, my last to the right
        sends = {}
        if left is not None:
            X, e = b.shard_get_image(1)
            sends[left] = np.concatenate([X.ravel(), [e]])
        if right is not None:
            X, e = b.shard_get_image(m)
            sends[right] = np.concatenate([X.ravel(), [e]])
        got = self.comm.exchange(sends)
        if left is not None:
            v = got[left]
            b.shard_set_ghost(0, v[:-1].reshape(-1, 3), v[-1])
        if right is not None:
            v = got[right]
            b.shard_set_ghost(1, v[:-1].reshape(-1, 3), v[-1])
        # climbing image: argmax of the interior energies, lowest index on ties
        mine = [(float(E[k]), self.lo + k - 1) for k in range(1, m + 1)]
        best = None
        for part in self.comm.allgather(mine):
            for e, i in part:
                if best is None or e > best[0] or (e == best[0] and i < best[1]):
                    best = (e, i)
        self.ci = best[1]
        ci_local = self.ci - self.lo + 1 if self.lo <= self.ci < self.hi else -1
        sums = b.shard_project(ci_local)
        tot = np.zeros(4)
        for s in self.comm.allgather(list(map(float, sums))):  # rank order
            tot[:3] += s[:3]
            tot[3] = max(tot[3], s[3])
        self.sums = tot
        self.fmax = math.sqrt(tot[3])
        return self.fmax

    def update(self):
        """Step 5: the FIRE decision on the global sums and the move."""
        self.band.shard_move(self.sums)
        self.steps += 1

    def step(self, n=1):
        for _ in range(n):
            self.compute()
            self.update()

    def relax(self, fmax, max_steps):
        """Steps until the global fmax is below the tolerance (tested before
        each move); returns (steps done, converged)."""
        start = self.steps
        while self.steps - start < max_steps:
            if self.compute() < fmax:
                return self.steps - start, True
            self.update()
        return self.steps - start, self.compute() < fmax

    def images(self):
        """(global indices, X of this rank's images)."""
        X = np.array([self.band.shard_get_image(k)[0]
                      for k in range(1, self.hi - self.lo + 1)])
        return list(range(self.lo, self.hi)), X
