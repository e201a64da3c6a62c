"""How far two FP64 runs of the same band drift apart when only the order of
their sums differs: the oracle against itself with the atoms listed in
another order (every force, energy, virial and NEB dot product then adds the
same terms in another order).  On the adaptive LJ band of the GPU parity
test (cell filter on, strained end cell, 120 FIRE steps with two insertions)
the two runs stay within ~1e-13 of each other: summation order alone moves
this band's trajectory by no more than that."""
import numpy as np

from _cases import lj_band_case, oracle_band


def _runs(o, nsteps, perm):
    R0, h0, R1, h1 = lj_band_case(strain_seed=3)
    kw = dict(k=1.0, dt=0.01, cell_filter=True, adaptive=True, n_min=4, n_max=8,
              alpha_ins=1.0)
    a = oracle_band(o, o.LJ(), R0, h0, R1, h1, 6, **kw)
    b = oracle_band(o, o.LJ(), R0[perm], h0, R1[perm], h1, 6, **kw)
    a.step(nsteps)
    b.step(nsteps)
    n = len(R0)
    rows = np.concatenate([perm, np.arange(n, n + 3)])
    d = max(np.max(np.abs(xa - xb[np.argsort(rows)])) / max(1.0, np.max(np.abs(xa)))
            for xa, xb in zip(a.X, b.X))
    return a, b, d


def test_sum_order_drift_stays_at_rounding_level(oracle_mod):
    perm = np.random.default_rng(11).permutation(31)
    a, b, d = _runs(oracle_mod, 120, perm)
    assert a.N == b.N == 8 and [e[0] for e in a.events] == [e[0] for e in b.events]
    assert d < 1e-12, d
