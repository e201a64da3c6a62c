"""The graphite -> hexagonal-diamond endpoints at any tiling describe the same
per-cell transformation: every tile of the final structure carries the
displacement of the 8-atom cell, so the linearly interpolated band of an
n1 x n2 x n3 tiling has exactly n1 n2 n3 times the 8-atom band's energies.
(A matching taken after tiling sends atoms whose target wrapped across the
8-atom cell boundary to the wrong periodic image: the 1 x 2 x 1 band then
starts at hundreds of eV per cell.)"""
import numpy as np
import pytest

import cfneb_inputs as ci


@pytest.mark.parametrize("reps", [(1, 2, 1), (2, 2, 1), (1, 1, 2)])
def test_tiled_displacements_repeat_the_cell(reps):
    R0c, h0c, R1c, h1c = ci.graphite_hexdiamond_path((1, 1, 1))
    R0, h0, R1, h1 = ci.graphite_hexdiamond_path(reps)
    # fractional displacement of every atom, in its own tile's cell units
    dc = R1c @ np.linalg.inv(h1c) - R0c @ np.linalg.inv(h0c)
    d = (R1 @ np.linalg.inv(h1) - R0 @ np.linalg.inv(h0)) * np.array(reps)
    ncell = int(np.prod(reps))
    assert np.allclose(d.reshape(ncell, 8, 3), dc[None], atol=1e-12)
    # no atom moves more than one bond length in the initial cell's metric
    assert np.max(np.linalg.norm(dc @ h0c, axis=1)) < 2.2


def test_tiled_band_energies_scale_with_cells(oracle_mod):
    pot = oracle_mod.Tersoff()
    E = {}
    for reps in [(1, 1, 1), (1, 2, 1)]:
        R0, h0, R1, h1 = ci.graphite_hexdiamond_path(reps)
        b = oracle_mod.make_band(pot, R0, h0, R1, h1, 5)
        E[reps] = np.array([b.image_fn(x)[0] for x in b.X])
    assert np.allclose(E[(1, 2, 1)], 2.0 * E[(1, 1, 1)], rtol=1e-11, atol=1e-9)
    # the interpolated band stays within a few eV per 8-atom cell
    assert np.max(E[(1, 1, 1)] - E[(1, 1, 1)][0]) < 10.0
