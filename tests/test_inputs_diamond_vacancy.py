"""The relaxed diamond vacancy hop (Tersoff carbon) used by the converged
barrier tests and the benchmark's converged band: the stored 4 x 4 x 4
endpoints are force-free under the oracle, the two endpoints are mirror
images (equal energies), exactly one atom changes site (one bond length),
and a larger supercell built around the stored field keeps the residual
forces of the embedding small and every far atom on its ideal site."""
import numpy as np
import pytest

import cfneb_inputs as ci


def _min_image(d, h):
    s = d @ np.linalg.inv(h)
    return (s - np.round(s)) @ h


def test_stored_endpoints_are_relaxed_and_symmetric(oracle_mod):
    R0, h, R1, _ = ci.diamond_vacancy_hop_relaxed((4, 4, 4))
    assert len(R0) == 511
    pot = oracle_mod.Tersoff()
    E0, _, F0, _ = oracle_mod.energy_forces_virial(pot, R0, h)
    E1, _, F1, _ = oracle_mod.energy_forces_virial(pot, R1, h)
    assert np.max(np.linalg.norm(F0, axis=1)) < 1e-5
    assert np.max(np.linalg.norm(F1, axis=1)) < 1e-5
    assert abs(E0 - E1) < 1e-8
    # a vacancy costs energy against the perfect crystal (Tersoff: ~-7.37 eV/atom)
    Rp, hp = ci.diamond(ci.DIAMOND_A, 4, 4, 4)
    Ep, _, _, _ = oracle_mod.energy_forces_virial(pot, Rp, hp)
    assert 0.0 < E0 - Ep * 511 / 512 < 10.0


def test_one_atom_hops_one_bond():
    R0, h, R1, _ = ci.diamond_vacancy_hop_relaxed((4, 4, 4))
    d = np.linalg.norm(_min_image(R1 - R0, h), axis=1)
    hop = int(np.argmax(d))
    # one bond (1.544 A) plus the hopping atom's relaxation away from the
    # vacancy at each end (~0.2 A)
    assert 1.5 < d[hop] < 2.1
    assert np.max(np.delete(d, hop)) < 0.5       # the others relax around the vacancy


def test_embedding_in_a_larger_cell():
    R0s, hs, R1s, _ = ci.diamond_vacancy_hop_relaxed((4, 4, 4))
    R0, h, R1, _ = ci.diamond_vacancy_hop_relaxed((6, 6, 5))
    Ri, _ = ci.diamond(ci.DIAMOND_A, 6, 6, 5)
    Ri = Ri[1:]
    # atoms beyond the 4 x 4 x 4 box around the vacancy sit on their sites
    off = _min_image(Ri - ci.diamond(ci.DIAMOND_A, 6, 6, 5)[0][0], h)
    far = np.any(np.abs(off) > 2.0 * ci.DIAMOND_A + 1e-9, axis=1)
    assert far.sum() > 0
    assert np.array_equal(R0[far], Ri[far]) and np.array_equal(R1[far], Ri[far])
    # the same displacement field as the stored cell, atom by atom
    d_small = np.sort(np.linalg.norm(R0s - ci.diamond(ci.DIAMOND_A, 4, 4, 4)[0][1:], axis=1))
    d_big = np.sort(np.linalg.norm(R0 - Ri, axis=1))
    assert np.allclose(d_big[-len(d_small) // 2:], d_small[-len(d_small) // 2:], atol=1e-12)


def test_embedding_residual_forces_are_small(oracle_mod):
    R0, h, R1, _ = ci.diamond_vacancy_hop_relaxed((6, 6, 6))
    pot = oracle_mod.Tersoff()
    for R in (R0, R1):
        _, _, F, _ = oracle_mod.energy_forces_virial(pot, R, h)
        assert np.max(np.linalg.norm(F, axis=1)) < 0.06


def test_too_small_a_supercell_is_refused():
    with pytest.raises(ValueError):
        ci.diamond_vacancy_hop_relaxed((3, 4, 4))
