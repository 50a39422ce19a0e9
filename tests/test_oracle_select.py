"""Pins of the oracle's truncation rule (oracle.dmrg._select, left_split, right_split):
keep the M largest density-matrix eigenvalues over all sectors (Sec. 2.1.2 two-site
algorithm with density-matrix truncation), drop eigenvalues at or below cutoff * largest,
and order near-ties (chains of neighbours within 1e-14 * largest) by sector, then by index in
the sector.  Every expected value below is worked out by hand from the spectra written in
the test, not taken from the function."""
import numpy as np
import pytest

from oracle import dmrg


def test_select_keeps_exactly_the_m_largest():
    spectra = [[5.0, 3.0, 1.0], [4.0, 2.0], [6.0]]
    # sorted: 6 (s2), 5 (s0), 4 (s1), 3 (s0), 2 (s1), 1 (s0)
    assert dmrg._select(spectra, 1, 1e-14) == [0, 0, 1]
    assert dmrg._select(spectra, 3, 1e-14) == [1, 1, 1]
    assert dmrg._select(spectra, 4, 1e-14) == [2, 1, 1]
    assert dmrg._select(spectra, 6, 1e-14) == [3, 2, 1]
    assert dmrg._select(spectra, 100, 1e-14) == [3, 2, 1]
    assert sum(dmrg._select(spectra, 5, 1e-14)) == 5


def test_select_drops_eigenvalues_at_or_below_the_cutoff():
    # largest = 1.0: 1e-15 and 0 are <= 1e-14 * 1.0 and go; 2e-14 stays
    spectra = [[1.0, 1e-15, 0.0], [0.5, 2e-14]]
    assert dmrg._select(spectra, 10, 1e-14) == [1, 2]
    # a looser cutoff (1e-3 of the largest) also drops 2e-14 but keeps 0.5
    assert dmrg._select(spectra, 10, 1e-3) == [1, 1]
    # the cutoff is relative to the largest eigenvalue of all sectors
    assert dmrg._select([[1e-20], [3e-35]], 5, 1e-14) == [1, 0]
    assert dmrg._select([[0.0, 0.0]], 5, 1e-14) == [0]
    # exactly at the cutoff counts as below it
    assert dmrg._select([[1.0, 1e-14]], 5, 1e-14) == [1]
    assert dmrg._select([[2.0], [2e-14, 2.0000001e-14]], 5, 1e-14) == [1, 1]


def test_select_breaks_exact_ties_by_sector_then_index():
    # three equal largest values: sectors 0, 1, 2 in that order, then index order
    spectra = [[0.5, 0.2], [0.5, 0.1], [0.5]]
    assert dmrg._select(spectra, 1, 1e-14) == [1, 0, 0]
    assert dmrg._select(spectra, 2, 1e-14) == [1, 1, 0]
    assert dmrg._select(spectra, 3, 1e-14) == [1, 1, 1]
    # ties inside one sector: equal values keep their in-sector order (counts only)
    assert dmrg._select([[0.3, 0.3, 0.3], [0.3]], 2, 1e-14) == [2, 0]


def test_select_chains_near_ties_across_the_group():
    # a = 1, b = 1 - 0.8e-14, c = 1 - 1.6e-14: a-b and b-c are within 1e-14 * 1 but a-c is
    # not; chaining puts all three in one group, ordered by sector: c (0), b (1), a (2)
    a, b, c = 1.0, 1.0 - 0.8e-14, 1.0 - 1.6e-14
    spectra = [[c], [b], [a]]
    assert dmrg._select(spectra, 1, 1e-14) == [1, 0, 0]
    assert dmrg._select(spectra, 2, 1e-14) == [1, 1, 0]
    # a gap larger than the tolerance ends the group: d well below stays last
    d = 1.0 - 5e-14
    assert dmrg._select([[d], [c], [b], [a]], 1, 1e-14) == [0, 1, 0, 0]
    assert dmrg._select([[d], [c], [b], [a]], 3, 1e-14) == [0, 1, 1, 1]


def _one_state_left_block(weights):
    """Two-site psi with one left-block state (label (0, 0)): row (0, s1) forms its own
    sector q(s1), whose single density-matrix eigenvalue is the squared norm of row s1."""
    rng = np.random.default_rng(3)
    mr = 3
    psi = np.zeros((1, 4, 4, mr))
    for s1, w in enumerate(weights):
        v = rng.standard_normal(4 * mr)
        psi[0, s1] = (np.sqrt(w) * v / np.linalg.norm(v)).reshape(4, mr)
    return psi


@pytest.mark.parametrize("M,kept_rows,dw", [
    (4, [0, 1, 2, 3], 0.0),
    (2, [0, 1], 0.15 + 0.05),
    (1, [0], 0.3 + 0.15 + 0.05),
])
def test_left_split_keeps_the_heaviest_sectors_and_reports_the_discarded_weight(M, kept_rows, dw):
    weights = [0.5, 0.3, 0.15, 0.05]
    psi = _one_state_left_block(weights)
    lab_l = np.array([[0, 0]])
    A, C, lab, disc = dmrg.left_split(psi, lab_l, M)
    assert A.shape == (1, 4, len(kept_rows))
    # A picks exactly the kept rows (one unit entry each, sign free)
    sel = np.abs(A[0]).sum(axis=1)
    assert np.allclose(sel[kept_rows], 1.0) and np.allclose(np.delete(sel, kept_rows), 0.0)
    q = np.array([[0, 0], [1, 1], [1, -1], [2, 0]])
    assert sorted(map(tuple, lab)) == sorted(map(tuple, q[kept_rows]))
    assert abs(disc - dw) <= 1e-14
    # the kept weight plus the discarded weight is the norm (1)
    assert abs(np.sum(C * C) + disc - 1.0) <= 1e-14


def test_right_split_discarded_weight_mirrors_the_left_one():
    # transpose roles: one right-block state, columns (s2, r) form the sectors
    weights = [0.4, 0.35, 0.2, 0.05]
    rng = np.random.default_rng(4)
    psi = np.zeros((3, 4, 4, 1))
    for s2, w in enumerate(weights):
        v = rng.standard_normal(3 * 4)
        psi[:, :, s2, 0] = (np.sqrt(w) * v / np.linalg.norm(v)).reshape(3, 4)
    lab_r = np.array([[4, 0]])
    B, C, lab, disc = dmrg.right_split(psi, lab_r, 3)
    assert B.shape == (3, 4, 1)
    assert abs(disc - 0.05) <= 1e-14
    assert abs(np.sum(C * C) + disc - 1.0) <= 1e-14
