"""Pins of the oracle's state-averaged DMRG (Sec. 2.1.3 (i)) and its block Davidson solver
against dense diagonalisation, FCI spectra and the Poincare separation theorem."""
import numpy as np

from oracle import dmrg, fci, mpo
from synth import ab_initio_integrals, hubbard_integrals, occupancies, random_mps, sector_sizes


def _fci_lowest(h, eri, n_elec, k):
    _, H = fci.fci_hamiltonian(h, eri, n_elec, 0)
    H = H.toarray() if hasattr(H, "toarray") else np.asarray(H)
    return np.linalg.eigvalsh(H)[:k]


def _problem(n, M, seed, kind="ab_initio"):
    h, eri = hubbard_integrals(n, 1.0, 4.0) if kind == "hubbard" else ab_initio_integrals(n, seed=seed)
    bonds = sector_sizes(n, n, 0, M, occupancies(n, n, kind))
    sites = random_mps(bonds, seed=seed + 100)
    return h, eri, bonds, sites


def test_davidson_roots_match_dense_eigh():
    h, eri, bonds, sites = _problem(6, 16, 41)
    d = dmrg.DMRG(mpo.MPO(h, eri), bonds, sites)
    H = d.heff(0)
    mask = d.psi != 0
    idx = np.argwhere(mask)
    dense = np.zeros((len(idx), len(idx)))
    for c, j in enumerate(idx):
        e = np.zeros(mask.shape)
        e[tuple(j)] = 1.0
        dense[:, c] = H.apply(e)[tuple(idx.T)]
    w = np.linalg.eigvalsh(dense)[:4]
    # the second guess is zero: completed by the lowest-diagonal unit vector rule
    X0 = [d.psi, np.zeros_like(d.psi), np.random.default_rng(1).standard_normal(d.psi.shape) * mask,
          np.zeros_like(d.psi)]
    th, vecs, nmv, rn2 = dmrg.davidson_roots(H.apply, H.diag(), X0, 1e-12, 400, 40, allowed=mask)
    assert all(not (v * ~mask).any() for v in vecs)
    assert np.abs(np.array(th) - w).max() < 1e-10
    G = np.array([[np.vdot(a, b) for b in vecs] for a in vecs])
    assert np.abs(G - np.eye(4)).max() < 1e-10
    for t, v in zip(th, vecs):
        assert np.linalg.norm(H.apply(v) - t * v) ** 2 <= 1e-11


def test_one_root_is_ground_state_dmrg():
    h, eri, bonds, sites = _problem(6, 8, 52)
    e1 = dmrg.DMRG(mpo.MPO(h, eri), bonds, sites).run([8] * 3, max_iter=100, max_sub=40)
    ek = dmrg.StateAveragedDMRG(mpo.MPO(h, eri), bonds, sites, 1).run([8] * 3)
    assert np.abs(np.array(e1) - np.array([e[0] for e in ek])).max() < 1e-9


def test_exact_bond_dimension_gives_fci_spectrum():
    n, k = 6, 3
    h, eri, bonds, sites = _problem(n, 64, 51)
    lam = _fci_lowest(h, eri, n, k)
    es = dmrg.StateAveragedDMRG(mpo.MPO(h, eri), bonds, sites, k).run([64] * 3)
    assert np.abs(np.array(es[-1]) - lam).max() < 1e-8


def test_truncated_roots_are_upper_bounds():
    """Ritz values of H restricted to the MPS subspace bound the exact eigenvalues from
    above, root by root (Poincare separation); more states per bond lower them."""
    n, k = 8, 3
    h, eri, bonds, sites = _problem(n, 6, 61, kind="hubbard")
    lam = _fci_lowest(h, eri, n, k)
    sa = dmrg.StateAveragedDMRG(mpo.MPO(h, eri), bonds, sites, k)
    small = sa.run([12] * 2)[-1]
    big = sa.run([40] * 2)[-1]
    assert all(e >= l - 1e-10 for e, l in zip(small, lam))
    assert all(e >= l - 1e-10 for e, l in zip(big, lam))
    assert sum(big) < sum(small)
