"""Pins of the oracle's density matrices (Sec. 2.5.1) against closed forms, the energy
expression of Sec. 2.1.1, trace identities and finite differences of the FCI energy."""
import itertools

import numpy as np
import pytest

from oracle import dmrg, fci, mpo, rdm
from synth import ab_initio_integrals, hubbard_integrals, occupancies, random_mps, sector_sizes


def _energy(h, eri, e_core, gamma, Gamma):
    return e_core + np.sum(h * gamma) + 0.5 * np.sum(eri * Gamma)


def test_rdm_single_determinant_closed_form():
    # For a determinant with spin-orbital occupations n_ps, Wick's theorem gives
    # gamma_pq = d_pq (n_pa + n_pb) and
    # Gamma_pqrs = sum_st n_ps n_rt (d_pq d_rs - d_st d_ps d_rq).
    n = 4
    occ = [(1, 1), (1, 0), (0, 1), (0, 0)]
    d = sum((a << (2 * p)) | (b << (2 * p + 1)) for p, (a, b) in enumerate(occ))
    dets = np.array([d], dtype=np.int64)
    gamma, Gamma = rdm.rdm12(dets, np.ones(1), n)
    nocc = np.array(occ, dtype=float)
    assert np.array_equal(gamma, np.diag(nocc.sum(1)))
    ref = np.zeros((n, n, n, n))
    eye = np.eye(n)
    for s, t in itertools.product(range(2), repeat=2):
        ns, nt = nocc[:, s], nocc[:, t]
        ref += np.einsum("p,r,pq,rs->pqrs", ns, nt, eye, eye)
        if s == t:
            ref -= np.einsum("p,r,ps,rq->pqrs", ns, nt, eye, eye)
    assert np.array_equal(Gamma, ref)


def test_rdm_hubbard_dimer_free_limit():
    # U = 0, t = 1: both electrons in the bonding orbital (1, 1)/sqrt(2), gamma = all ones
    h, eri = hubbard_integrals(2, 1.0, 0.0)
    e, c, dets = fci.fci_ground_state(h, eri, 2, 0)
    assert abs(e + 2.0) < 1e-12
    gamma, Gamma = rdm.rdm12(dets, c, 2)
    assert np.abs(gamma - 1.0).max() < 1e-12
    # two electrons: sum_pr Gamma_pprr = N (N - 1) = 2, and every Gamma_pqrs = 1/2
    assert np.abs(Gamma - 0.5).max() < 1e-12


@pytest.mark.parametrize("n,n_elec,seed", [(5, 6, 3), (6, 6, 4)])
def test_rdm_energy_traces_and_symmetries(n, n_elec, seed):
    h, eri = ab_initio_integrals(n, seed=seed)
    e_core = 0.7
    e, c, dets = fci.fci_ground_state(h, eri, n_elec, 0, e_core)
    gamma, Gamma = rdm.rdm12(dets, c, n)
    assert abs(_energy(h, eri, e_core, gamma, Gamma) - e) < 1e-10
    assert abs(np.trace(gamma) - n_elec) < 1e-12
    assert abs(np.einsum("pprr->", Gamma) - n_elec * (n_elec - 1)) < 1e-11
    # sum_r Gamma_pqrr = (N - 1) gamma_pq
    assert np.abs(np.einsum("pqrr->pq", Gamma) - (n_elec - 1) * gamma).max() < 1e-11
    assert np.abs(gamma - gamma.T).max() < 1e-12
    assert np.abs(Gamma - Gamma.transpose(2, 3, 0, 1)).max() < 1e-12
    assert np.abs(Gamma - Gamma.transpose(1, 0, 3, 2)).max() < 1e-12


def test_rdm_finite_differences_of_fci_energy():
    # Hellmann-Feynman at the exact ground state: a symmetric perturbation of h_pq (and
    # h_qp) changes E by gamma_pq + gamma_qp; one of the 8 equivalent (pq|rs) by half the
    # sum of Gamma over the equivalent index orders.
    n, n_elec = 5, 4
    h, eri = ab_initio_integrals(n, seed=8)
    e0, c, dets = fci.fci_ground_state(h, eri, n_elec, 0)
    gamma, Gamma = rdm.rdm12(dets, c, n)
    eps = 1e-4

    def energy(hh, ee):
        return fci.fci_ground_state(hh, ee, n_elec, 0)[0]

    for p, q in [(0, 0), (1, 3), (4, 2)]:
        dh = np.zeros_like(h)
        dh[p, q] = dh[q, p] = 1.0
        fd = (energy(h + eps * dh, eri) - energy(h - eps * dh, eri)) / (2 * eps)
        assert abs(fd - np.sum(dh * gamma)) < 1e-7
    for idx in [(0, 1, 2, 3), (1, 1, 0, 4), (2, 2, 2, 2)]:
        de = np.zeros_like(eri)
        p, q, r, s = idx
        for a, b, c2, d in [(p, q, r, s), (q, p, r, s), (p, q, s, r), (q, p, s, r),
                            (r, s, p, q), (s, r, p, q), (r, s, q, p), (s, r, q, p)]:
            de[a, b, c2, d] = 1.0
        fd = (energy(h, eri + eps * de) - energy(h, eri - eps * de)) / (2 * eps)
        assert abs(fd - 0.5 * np.sum(de * Gamma)) < 1e-7


def test_mps_state_matches_oracle_heff_energy_and_norm():
    # The MPS -> determinant-amplitude map: the full weight lies in the (N, 2Sz) sector and
    # the FCI Rayleigh quotient equals the oracle's H_eff Rayleigh quotient of the same MPS.
    n = 6
    h, eri = ab_initio_integrals(n, seed=21)
    bonds = sector_sizes(n, n, 0, 12, occupancies(n, n, "ab_initio"))
    sites = random_mps(bonds, seed=22)
    dets, c = rdm.mps_state(bonds, sites, n, 0)
    assert abs(np.dot(c, c) - 1.0) < 1e-12
    _, H = fci.fci_hamiltonian(h, eri, n, 0)
    e_fci = c @ (H @ c)
    d = dmrg.DMRG(mpo.MPO(h, eri), bonds, sites)
    psi = d.psi
    e_heff = np.sum(psi * d.heff(0).apply(psi)) / np.sum(psi * psi)
    assert abs(e_fci - e_heff) < 1e-11
    gamma, Gamma = rdm.mps_rdm12(bonds, sites, n, 0)
    assert abs(_energy(h, eri, 0.0, gamma, Gamma) - e_fci) < 1e-11


@pytest.mark.parametrize("n,n_elec,two_sz,M,center,seed", [
    (5, 5, 1, 12, 0, 31),    # open shell, centre at site 0
    (6, 6, 0, 20, 0, 32),
    (6, 4, 0, 16, 2, 33),    # norm carried by an inner site
])
def test_transfer_matrix_rdm_matches_the_determinant_route(n, n_elec, two_sz, M, center, seed):
    # the single-string transfer-matrix contraction (used where the state is far too large
    # for the determinant basis) against the definition evaluated on the FCI-sized vector;
    # the MPS is scaled by 3 so that the division by the norm is exercised
    bonds = sector_sizes(n, n_elec, two_sz, M, occupancies(n, n_elec, "ab_initio"))
    sites = random_mps(bonds, seed=seed, center=center)
    sites = [{k: (3.0 * v if i == center else v) for k, v in blk.items()}
             for i, blk in enumerate(sites)]
    gamma, Gamma = rdm.mps_rdm12(bonds, sites, n_elec, two_sz)
    pairs = [(p, q) for p in range(n) for q in range(n)]
    rng = np.random.default_rng(seed)
    quads = [tuple(int(x) for x in rng.integers(0, n, 4)) for _ in range(40)]
    quads += [(0, 0, 1, 1), (1, 2, 2, 1), (n - 1, 0, 0, n - 1), (2, 2, 2, 2)]
    g, G = rdm.rdm_elements_mps(bonds, sites, pairs, quads)
    assert np.abs(g - np.array([gamma[p, q] for p, q in pairs])).max() <= 1e-12
    assert np.abs(G - np.array([Gamma[q4] for q4 in quads])).max() <= 1e-12
    assert abs(sum(g[p * n + p] for p in range(n)) - n_elec) <= 1e-12


def test_jordan_wigner_site_matrices_anticommute():
    # {a_i, a+_j} = delta_ij and {a_i, a_j} = 0 for the site-by-site representation, checked
    # on the dense Kronecker products of n = 3 sites (6 modes)
    n = 3

    def dense(op_list):
        mats = rdm.jordan_wigner_site_matrices(n, op_list)
        out = np.ones((1, 1))
        for m in mats:
            out = np.kron(out, m)
        return out

    eye = np.eye(4 ** n)
    for i in range(2 * n):
        for j in range(2 * n):
            ai, adj = dense([(i, False)]), dense([(j, True)])
            assert np.abs(ai @ adj + adj @ ai - (eye if i == j else 0.0)).max() == 0.0
            aj = dense([(j, False)])
            assert np.abs(ai @ aj + aj @ ai).max() == 0.0
            # a product is the product of the single-operator representations
            assert np.array_equal(dense([(i, False), (j, True)]), ai @ adj)
