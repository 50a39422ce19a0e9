"""Pins of the CPU oracle against facts fixed outside it: the paper's printed numbers,
closed forms, textbook identities and brute force on tiny systems."""
import itertools
import json
import os

import numpy as np
import pytest

from oracle import dmrg, fci, mpo, ops
from synth import (ab_initio_integrals, hubbard_integrals, occupancies, random_mps,
                   sector_sizes)

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ------------------------------------------------------------------ local operators
def test_local_operators_are_listing_matrices():
    # Listing 1, Part A: basis [0, a, b, ab] and the c, d, C, D matrices, verbatim values
    with open(os.path.join(GOLDEN, "listing1_site_ops.json")) as f:
        ref = json.load(f)
    assert np.array_equal(ops.CRE_A, np.array(ref["c"]))
    assert np.array_equal(ops.ANN_A, np.array(ref["d"]))
    assert np.array_equal(ops.CRE_B, np.array(ref["C"]))
    assert np.array_equal(ops.ANN_B, np.array(ref["D"]))
    assert [tuple(q) for q in ref["basis_q"]] == list(ops.SITE_Q)


def test_local_anticommutators():
    e = [np.eye(4)[:, i] for i in range(4)]
    c = {(s, d): ops.elementary(s, d) for s in (0, 1) for d in (True, False)}
    for s, t in itertools.product((0, 1), repeat=2):
        ac = c[(s, False)] @ c[(t, True)] + c[(t, True)] @ c[(s, False)]
        assert np.array_equal(ac, np.eye(4) * (s == t))
        cc = c[(s, True)] @ c[(t, True)] + c[(t, True)] @ c[(s, True)]
        assert not cc.any()
    # |ab> = a+_a a+_b |0> and a+_b |a> = -|ab>
    assert np.array_equal(ops.CRE_A @ ops.CRE_B @ e[0], e[3])
    assert np.array_equal(ops.CRE_B @ e[1], -e[3])


def _dense_mode_op(n, mode, dagger):
    """Jordan-Wigner dense operator of one spin orbital on n sites (kron order)."""
    site, sigma = divmod(mode, 2)
    mats = [ops.PARITY] * site + [ops.elementary(sigma, dagger)] + [np.eye(4)] * (n - site - 1)
    out = mats[0]
    for m in mats[1:]:
        out = np.kron(out, m)
    return out


def test_fock_space_anticommutators_n3():
    n = 3
    a = [_dense_mode_op(n, m, False) for m in range(2 * n)]
    ad = [_dense_mode_op(n, m, True) for m in range(2 * n)]
    eye = np.eye(4 ** n)
    for p, q in itertools.product(range(2 * n), repeat=2):
        assert np.allclose(a[p] @ ad[q] + ad[q] @ a[p], eye * (p == q), atol=0)
        assert not (a[p] @ a[q] + a[q] @ a[p]).any()


# ------------------------------------------------------------------------- FCI
@pytest.mark.parametrize("L", [4, 6, 8])
def test_hubbard_free_band_energy(L):
    # U = 0, open chain, half filling, Sz = 0: E = 2 sum_{k=1}^{N/2} -2t cos(k pi / (L+1))
    h, eri = hubbard_integrals(L, 1.0, 0.0)
    e0, _, _ = fci.fci_ground_state(h, eri, L, 0)
    exact = 2 * sum(-2.0 * np.cos(k * np.pi / (L + 1)) for k in range(1, L // 2 + 1))
    assert abs(e0 - exact) < 1e-12


@pytest.mark.parametrize("U", [0.5, 4.0, 8.0])
def test_hubbard_dimer(U):
    # L = 2, N = 2, Sz = 0: E = (U - sqrt(U^2 + 16 t^2)) / 2
    h, eri = hubbard_integrals(2, 1.0, U)
    e0, _, _ = fci.fci_ground_state(h, eri, 2, 0)
    assert abs(e0 - (U - np.sqrt(U * U + 16.0)) / 2) < 1e-13


def test_two_electron_spectrum_first_quantised():
    h, eri = ab_initio_integrals(5, seed=11)
    _, H = fci.fci_hamiltonian(h, eri, 2, 0)
    w1 = np.sort(np.linalg.eigvalsh(H.toarray()))
    w2 = np.sort(np.linalg.eigvalsh(fci.two_electron_first_quantised(h, eri)))
    assert np.abs(w1 - w2).max() < 1e-12


def test_slater_condon_diagonal():
    n = 5
    h, eri = ab_initio_integrals(n, seed=12)
    dets, H = fci.fci_hamiltonian(h, eri, 5, 1)
    Hd = H.diagonal()
    for i, d in enumerate(dets[::7]):
        occ = [(m // 2, m % 2) for m in range(2 * n) if (int(d) >> m) & 1]
        e = sum(h[p, p] for p, _ in occ)
        for (p, s), (q, t) in itertools.product(occ, repeat=2):
            e += 0.5 * eri[p, p, q, q] - 0.5 * (s == t) * eri[p, q, q, p]
        assert abs(Hd[i * 7] - e) < 1e-12


def test_fci_dense_matches_sparse_n8():
    h, eri = ab_initio_integrals(8, seed=0)
    dets, H = fci.fci_hamiltonian(h, eri, 8, 0)
    assert len(dets) == 4900
    wd = np.linalg.eigvalsh(H.toarray())[0]
    import scipy.sparse.linalg as spla
    ws = spla.eigsh(H, k=1, which="SA", tol=1e-14)[0][0]
    assert abs(wd - ws) < 1e-12


def test_hubbard_holstein_listing_energy():
    # Listing 1 caption: the expected ground-state energy is -6.956893 (printed to 6 places)
    e0 = fci.hubbard_holstein_ground_energy(4, 4, 11, 2.0, 0.25, 0.5)
    assert abs(e0 - (-6.956893)) < 5e-7


# ------------------------------------------------------------------------- MPO
@pytest.mark.parametrize("kind", ["trie", "ncn"])
@pytest.mark.parametrize("n", [3, 4, 5])
def test_mpo_equals_fci_hamiltonian(kind, n):
    h, eri = ab_initio_integrals(n, seed=7)
    m = mpo.MPO(h, eri, e_core=0.3, kind=kind)
    Hd = m.dense()
    pos = {d: i for i, d in enumerate(mpo.product_state_dets(n))}
    for ne, tsz in [(n, 0), (n - 1, 1), (2, 0), (n + 1, -1)]:
        dets, H = fci.fci_hamiltonian(h, eri, ne, tsz, e_core=0.3)
        idx = np.array([pos[d] for d in dets])
        assert np.abs(Hd[np.ix_(idx, idx)] - H.toarray()).max() <= 1e-13


def test_mpo_dense_conserves_quantum_numbers():
    n = 4
    h, eri = ab_initio_integrals(n, seed=3)
    Hd = mpo.MPO(h, eri).dense()
    occ = [(0, 0), (1, 1), (1, -1), (2, 0)]
    q = []
    for idx in range(4 ** n):
        N = S = 0
        for j in range(n):
            s = (idx // 4 ** (n - 1 - j)) % 4
            N += occ[s][0]
            S += occ[s][1]
        q.append((N, S))
    q = np.array(q)
    nz = np.argwhere(np.abs(Hd) > 0)
    assert np.all(q[nz[:, 0]] == q[nz[:, 1]])


def test_ncn_normal_pairs_are_site_ordered_once():
    # A_ij = -A_ji (Sec. 2.3): a+_i a+_j and a+_j a+_i give ONE normal-operator channel
    h, eri = ab_initio_integrals(6, seed=5)
    m = mpo.MPO(h, eri)
    for k in range(m.n + 1):
        pairs = [key[1] for key in m.chans[k] if key not in ("I", "H") and key[0] == "L"
                 and sum(c for _, _, c in key[1]) == 2 and len(key[1]) == 2]
        sites = [tuple(s for s, _, _ in p) for p in pairs]
        assert all(a < b for a, b in sites)


# ------------------------------------------------------------------- H_eff / DMRG
def _small_problem(n=6, M=16, seed=21, kind="ncn", n_elec=None):
    n_elec = n if n_elec is None else n_elec
    h, eri = ab_initio_integrals(n, seed=seed)
    bonds = sector_sizes(n, n_elec, 0, M, occupancies(n, n_elec, "ab_initio"))
    sites = random_mps(bonds, seed=seed + 100)
    return h, eri, bonds, sites, mpo.MPO(h, eri, kind=kind)


def _basis_vectors(labels_A, As, side):
    """Block basis states as vectors in the block's Fock space (kron order)."""
    if side == "left":
        v = np.ones((1, 1))                        # (fock, states)
        for A in As:
            v = np.einsum("fl,lsr->fsr", v, A).reshape(-1, A.shape[2])
        return v
    v = np.ones((1, 1))                            # (states, fock)
    for A in reversed(As):
        v = np.einsum("lsr,rf->lsf", A, v).reshape(A.shape[0], -1)
    return v


def test_heff_matches_projected_hamiltonian():
    """Y = P^T H P psi with P built from the block basis states and H the dense FCI
    Hamiltonian over the full Fock space: the plain definition of the effective H."""
    n = 6
    h, eri, bonds, sites, m = _small_problem(n)
    d = dmrg.DMRG(m, bonds, sites)
    d.optimise(0, 1e-10, 30, 30)
    d.move_right(0, 16, 1e-14)
    d.optimise(1, 1e-10, 30, 30)
    d.move_right(1, 16, 1e-14)                     # window 2 now has a nontrivial left block
    i = 2
    Lv = _basis_vectors(None, d.A[:i], "left")     # (4^i, M_i)
    Rv = _basis_vectors(None, d.A[i + 2:], "right")  # (M_{i+2}, 4^(n-i-2))
    Hd = mpo.MPO(h, eri, kind="trie").dense()
    rng = np.random.default_rng(3)
    psi = rng.standard_normal(d.psi.shape) * (d.psi != 0)
    P = np.einsum("fl,st,rg->fsgltr", Lv, np.eye(16), Rv)   # rows (left, s1 s2, right)
    P = P.reshape(4 ** n, -1)
    y_ref = (P.T @ (Hd @ (P @ psi.reshape(-1))))
    # project out quantum-number-forbidden entries (the projector is exact on the allowed)
    y = d.heff(i).apply(psi)
    mask = (d.psi != 0).reshape(-1) | (y.reshape(-1) != 0)
    assert np.abs(y.reshape(-1) - y_ref).max() < 1e-12 * max(1.0, np.abs(y_ref).max())
    assert np.abs(y_ref[~mask]).max(initial=0.0) < 1e-12


def test_heff_hermitian_and_mpo_independent():
    h, eri, bonds, sites, m = _small_problem(7, 24, seed=31, n_elec=6)
    m_trie = mpo.MPO(h, eri, kind="trie")
    d1, d2 = dmrg.DMRG(m, bonds, sites), dmrg.DMRG(m_trie, bonds, sites)
    for d in (d1, d2):
        for i in range(3):
            d.optimise(i, 1e-10, 30, 30)
            d.move_right(i, 24, 1e-14)
    i = 3
    rng = np.random.default_rng(0)
    mask = d1.psi != 0
    x = rng.standard_normal(mask.shape) * mask
    yv = rng.standard_normal(mask.shape) * mask
    H1, H2 = d1.heff(i), d2.heff(i)
    hx, hy = H1.apply(x), H1.apply(yv)
    scale = np.linalg.norm(hx) * np.linalg.norm(yv)
    assert abs(np.vdot(yv, hx) - np.vdot(hy, x)) < 1e-13 * scale
    # the effective Hamiltonian does not depend on how the MPO is built (same MPS)
    np.testing.assert_allclose(H2.apply(x), hx, atol=1e-12 * np.abs(hx).max())
    np.testing.assert_allclose(H2.diag(), H1.diag(), atol=1e-12 * np.abs(hx).max())
    # the diagonal is the diagonal
    ml, mr = x.shape[0], x.shape[3]
    idx = [(a, s, t, b) for a in range(ml) for s in range(4) for t in range(4)
           for b in range(mr) if mask[a, s, t, b]]
    dg = H1.diag()
    for k in rng.choice(len(idx), 20, replace=False):
        e = np.zeros(mask.shape)
        e[idx[k]] = 1.0
        assert abs(H1.apply(e)[idx[k]] - dg[idx[k]]) < 1e-12


def test_davidson_matches_dense_eigh():
    h, eri, bonds, sites, m = _small_problem(6, 16, seed=41)
    d = dmrg.DMRG(m, bonds, sites)
    H = d.heff(0)
    mask = d.psi != 0
    idx = np.argwhere(mask)
    dense = np.zeros((len(idx), len(idx)))
    for c, j in enumerate(idx):
        e = np.zeros(mask.shape)
        e[tuple(j)] = 1.0
        dense[:, c] = H.apply(e)[tuple(idx.T)]
    w = np.linalg.eigvalsh(dense)[0]
    theta, _, _, rn2 = dmrg.davidson(H.apply, H.diag(), d.psi, 1e-12, 60, 60)
    assert abs(theta - w) < 1e-10


def test_dmrg_exact_bond_dimension_reaches_fci():
    n = 6
    h, eri = ab_initio_integrals(n, seed=51)
    M = 64  # >= 4^3 = every bond of n = 6 untruncated
    bonds = sector_sizes(n, n, 0, M, occupancies(n, n, "ab_initio"))
    sites = random_mps(bonds, seed=151)
    e_fci, _, _ = fci.fci_ground_state(h, eri, n, 0)
    es = dmrg.DMRG(mpo.MPO(h, eri), bonds, sites).run([M] * 3)
    assert abs(es[-1] - e_fci) < 1e-9


def test_dmrg_truncated_variational_and_monotone():
    n = 6
    h, eri = ab_initio_integrals(n, seed=52)
    M = 8
    bonds = sector_sizes(n, n, 0, M, occupancies(n, n, "ab_initio"))
    sites = random_mps(bonds, seed=152)
    e_fci, _, _ = fci.fci_ground_state(h, eri, n, 0)
    es = dmrg.DMRG(mpo.MPO(h, eri), bonds, sites).run([M] * 4)
    assert es[-1] >= e_fci - 1e-10
    assert all(b <= a + 1e-10 for a, b in zip(es, es[1:]))


def test_dmrg_hubbard_chain_free_limit():
    L = 6
    h, eri = hubbard_integrals(L, 1.0, 0.0)
    M = 64
    bonds = sector_sizes(L, L, 0, M, occupancies(L, L, "hubbard"))
    sites = random_mps(bonds, seed=7)
    es = dmrg.DMRG(mpo.MPO(h, eri), bonds, sites).run([M] * 4)
    exact = 2 * sum(-2.0 * np.cos(k * np.pi / (L + 1)) for k in range(1, L // 2 + 1))
    assert abs(es[-1] - exact) < 1e-8


# ------------------------------------------------------------------ synthetic inputs
def test_random_mps_is_right_canonical_and_normalised():
    n = 8
    bonds = sector_sizes(n, n, 0, 40, occupancies(n, n, "ab_initio"))
    sites = random_mps(bonds, seed=9)
    lab, A = dmrg.blocks_to_dense(bonds, sites)
    for k in range(1, n):
        B = A[k].reshape(A[k].shape[0], -1)
        assert np.abs(B @ B.T - np.eye(B.shape[0])).max() < 1e-12
    assert abs(np.sum(A[0] ** 2) - 1.0) < 1e-12
    for k, blocks in enumerate(sites):
        for (jl, s, jr) in blocks:
            ql, qr = bonds[k][jl], bonds[k + 1][jr]
            assert ql[0] + ops.SITE_Q[s][0] == qr[0] and ql[1] + ops.SITE_Q[s][1] == qr[1]


def test_graded_density_matrices_have_the_stated_spectrum():
    # the eigensolver benchmark's inputs: symmetric, positive semidefinite, eigenvalues
    # 10^(-16 i/(r-1)) for i < r = floor(0.7 m) + 1 and zero beyond, and seeded
    from synth import TRUNCATION_BATCH_DIMS, graded_density_matrices
    dims = [1, 2, 17, 64]
    mats = graded_density_matrices(dims, seed=5)
    again = graded_density_matrices(dims, seed=5)
    for m, a, b in zip(dims, mats, again):
        assert np.array_equal(a, b)
        assert np.array_equal(a, a.T)
        r = int(0.7 * m) + 1
        lam = np.zeros(m)
        lam[:r] = 10.0 ** (-16.0 * np.arange(r) / max(r - 1, 1))
        w = np.sort(np.linalg.eigvalsh(a))[::-1]
        assert np.abs(w - lam).max() < 1e-14
    assert len(TRUNCATION_BATCH_DIMS) == 43 and max(TRUNCATION_BATCH_DIMS) == 147
