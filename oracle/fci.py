"""Determinant full configuration interaction (test infrastructure only).

Exact ground states of small systems, used to pin the oracle's MPO and DMRG.  A
determinant is a 2n-bit integer over spin orbitals in Jordan-Wigner order (mode 2p + s,
alpha before beta on each site); |d> = prod_{modes P ascending, occupied} a+_P |vac>.
a+_P and a_P acting on |d> pick up (-1)^(number of occupied modes below P).  This is the
same state as the product of the local states of ``ops`` (site-major, alpha before beta),
so determinant and product-state bases coincide without extra signs.
"""
from itertools import combinations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .hamiltonian import spin_orbital_terms


def determinants(n, n_elec, two_sz):
    """Sorted int64 array of all determinants with N = n_elec, 2Sz = two_sz."""
    na, nb = (n_elec + two_sz) // 2, (n_elec - two_sz) // 2
    dets = []
    for ca in combinations(range(n), na):
        a = sum(1 << (2 * p) for p in ca)
        for cb in combinations(range(n), nb):
            dets.append(a | sum(1 << (2 * p + 1) for p in cb))
    return np.array(sorted(dets), dtype=np.int64)


def apply_string(dets, op_list):
    """Apply a product of elementary operators (operator order, rightmost acts first) to
    every determinant.  Returns (new determinants, signs, mask of nonvanishing results)."""
    d = dets.copy()
    sign = np.ones(len(d))
    ok = np.ones(len(d), dtype=bool)
    for mode, dagger in reversed(op_list):
        bit = np.int64(1) << np.int64(mode)
        occ = (d & bit) != 0
        ok &= ~occ if dagger else occ
        below = np.bitwise_count(d & (bit - 1))
        sign = np.where(below % 2 == 1, -sign, sign)
        d = d ^ bit
    return d, sign, ok


def operator_matrix(dets, terms, dets_out=None):
    """Sparse matrix <d'| sum_t c_t O_t |d> for terms [(c, op_list)]; rows index dets_out
    (defaults to dets), columns index dets."""
    if dets_out is None:
        dets_out = dets
    rows, cols, vals = [], [], []
    col_all = np.arange(len(dets))
    for coef, ol in terms:
        nd, sg, ok = apply_string(dets, ol)
        if not ok.any():
            continue
        nd, sg, c = nd[ok], sg[ok], col_all[ok]
        pos = np.searchsorted(dets_out, nd)
        pos = np.minimum(pos, len(dets_out) - 1)
        hit = dets_out[pos] == nd
        rows.append(pos[hit])
        cols.append(c[hit])
        vals.append(coef * sg[hit])
    if not rows:
        return sp.csr_matrix((len(dets_out), len(dets)))
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(len(dets_out), len(dets)))


def fci_hamiltonian(h1, eri, n_elec, two_sz, e_core=0.0):
    """(determinants, sparse H) of the ab initio Hamiltonian in the (N, Sz) sector."""
    n = h1.shape[0]
    dets = determinants(n, n_elec, two_sz)
    H = operator_matrix(dets, spin_orbital_terms(h1, eri))
    if e_core:
        H = H + e_core * sp.identity(len(dets), format="csr")
    return dets, H


def fci_ground_state(h1, eri, n_elec, two_sz, e_core=0.0, dense_limit=6000):
    """Lowest eigenpair: dense numpy.linalg.eigh up to dense_limit determinants, otherwise
    scipy's eigsh.  Returns (E0, vector, dets)."""
    dets, H = fci_hamiltonian(h1, eri, n_elec, two_sz, e_core)
    if len(dets) <= dense_limit:
        w, v = np.linalg.eigh(H.toarray())
        return float(w[0]), v[:, 0], dets
    w, v = spla.eigsh(H, k=1, which="SA", tol=1e-14)
    return float(w[0]), v[:, 0], dets


def two_electron_first_quantised(h1, eri):
    """H on the n^2 space of orbital pairs (p, q) for two distinguishable electrons:
    H[(pq),(rs)] = h_pr d_qs + d_pr h_qs + (pr|qs).  Its spectrum is the spectrum of the
    N = 2, Sz = 0 second-quantised Hamiltonian (singlets: symmetric pair functions;
    Sz = 0 triplets: antisymmetric ones)."""
    n = h1.shape[0]
    eye = np.eye(n)
    H = (np.einsum("pr,qs->pqrs", h1, eye) + np.einsum("pr,qs->pqrs", eye, h1)
         + np.einsum("prqs->pqrs", eri))
    return H.reshape(n * n, n * n)


def hubbard_holstein_ground_energy(n_sites=4, n_elec=4, n_ph=11, U=2.0, omega=0.25, g=0.5,
                                   t=1.0):
    """Ground energy of the Hubbard-Holstein chain of the paper's Listing 1: open chain of
    n_sites electronic sites with hopping -t, on-site U, one phonon mode (n_ph levels) per
    site with energy omega, coupled as g (n_i,alpha + n_i,beta)(b+_i + b_i); Sz = 0."""
    n = n_sites
    dets = determinants(n, n_elec, 0)
    hop = []
    for i in range(n - 1):
        for s in (0, 1):
            hop.append((-t, ((2 * i + s, True), (2 * (i + 1) + s, False))))
            hop.append((-t, ((2 * (i + 1) + s, True), (2 * i + s, False))))
    onsite = [(U, ((2 * i, True), (2 * i, False), (2 * i + 1, True), (2 * i + 1, False)))
              for i in range(n)]
    h_el = operator_matrix(dets, hop + onsite)
    dens = [operator_matrix(dets, [(1.0, ((2 * i, True), (2 * i, False))),
                                   (1.0, ((2 * i + 1, True), (2 * i + 1, False)))])
            for i in range(n)]
    bdag = sp.diags(np.sqrt(np.arange(1, n_ph)), -1, format="csr")
    num = sp.diags(np.arange(n_ph, dtype=float), 0, format="csr")
    eye_ph = sp.identity(n_ph, format="csr")

    def on_mode(op, i):
        mats = [eye_ph] * n
        mats[i] = op
        out = mats[0]
        for m in mats[1:]:
            out = sp.kron(out, m, format="csr")
        return out

    dim_ph = n_ph ** n
    eye_el = sp.identity(len(dets), format="csr")
    H = sp.kron(h_el, sp.identity(dim_ph, format="csr"), format="csr")
    ph = sum(omega * on_mode(num, i) for i in range(n))
    H = H + sp.kron(eye_el, ph, format="csr")
    for i in range(n):
        H = H + g * sp.kron(dens[i], on_mode(bdag + bdag.T, i), format="csr")
    w = spla.eigsh(H, k=1, which="SA", tol=1e-12)[0]
    return float(w[0])
