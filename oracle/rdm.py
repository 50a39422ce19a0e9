"""Spin-traced one- and two-particle density matrices (test infrastructure only).

Sec. 2.5.1 lists N-particle density matrices among the quantities extracted from an MPS;
with the ab initio Hamiltonian of Sec. 2.1.1,
    E = e_core + sum_pq h_pq gamma_pq + 1/2 sum_pqrs (pq|rs) Gamma_pqrs,
    gamma_pq     = sum_s  <a+_ps a_qs>,
    Gamma_pqrs   = sum_st <a+_ps a+_rt a_st a_qs>,
so gamma and Gamma / 2 are the derivatives of E with respect to the integral arrays at a
fixed state.  Everything here works in the determinant basis of ``fci`` (Jordan-Wigner
order: mode 2p + s, alpha before beta), by the definition, one operator string at a time.
"""
import numpy as np

from .dmrg import blocks_to_dense
from .fci import apply_string, determinants
from .mpo import product_state_dets


def expectation(dets, c, op_list):
    """<c| O |c> for O a product of elementary operators (``fci.apply_string`` order);
    c indexed like the sorted determinant array dets."""
    nd, sg, ok = apply_string(dets, op_list)
    if not ok.any():
        return 0.0
    nd, sg, src = nd[ok], sg[ok], np.nonzero(ok)[0]
    pos = np.minimum(np.searchsorted(dets, nd), len(dets) - 1)
    hit = dets[pos] == nd
    return float(np.sum(c[pos[hit]] * sg[hit] * c[src[hit]]))


def rdm12(dets, c, n):
    """(gamma [n, n], Gamma [n, n, n, n]) of the normalised state c (Sec. 2.5.1)."""
    c = np.asarray(c, dtype=np.float64)
    c = c / np.linalg.norm(c)
    gamma = np.zeros((n, n))
    Gamma = np.zeros((n, n, n, n))
    for p in range(n):
        for q in range(n):
            gamma[p, q] = sum(expectation(dets, c, [(2 * p + s, True), (2 * q + s, False)])
                              for s in range(2))
    for p in range(n):
        for q in range(n):
            for r in range(n):
                for s in range(n):
                    v = 0.0
                    for a in range(2):
                        for b in range(2):
                            v += expectation(dets, c, [(2 * p + a, True), (2 * r + b, True),
                                                       (2 * s + b, False), (2 * q + a, False)])
                    Gamma[p, q, r, s] = v
    return gamma, Gamma


def mps_state(bonds, sites, n_elec, two_sz):
    """Amplitudes of a block-sparse MPS (``synth`` format) on the determinants of the
    (N, 2Sz) sector: contract the dense site tensors into the 4^n product-state vector
    (site 0 most significant) and read it at each determinant (the product-state and
    determinant bases coincide, ``fci``)."""
    _, A = blocks_to_dense(bonds, sites)
    v = np.ones((1, 1))
    for a in A:
        v = (v @ a.reshape(a.shape[0], -1)).reshape(-1, a.shape[2])
    v = v[:, 0]
    n = len(sites)
    dets = determinants(n, n_elec, two_sz)
    order = product_state_dets(n)          # determinant of each product-state index
    by_det = np.argsort(order)
    idx = by_det[np.searchsorted(order[by_det], dets)]
    return dets, v[idx]


def mps_rdm12(bonds, sites, n_elec, two_sz):
    dets, c = mps_state(bonds, sites, n_elec, two_sz)
    return rdm12(dets, c, len(sites))
