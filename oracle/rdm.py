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

from . import ops
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


# ------------------------------------------------------------ MPS transfer matrices
def jordan_wigner_site_matrices(n, op_list):
    """Site-by-site 4 x 4 matrices of a product of elementary operators (operator order,
    rightmost acts first).  With the Jordan-Wigner order of ``ops`` (mode 2p + s, alpha
    before beta), a+_{ps} / a_{ps} is P on every site k < p, the local matrix of
    ``ops.elementary`` on site p (which carries the sign of the alpha mode of its own site)
    and the identity on sites k > p.  A product of such Kronecker products is the
    Kronecker product of the site-wise products, in operator order."""
    mats = [np.eye(4) for _ in range(n)]
    for mode, dagger in op_list:
        p, s = mode // 2, mode % 2
        for k in range(n):
            if k < p:
                f = ops.PARITY
            elif k == p:
                f = ops.elementary(s, dagger)
            else:
                continue
            mats[k] = mats[k] @ f
    return mats


def string_expectation(bonds, sites, op_list, norm2=None):
    """<psi| O |psi> / <psi|psi> for O a product of elementary operators, by plain
    transfer-matrix contraction of the block-sparse MPS (``synth`` format) from site 0 to
    site n-1.  The transfer object on bond k is a dict {(bra sector, ket sector): matrix}:
        E_{k+1}[jr', jr] = sum_{s', s} M_k[s', s] sum_{jl', jl} A_k[jl', s', jr']^T
                           E_k[jl', jl] A_k[jl, s, jr],
    M_k the site matrices of ``jordan_wigner_site_matrices``; the norm is the same
    contraction with every M_k = 1."""
    n = len(sites)
    mats = jordan_wigner_site_matrices(n, op_list)

    def contract(site_mats):
        E = {(0, 0): np.ones((1, 1))}
        for k in range(n):
            by_left = {}
            for (jl, s, jr), blk in sites[k].items():
                by_left.setdefault(jl, []).append((s, jr, blk))
            new = {}
            M = site_mats[k]
            for (jb, jk), e in E.items():
                for sk, jrk, ak in by_left.get(jk, ()):
                    t = e @ ak                                  # (m_jb, m_jrk)
                    for sb, jrb, ab in by_left.get(jb, ()):
                        x = M[sb, sk]
                        if x == 0.0:
                            continue
                        key = (jrb, jrk)
                        new[key] = new.get(key, 0.0) + x * (ab.T @ t)
            E = new
        return sum(float(v.sum()) for v in E.values())

    if norm2 is None:
        norm2 = contract([np.eye(4)] * n)
    return contract(mats) / norm2


def mps_norm2(bonds, sites):
    """<psi|psi> by the same contraction (the identity string)."""
    return string_expectation(bonds, sites, [], norm2=1.0)


def rdm_elements_mps(bonds, sites, gamma_pairs, Gamma_quads):
    """Selected elements of gamma and Gamma (definitions of Sec. 2.5.1 above) of a
    block-sparse MPS by ``string_expectation``, one spin-summed operator string at a time."""
    nrm = mps_norm2(bonds, sites)
    g = [sum(string_expectation(bonds, sites, [(2 * p + s, True), (2 * q + s, False)], nrm)
             for s in range(2)) for p, q in gamma_pairs]
    G = []
    for p, q, r, s in Gamma_quads:
        v = 0.0
        for a in range(2):
            for b in range(2):
                v += string_expectation(bonds, sites, [(2 * p + a, True), (2 * r + b, True),
                                                       (2 * s + b, False), (2 * q + a, False)],
                                        nrm)
        G.append(v)
    return np.array(g), np.array(G)
