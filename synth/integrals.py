"""Seeded one- and two-electron integrals for the synthetic workloads.

Conventions: ``h`` is an n x n symmetric array h[p, q]; ``eri`` is the n^4 array of
chemist-notation integrals (pq|rs), 8-fold symmetric.  The Hamiltonian they define is
H = E_core + sum_pq h_pq sum_s a+_ps a_qs + 1/2 sum_pqrs (pq|rs) sum_st a+_ps a+_rt a_st a_qs;
this module only draws the numbers.
"""
import numpy as np


def _sym_normal(rng, n, sigma):
    """Symmetric matrix: upper triangle (with diagonal) drawn N(0, sigma), mirrored."""
    s = np.zeros((n, n))
    iu = np.triu_indices(n)
    s[iu] = rng.normal(0.0, sigma, size=len(iu[0]))
    return s + np.triu(s, 1).T


def ab_initio_integrals(n, seed, n_chol=12, sigma_h=0.1, sigma_b=0.05, decay=None):
    """Random ab initio integrals.

    h = S + diag(linspace(-2, 0, n)) with S symmetric, entries N(0, sigma_h).
    (pq|rs) = sum_k B^k_pq B^k_rs with B^k symmetric, entries N(0, sigma_b), optionally
    damped by exp(-|p-q|/decay).  h is drawn first, then B^0 .. B^{n_chol-1}, all from one
    ``numpy.random.default_rng(seed)`` stream.  The eri is positive semidefinite as a
    (pq),(rs) matrix and has the 8-fold permutational symmetry.
    """
    rng = np.random.default_rng(seed)
    h = _sym_normal(rng, n, sigma_h) + np.diag(np.linspace(-2.0, 0.0, n))
    damp = np.ones((n, n))
    if decay is not None:
        idx = np.arange(n)
        damp = np.exp(-np.abs(idx[:, None] - idx[None, :]) / float(decay))
    bs = np.empty((n_chol, n, n))
    for k in range(n_chol):
        bs[k] = _sym_normal(rng, n, sigma_b) * damp
    eri = np.einsum("kpq,krs->pqrs", bs, bs)
    return h, eri


def hubbard_integrals(L, t=1.0, U=4.0):
    """1D Hubbard chain with open boundaries written as integrals:
    h[i, i+1] = h[i+1, i] = -t and (ii|ii) = U, everything else zero."""
    h = np.zeros((L, L))
    for i in range(L - 1):
        h[i, i + 1] = h[i + 1, i] = -t
    eri = np.zeros((L, L, L, L))
    for i in range(L):
        eri[i, i, i, i] = U
    return h, eri


def config_integrals(name):
    """Integrals, electron count and 2*Sz for the named synthetic workloads.

    Returns (h, eri, n_elec, two_sz, kind) where kind is "ab_initio" or "hubbard".
    """
    if name == "abinitio_n8":        # n=8, N=8, 12 Cholesky vectors, seed 0
        h, eri = ab_initio_integrals(8, seed=0)
        return h, eri, 8, 0, "ab_initio"
    if name == "hubbard_L32":        # L=32, t=1, U=4, half filling
        h, eri = hubbard_integrals(32, 1.0, 4.0)
        return h, eri, 32, 0, "hubbard"
    if name == "abinitio_n36":       # n=36, N=36, 60 decaying Cholesky vectors, seed 2
        h, eri = ab_initio_integrals(36, seed=2, n_chol=60, decay=6.0)
        return h, eri, 36, 0, "ab_initio"
    if name == "abinitio_n24":       # n=24, N=24, seed 4
        h, eri = ab_initio_integrals(24, seed=4)
        return h, eri, 24, 0, "ab_initio"
    raise KeyError(name)


def batch_problem(j):
    """Problem j of the 64-problem batch (seed 1000 + j).

    Draws the type (Hubbard or ab initio, 50/50), then for Hubbard the length L in
    [12, 40] and U in [1, 8], for ab initio the orbital count n in [10, 24] (integrals from
    ``ab_initio_integrals`` with the same seed), then the bond dimension M in [100, 800].
    All at half filling with the lowest |Sz| (2Sz = 0, or 1 for an odd electron count).
    Returns a dict.
    """
    rng = np.random.default_rng(1000 + j)
    kind = "hubbard" if rng.random() < 0.5 else "ab_initio"
    if kind == "hubbard":
        L = int(rng.integers(12, 41))
        U = float(rng.uniform(1.0, 8.0))
        M = int(rng.integers(100, 801))
        h, eri = hubbard_integrals(L, 1.0, U)
        n = L
    else:
        n = int(rng.integers(10, 25))
        M = int(rng.integers(100, 801))
        h, eri = ab_initio_integrals(n, seed=1000 + j)
    return {"kind": kind, "n": n, "n_elec": n, "two_sz": n % 2, "M": M, "h": h, "eri": eri,
            "seed": 1000 + j}
