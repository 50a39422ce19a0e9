"""Seeded density-matrix-like symmetric matrices for the batched eigensolver.

Each matrix is Q diag(lam) Q^T with Q a random orthogonal matrix (QR of a Gaussian
matrix) and a graded spectrum: lam_i = 10^(-decades * i / (r - 1)) for i < r =
floor(rank_frac * m) + 1, zero beyond -- the shape of a DMRG reduced density matrix
sector (eigenvalues falling off over many decades, rank-deficient).  Inputs only: no
eigensolver arithmetic here.
"""
import numpy as np

# one truncation step of the Hubbard L = 32, M = 500 sweep (its largest during bond growth):
# 43 sectors, dims 147, 116, 110, 104 and 39 more evenly spaced from 100 down to 2
TRUNCATION_BATCH_DIMS = [147, 116, 110, 104] + [int(x) for x in np.linspace(100, 2, 39)]


def graded_density_matrices(dims, seed, rank_frac=0.7, decades=16.0):
    rng = np.random.default_rng(seed)
    mats = []
    for m in dims:
        q, _ = np.linalg.qr(rng.standard_normal((m, m)))
        r = int(rank_frac * m) + 1
        lam = np.zeros(m)
        lam[:r] = 10.0 ** (-decades * np.arange(r) / max(r - 1, 1))
        a = (q * lam) @ q.T
        mats.append(0.5 * (a + a.T))
    return mats
