"""Seeded random initial MPS for the synthetic workloads, and its file format.

Sector sizes follow the occupancy-based initial quantum-number distribution of the
paper (Sec. 2.1.6, "Initial guesses" (ii)): each spin orbital p is occupied independently
with probability f_p, so the (N_alpha, N_beta) content of the left block at bond k is the
product of two Poisson-binomial distributions.  The site tensors are Gaussian random
numbers made into a right-canonical MPS by a per-sector LQ decomposition (a random
isometry), so both the oracle and the GPU library can start from the same file.

Bond k sits between sites k-1 and k.  Every bond sector is labelled by the quantum
number q = (N, 2Sz) of the LEFT block (sites 0..k-1).  Site k's tensor has blocks
(jl, s, jr) with q_left[jl] + q(s) = q_right[jr], each a dense row-major m_jl x m_jr array.
Local states s = 0, 1, 2, 3 are |0>, |alpha>, |beta>, |alpha beta> with (N, 2Sz) =
(0,0), (1,1), (1,-1), (2,0).
"""
import math
import numpy as np

SITE_Q = ((0, 0), (1, 1), (1, -1), (2, 0))


def occupancies(n, n_elec, kind, tau=2.0):
    """Per-spin occupation probabilities f_p.  Ab initio: a Fermi function centred at
    N/2 with width tau; Hubbard: 1/2 on every site."""
    if kind == "hubbard":
        return np.full(n, 0.5)
    p = np.arange(n, dtype=float)
    return 1.0 / (1.0 + np.exp((p + 0.5 - n_elec / 2.0) / tau))


def _poisson_binomial(f):
    """pmf of the number of successes of independent Bernoulli(f_i)."""
    pmf = np.zeros(len(f) + 1)
    pmf[0] = 1.0
    for x in f:
        pmf[1:] = pmf[1:] * (1.0 - x) + pmf[:-1] * x
        pmf[0] *= (1.0 - x)
    return pmf


def sector_sizes(n, n_elec, two_sz, M, f):
    """Sector dimensions for every bond: a list (bond 0..n) of dicts {(N, 2Sz): m}.

    m_q = max(1, round(M P(q))) over sectors with P(q) >= 1e-12 that are compatible with
    the remaining sites, capped by the Fock-space dimension of both blocks, scaled down
    until sum_q m_q <= M, then made consistent between neighbouring bonds
    (m_{k+1}(q) <= sum_s m_k(q - q_s) and m_k(q) <= sum_s m_{k+1}(q + q_s)).
    """
    na, nb = (n_elec + two_sz) // 2, (n_elec - two_sz) // 2
    bonds = [dict() for _ in range(n + 1)]
    bonds[0][(0, 0)] = 1
    bonds[n][(n_elec, two_sz)] = 1
    for k in range(1, n):
        pa = _poisson_binomial(f[:k])
        rng_a = range(max(0, na - (n - k)), min(k, na) + 1)
        rng_b = range(max(0, nb - (n - k)), min(k, nb) + 1)
        probs = {}
        for xa in rng_a:
            for xb in rng_b:
                probs[(xa, xb)] = pa[xa] * pa[xb]
        tot = sum(probs.values())
        cand = {}
        for (xa, xb), p in probs.items():
            p /= tot
            if p < 1e-12:
                continue
            cap = min(math.comb(k, xa) * math.comb(k, xb),
                      math.comb(n - k, na - xa) * math.comb(n - k, nb - xb))
            cand[(xa, xb)] = (p, min(cap, max(1, int(round(M * p)))))
        ms = {key: v[1] for key, v in cand.items()}
        while sum(ms.values()) > M:
            scale = M / float(sum(ms.values()))
            new = {key: max(1, int(math.floor(m * scale))) for key, m in ms.items()}
            if new == ms or sum(new.values()) > M and all(v == 1 for v in new.values()):
                # only single states left: drop the least probable sectors
                order = sorted(new, key=lambda kk: cand[kk][0])
                while sum(new.values()) > M:
                    new.pop(order.pop(0))
            ms = new
        for (xa, xb), m in ms.items():
            bonds[k][(xa + xb, xa - xb)] = m
    changed = True
    while changed:
        changed = False
        for k in range(1, n + 1):
            for q in list(bonds[k]):
                lim = sum(bonds[k - 1].get((q[0] - d[0], q[1] - d[1]), 0) for d in SITE_Q)
                if lim < bonds[k][q]:
                    changed = True
                    if lim == 0:
                        del bonds[k][q]
                    else:
                        bonds[k][q] = lim
        for k in range(n - 1, -1, -1):
            for q in list(bonds[k]):
                lim = sum(bonds[k + 1].get((q[0] + d[0], q[1] + d[1]), 0) for d in SITE_Q)
                if lim < bonds[k][q]:
                    changed = True
                    if lim == 0:
                        del bonds[k][q]
                    else:
                        bonds[k][q] = lim
    return [sorted((q[0], q[1], m) for q, m in b.items()) for b in bonds]


def random_mps(bonds, seed, center=0):
    """Random MPS on the given sectors, in canonical form with centre ``center``.

    Blocks are drawn N(0, 1) from ``default_rng(seed)`` site by site, in (jl, s) order.
    Sites n-1 .. center+1 are then made right-orthonormal by an LQ decomposition of each
    left sector's row block (the L factor is pushed into the site on the left), sites
    0 .. center-1 left-orthonormal by a QR decomposition of each right sector's column
    block (R pushed into the site on the right), and site ``center`` is scaled to unit
    norm.  Returns a list of dicts {(jl, s, jr): array}.
    """
    rng = np.random.default_rng(seed)
    n = len(bonds) - 1
    index = [{(b[0], b[1]): j for j, b in enumerate(bonds[k])} for k in range(n + 1)]
    sites = []
    for k in range(n):
        blocks = {}
        for jl, (N, tsz, ml) in enumerate(bonds[k]):
            for s, d in enumerate(SITE_Q):
                jr = index[k + 1].get((N + d[0], tsz + d[1]))
                if jr is None:
                    continue
                blocks[(jl, s, jr)] = rng.standard_normal((ml, bonds[k + 1][jr][2]))
        sites.append(blocks)
    for k in range(center):
        for jr in range(len(bonds[k + 1])):
            keys = sorted(key for key in sites[k] if key[2] == jr)
            x = np.vstack([sites[k][key] for key in keys])
            qmat, rmat = np.linalg.qr(x)
            row = 0
            for key in keys:
                h = sites[k][key].shape[0]
                sites[k][key] = np.ascontiguousarray(qmat[row:row + h])
                row += h
            for key in sites[k + 1]:
                if key[0] == jr:
                    sites[k + 1][key] = rmat @ sites[k + 1][key]
    for k in range(n - 1, center, -1):
        for jl in range(len(bonds[k])):
            keys = sorted(key for key in sites[k] if key[0] == jl)
            x = np.hstack([sites[k][key] for key in keys])
            qmat, rmat = np.linalg.qr(x.T)
            bt = qmat.T
            col = 0
            for key in keys:
                w = sites[k][key].shape[1]
                sites[k][key] = np.ascontiguousarray(bt[:, col:col + w])
                col += w
            lfac = rmat.T
            for key in sites[k - 1]:
                if key[2] == jl:
                    sites[k - 1][key] = sites[k - 1][key] @ lfac
    norm = math.sqrt(sum(float(np.sum(b * b)) for b in sites[center].values()))
    for key in sites[center]:
        sites[center][key] = sites[center][key] / norm
    return sites


def save_mps(path, bonds, sites):
    """Write an MPS as .npz: bond{k} [ns x 3] (N, 2Sz, m); site{k}_idx [nb x 3] (jl, s, jr)
    in lexicographic order; site{k}_data the row-major blocks concatenated in that order."""
    arrays = {"n": np.array(len(sites))}
    for k, b in enumerate(bonds):
        arrays["bond%d" % k] = np.array(b, dtype=np.int64).reshape(-1, 3)
    for k, blocks in enumerate(sites):
        keys = sorted(blocks)
        arrays["site%d_idx" % k] = np.array(keys, dtype=np.int64).reshape(-1, 3)
        arrays["site%d_data" % k] = (np.concatenate([blocks[key].ravel() for key in keys])
                                     if keys else np.zeros(0))
    np.savez(path, **arrays)


def load_mps(path):
    """Inverse of ``save_mps``: returns (bonds, sites)."""
    z = np.load(path)
    n = int(z["n"])
    bonds = [[tuple(int(v) for v in row) for row in z["bond%d" % k]] for k in range(n + 1)]
    sites = []
    for k in range(n):
        idx = z["site%d_idx" % k]
        data = z["site%d_data" % k]
        blocks, off = {}, 0
        for jl, s, jr in idx:
            ml, mr = bonds[k][jl][2], bonds[k + 1][jr][2]
            blocks[(int(jl), int(s), int(jr))] = data[off:off + ml * mr].reshape(ml, mr).copy()
            off += ml * mr
        sites.append(blocks)
    return bonds, sites
