"""Ab initio Hamiltonian as operator strings (test infrastructure only).

H = E_core + sum_{pq} h_pq sum_s a+_{ps} a_{qs}
          + 1/2 sum_{pqrs} (pq|rs) sum_{st} a+_{ps} a+_{rt} a_{st} a_{qs},

i.e. the standard second-quantised electronic Hamiltonian with chemist-notation
integrals that the paper's ab initio DMRG works with (Sec. 2.1.1; the paper states the
problem in words: integrals in an orthonormal orbital basis define the Hamiltonian whose
ground state DMRG finds).  The two-body operator order is a+_{ps} a+_{rt} a_{st} a_{qs}.

A "site-ordered string" is a tuple ((site, opkey, count), ...) with strictly increasing
sites; opkey identifies the 4x4 local matrix (``ops.op_key``) that is the product, in the
original order, of the ``count`` elementary operators acting on that site.  Moving the elementary
operators into site order costs the fermionic sign of the permutation.
"""
import numpy as np

from . import ops


def spin_orbital_terms(h1, eri, cutoff=0.0):
    """List of (coefficient, ((mode, dagger), ...)) in operator order; mode = 2*site + spin.

    Integrals with |value| <= cutoff are skipped (cutoff 0 keeps every nonzero)."""
    n = h1.shape[0]
    terms = []
    for p, q in zip(*np.nonzero(np.abs(h1) > cutoff)):
        for s in (0, 1):
            terms.append((float(h1[p, q]), ((2 * p + s, True), (2 * q + s, False))))
    for p, q, r, s in np.argwhere(np.abs(eri) > cutoff):
        v = 0.5 * float(eri[p, q, r, s])
        for a in (0, 1):
            for b in (0, 1):
                terms.append((v, ((2 * p + a, True), (2 * r + b, True),
                                  (2 * s + b, False), (2 * q + a, False))))
    assert all(0 <= m < 2 * n for _, t in terms for m, _ in t)
    return terms


def site_ordered(coef, op_list):
    """Rewrite coef * (product of elementary operators) as a site-ordered string.

    Returns (signed coefficient, string) or None when a local product vanishes."""
    sites = [m // 2 for m, _ in op_list]
    sign = 1.0
    for i in range(len(op_list)):
        for j in range(i + 1, len(op_list)):
            if sites[i] > sites[j]:
                sign = -sign
    order = sorted(range(len(op_list)), key=lambda i: sites[i])
    merged = []
    for i in order:
        mode, dagger = op_list[i]
        mat = ops.elementary(mode % 2, dagger)
        if merged and merged[-1][0] == sites[i]:
            merged[-1][1] = merged[-1][1] @ mat
            merged[-1][2] += 1
        else:
            merged.append([sites[i], mat.copy(), 1])
    if any(not mat.any() for _, mat, _ in merged):
        return None
    return sign * coef, tuple((site, ops.op_key(mat), cnt) for site, mat, cnt in merged)


def hamiltonian_strings(h1, eri, cutoff=0.0):
    """Dict {site-ordered string: coefficient} of the electronic Hamiltonian (no E_core);
    strings whose coefficients cancel exactly are dropped."""
    out = {}
    for coef, ol in spin_orbital_terms(h1, eri, cutoff):
        res = site_ordered(coef, ol)
        if res is None:
            continue
        c, key = res
        out[key] = out.get(key, 0.0) + c
    return {k: v for k, v in out.items() if v != 0.0}


def string_parity(key):
    """Fermion parity of a site-ordered string."""
    return sum(cnt for _, _, cnt in key) % 2


def string_dq(key):
    """(dN, d2Sz) of a site-ordered string."""
    dn = dz = 0
    for _, k, _ in key:
        d = ops.op_dq(ops.key_matrix(k))
        dn += d[0]
        dz += d[1]
    return dn, dz
