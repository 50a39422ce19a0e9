"""Exact MPOs of a sum of operator strings (test infrastructure only).

The paper builds MPOs automatically from a symbolic list of operator strings (Sec. 2.3,
"General MPO construction for Hamiltonians") and, for ab initio Hamiltonians, arranges
the renormalized operators into normal and complementary sets, switching from the
normal/complementary (NC) to the complementary/normal (CN) partition at the middle site
(the symbolic MPO construction of Sec. 2.3).  Two constructions are written here:

``kind="trie"``  the plainest exact MPO: the channels on bond k (between sites k-1 and k)
    are "I" (nothing of the term applied yet), "H" (term complete) and the prefix (the
    part of a term on sites < k) of every term that continues to the right.  A term's
    coefficient is attached at its last site.  Bond dimension O(n^3) for ab initio H.

``kind="ncn"``  the same strings, but a term whose left part holds at least three
    elementary operators (NC bonds, k <= n // 2), or whose right part holds at most two
    (CN bonds, k > n // 2), is carried on a channel keyed by its RIGHT part: the left
    side then holds the coefficient-weighted sum of left parts (a complementary
    operator).  Every other term is keyed by its left part (a normal operator).  Bond
    dimension O(n^2).

Channel keys: "I", "H", ("L", prefix) and ("R", suffix).  W[k][(w, w')] is the 4x4 local
operator on site k that maps channel w on bond k to channel w' on bond k+1.

Fermion convention: each channel w carries the parity p(w) of its left part.  Acting with
(left part) x (site op) on |l>|s> costs (-1)^{p(site op) n(l)}, n(l) the particle number of
the left ket; the dense Jordan-Wigner form of W_k[w, w'] is W_k[w, w'] P^{p(w')} with
P = diag(1, -1, -1, 1).
"""
import numpy as np

from . import ops
from .hamiltonian import hamiltonian_strings, string_parity, string_dq


def _ncn_key(term, k, n):
    """Channel of a term on bond k for the NC (k <= n//2) / CN (k > n//2) rule."""
    n_left = sum(c for s, _, c in term if s < k)
    n_right = sum(c for s, _, c in term if s >= k)
    if n_left == 0:
        return "I"
    if n_right == 0:
        return "H"
    left_keyed = n_left <= 2 if k <= n // 2 else n_right >= 3
    if left_keyed:
        return ("L", tuple(e for e in term if e[0] < k))
    return ("R", tuple(e for e in term if e[0] >= k))


def _trie_key(term, k, n):
    if all(s >= k for s, _, _ in term):
        return "I"
    if all(s < k for s, _, _ in term):
        return "H"
    return ("L", tuple(e for e in term if e[0] < k))


class MPO:
    """chans[k]: dict key -> index on bond k; W[k]: dict (w, w') -> 4x4 matrix;
    parity[k][w], dq[k][w]: fermion parity and (dN, d2Sz) of the left part of channel w."""

    def __init__(self, h1, eri, e_core=0.0, cutoff=0.0, kind="ncn", strings=None):
        if strings is None:
            strings = hamiltonian_strings(h1, eri, cutoff)
        n = h1.shape[0]
        self.n = n
        self.kind = kind
        keyf = _ncn_key if kind == "ncn" else _trie_key
        self.chans = [dict() for _ in range(n + 1)]
        self.W = [dict() for _ in range(n)]
        eye = ops.IDENT

        def chan(k, key):
            d = self.chans[k]
            if key not in d:
                d[key] = len(d)
            return d[key]

        for k in range(n):
            chan(k, "I")
        for k in range(1, n + 1):
            chan(k, "H")
        for k in range(n - 1):
            self.W[k][(chan(k, "I"), chan(k + 1, "I"))] = eye.copy()
        for k in range(1, n):
            self.W[k][(chan(k, "H"), chan(k + 1, "H"))] = eye.copy()
        if e_core:
            self.W[0][(0, chan(1, "H"))] = e_core * eye
        for term, coef in strings.items():
            local = {s: o for s, o, _ in term}
            first, last = term[0][0], term[-1][0]
            for k in range(first, last + 1):
                src_key, dst_key = keyf(term, k, n), keyf(term, k + 1, n)
                src, dst = chan(k, src_key), chan(k + 1, dst_key)
                mat = ops.key_matrix(local[k]) if k in local else eye
                src_plain = src_key == "I" or src_key[0] == "L"
                dst_plain = dst_key != "H" and dst_key[0] == "L"
                if src_plain and not dst_plain:
                    # the coefficient enters here, summed over every term using this edge
                    self.W[k][(src, dst)] = self.W[k].get((src, dst), 0.0) + coef * mat
                else:
                    assert src_plain or not dst_plain, "right-keyed channel cannot turn left-keyed"
                    old = self.W[k].get((src, dst))
                    assert old is None or np.array_equal(old, mat)
                    self.W[k][(src, dst)] = mat
        self.parity, self.dq = [], []
        for k in range(n + 1):
            par = [0] * len(self.chans[k])
            dq = [(0, 0)] * len(self.chans[k])
            for key, i in self.chans[k].items():
                if key in ("I", "H"):
                    continue
                par[i] = string_parity(key[1])
                d = string_dq(key[1])
                dq[i] = d if key[0] == "L" else (-d[0], -d[1])
            self.parity.append(par)
            self.dq.append(dq)

    def bond_dims(self):
        return [len(c) for c in self.chans]

    def dense(self):
        """Dense 4^n x 4^n matrix (site 0 most significant), for small n only."""
        import scipy.sparse as sp   # the same Kronecker products, stored sparse
        T = {0: sp.csr_matrix(np.ones((1, 1)))}
        for k in range(self.n):
            new = {}
            for (w, w2), m in self.W[k].items():
                if w not in T:
                    continue
                mp = m @ ops.PARITY if self.parity[k + 1][w2] else m
                t = sp.kron(T[w], sp.csr_matrix(mp), format="csr")
                new[w2] = new[w2] + t if w2 in new else t
            T = new
        return T[self.chans[self.n]["H"]].toarray()


def product_state_dets(n):
    """Determinant integer of every product state |s_0 ... s_{n-1}> in kron order."""
    occ = [(0, 0), (1, 0), (0, 1), (1, 1)]
    dets = np.zeros(4 ** n, dtype=np.int64)
    for idx in range(4 ** n):
        d, rem = 0, idx
        for j in range(n - 1, -1, -1):
            s = rem % 4
            rem //= 4
            a, b = occ[s]
            d |= (a << (2 * j)) | (b << (2 * j + 1))
        dets[idx] = d
    return dets
