"""Plain two-site DMRG in FP64 on the CPU (test infrastructure only).

Follows the two-site sweep algorithm of the paper (Sec. 2.1.2: the renormalized
wavefunction lives on the product of the left block states, the d = 16 two-site local
space and the right block states), with the standard Davidson solver (Sec. 2.1.3 (iv)
names it; settings thrds = 1e-10 on the squared residual and dav_max_iter = 30 as in
Listing 1), density-matrix truncation to M states per bond, and environments
(renormalized operators) built from an MPO (Sec. 2.3).

Representation (deliberately simple): every bond index runs over all its states in
sector order, tensors are dense numpy arrays whose forbidden (quantum-number violating)
entries are zero, and a label array gives (N, 2Sz) of each state.  Truncation works per
quantum-number sector, so the zeros stay exact zeros.

Index conventions
  A[k]      (M_k, 4, M_{k+1}) site tensor, bond k between sites k-1 and k
  L[k][w]   (M_k, M_k) left environment of channel w on bond k: <l'| left part of w |l>
  R[k][w]   (M_k, M_k) right environment of channel w on bond k (right block states are
            labelled by bond k's left-block quantum numbers)
  psi       (M_i, 4, 4, M_{i+2}) two-site wavefunction of window (i, i+1)
Operator ordering on |l s1 s2 r> is (left part)(site i)(site i+1)(right part); moving an
odd operator past an odd number of fermions costs a sign (Sec. "Fermion convention" of
``mpo``).
"""
import numpy as np

from . import ops

SITE_Q = np.array(ops.SITE_Q)


# ----------------------------------------------------------------------------- layout
def blocks_to_dense(bonds, sites):
    """Block-sparse MPS (the ``synth`` file format) -> (labels, dense site tensors)."""
    labels = []
    for b in bonds:
        lab = [(N, tsz) for (N, tsz, m) in b for _ in range(m)]
        labels.append(np.array(lab, dtype=np.int64).reshape(-1, 2))
    offs = [np.cumsum([0] + [m for (_, _, m) in b]) for b in bonds]
    A = []
    for k, blocks in enumerate(sites):
        t = np.zeros((len(labels[k]), 4, len(labels[k + 1])))
        for (jl, s, jr), blk in blocks.items():
            t[offs[k][jl]:offs[k][jl + 1], s, offs[k + 1][jr]:offs[k + 1][jr + 1]] = blk
        A.append(t)
    return labels, A


def parity_of(labels):
    """(-1)^N for every state of a bond."""
    return np.where(labels[:, 0] % 2 == 1, -1.0, 1.0)


# ------------------------------------------------------------------------ environments
def left_boundary():
    return [np.ones((1, 1))]


def right_boundary():
    return [np.ones((1, 1))]


def left_env_update(Lk, A, Wk, lab_k, n_chan_next):
    """L_{k+1}[w'] = sum_{w,s',s} W_k[w,w']_{s's} (-1)^{p(op) n(l)} A_{s'}^T L_k[w] A_s."""
    par = parity_of(lab_k)
    out = [np.zeros((A.shape[2], A.shape[2])) for _ in range(n_chan_next)]
    for (w, w2), m in Wk.items():
        if Lk[w] is None:
            continue
        for s2, s in zip(*np.nonzero(m)):
            odd = (ops.SITE_N[s2] + ops.SITE_N[s]) % 2
            Lw = Lk[w] * par[None, :] if odd else Lk[w]
            out[w2] += m[s2, s] * (A[:, s2, :].T @ Lw @ A[:, s, :])
    return out


def right_env_update(Rk1, B, Wk, parity_next, n_chan):
    """R_k[w] = sum_{w',s',s} W_k[w,w']_{s's} (-1)^{p(w') n(s)} B_{s'} R_{k+1}[w'] B_s^T."""
    out = [np.zeros((B.shape[0], B.shape[0])) for _ in range(n_chan)]
    for (w, w2), m in Wk.items():
        if Rk1[w2] is None:
            continue
        for s2, s in zip(*np.nonzero(m)):
            sign = -1.0 if (parity_next[w2] and ops.SITE_N[s] % 2) else 1.0
            out[w] += (sign * m[s2, s]) * (B[:, s2, :] @ Rk1[w2] @ B[:, s, :].T)
    return out


# ----------------------------------------------------------------- effective Hamiltonian
def two_site_operators(mpo, i):
    """{(a, b): O_ab} for window (i, i+1): O_ab = sum_w' W_i[a,w'] (x) W_{i+1}[w',b] as a
    16 x 16 matrix over (s1, s2) = 4*s1 + s2, including the sign (-1)^{p(op2) n(s1)} of
    moving the site-(i+1) operator past the site-i ket."""
    right = {}
    for (w2, b), m2 in mpo.W[i + 1].items():
        right.setdefault(w2, []).append((b, m2))
    out = {}
    for (a, w2), m1 in mpo.W[i].items():
        for b, m2 in right.get(w2, ()):
            p2 = ops.op_parity(m2)
            o = np.kron(m1 @ ops.PARITY if p2 else m1, m2)
            out[(a, b)] = out.get((a, b), 0.0) + o
    return {k: v for k, v in out.items() if np.any(v)}


class Heff:
    """H_eff of window (i, i+1) from L_i, R_{i+2} and the MPO (Sec. 2.1.2, Sec. 2.3).

    Applied to psi: Y = sum_{a,b} (L_a P^{p(a)}) (x) O'_ab (x) R_b, where P is the parity of
    the left ket and O'_ab = O_ab diag((-1)^{p(b) (n(s1) + n(s2))}) carries the sign of
    moving the right part past the two site kets."""

    def __init__(self, mpo, i, L, R, lab_l):
        self.terms = two_site_operators(mpo, i)
        self.dq_l = mpo.dq[i]
        self.dq_r = mpo.dq[i + 2]
        self.L, self.R = L, R
        self.par_l = parity_of(lab_l)
        self.pa = mpo.parity[i]
        self.pb = mpo.parity[i + 2]
        n_in = np.add.outer(ops.SITE_N, ops.SITE_N).ravel()
        self.sgn_in = np.where(n_in % 2 == 1, -1.0, 1.0)
        by_a = {}
        for (a, b), o in self.terms.items():
            o2 = o * self.sgn_in[None, :] if self.pb[b] else o
            by_a.setdefault(a, []).append((b, o2))
        # per left channel a: the signed left operator, the stacked O'_ab and R_b^T
        self.groups = []
        for a, lst in by_a.items():
            La = self.L[a] * self.par_l[None, :] if self.pa[a] else self.L[a]
            Os = np.array([o for _, o in lst])                        # (nb, 16, 16)
            RsT = np.array([self.R[b].T for b, _ in lst])             # (nb, mr, mr')
            self.groups.append((La, Os, RsT))

    def algorithmic_flops(self, lab_l, lab_r):
        """Floating-point operations of the block-sparse form of this product: for every
        operator pair (a, b), every nonzero local element O_ab[(s1' s2'), (s1 s2)] and every
        pair of sectors (l, r) of psi that it connects to an existing output block (l', r'),
        2 m_l' m_l m_r (L_a psi) + 2 m_l' m_r m_r' (times R_b^T).  Counts the work of the
        product itself (used to express the oracle's speed in the unit of the benchmark)."""
        def sectors(lab):
            out = {}
            for q in map(tuple, lab):
                out[q] = out.get(q, 0) + 1
            return out
        ml, mr = sectors(lab_l), sectors(lab_r)
        q = [tuple(x) for x in SITE_Q]
        flops = 0.0
        for (a, b), o in self.terms.items():
            dqa = self.dq_l[a]
            dqb = self.dq_r[b]
            for u, v in zip(*np.nonzero(o)):
                s1p, s2p, s1, s2 = u // 4, u % 4, v // 4, v % 4
                for ql, m_l in ml.items():
                    qr = (ql[0] + q[s1][0] + q[s2][0], ql[1] + q[s1][1] + q[s2][1])
                    m_r = mr.get(qr)
                    if m_r is None:
                        continue
                    qlp = (ql[0] + dqa[0], ql[1] + dqa[1])
                    qrp = (qr[0] + dqb[0], qr[1] + dqb[1])
                    m_lp, m_rp = ml.get(qlp), mr.get(qrp)
                    if m_lp is None or m_rp is None:
                        continue
                    if (qlp[0] + q[s1p][0] + q[s2p][0], qlp[1] + q[s1p][1] + q[s2p][1]) != qrp:
                        continue
                    flops += 2.0 * m_lp * m_l * m_r + 2.0 * m_lp * m_r * m_rp
        return flops

    def apply(self, psi):
        ml, mr = psi.shape[0], psi.shape[3]
        x = psi.reshape(ml, 16 * mr)
        y = np.zeros((ml, 16, mr))
        for La, Os, RsT in self.groups:
            t = (La @ x).reshape(ml, 16, mr)
            u = np.matmul(t[None], RsT[:, None])                     # (nb, ml, 16, mr')
            # y[x, u, y'] += sum_{b, v} O'_b[u, v] u[b, x, v, y']
            y += np.tensordot(Os, u, axes=([0, 2], [0, 2])).transpose(1, 0, 2)
        return y.reshape(psi.shape)

    def diag(self):
        ml = self.L[0].shape[0]
        mr = self.R[0].shape[0]
        d = np.zeros((ml, 16, mr))
        for (a, b), o in self.terms.items():
            dl = np.diag(self.L[a]) * (self.par_l if self.pa[a] else 1.0)
            dr = np.diag(self.R[b])
            do = np.diag(o) * (self.sgn_in if self.pb[b] else 1.0)
            d += dl[:, None, None] * do[None, :, None] * dr[None, None, :]
        return d.reshape(ml, 4, 4, mr)


class Heff1:
    """H_eff of the one-site window of site i from L_i, R_{i+1} and the MPO (Sec. 2.1.2,
    one-site algorithm: the d = 4 space of one site between the two blocks).

    Applied to psi (M_i, 4, M_{i+1}): Y = sum_{a,b} (L_a P^{p(a)}) (x) O'_ab (x) R_b with
    O_ab = W_i[a, b] and O'_ab = O_ab diag((-1)^{p(b) n(s)}), the sign of moving the right
    part past the site ket (the two-site rule with one site)."""

    def __init__(self, mpo, i, L, R, lab_l):
        self.L, self.R = L, R
        self.par_l = parity_of(lab_l)
        self.pa = mpo.parity[i]
        self.pb = mpo.parity[i + 1]
        self.sgn_in = np.where(ops.SITE_N % 2 == 1, -1.0, 1.0)
        self.terms = {}
        for (a, b), m in mpo.W[i].items():
            if np.any(m):
                self.terms[(a, b)] = m * self.sgn_in[None, :] if self.pb[b] else m

    def apply(self, psi):
        ml, _, mr = psi.shape
        x = psi.reshape(ml, 4 * mr)
        y = np.zeros(psi.shape)
        by_a = {}
        for (a, b), o in self.terms.items():
            by_a.setdefault(a, []).append((b, o))
        for a, lst in by_a.items():
            La = self.L[a] * self.par_l[None, :] if self.pa[a] else self.L[a]
            t = (La @ x).reshape(ml, 4, mr)                       # L_a psi
            for b, o in lst:
                # y[l', s', r'] += sum_{s, r} o[s', s] t[l', s, r] R_b[r', r]
                y += np.einsum("uv,xvr->xur", o, t) @ self.R[b].T
        return y

    def diag(self):
        ml, mr = self.L[0].shape[0], self.R[0].shape[0]
        d = np.zeros((ml, 4, mr))
        for (a, b), o in self.terms.items():
            dl = np.diag(self.L[a]) * (self.par_l if self.pa[a] else 1.0)
            d += dl[:, None, None] * np.diag(o)[None, :, None] * np.diag(self.R[b])[None, None, :]
        return d


# ------------------------------------------------------------------------------ Davidson
def davidson(matvec, diag, x0, tol=1e-10, max_iter=30, max_sub=30):
    """Lowest eigenpair by the standard Davidson method (Davidson 1975).

    Subspace V (orthonormal) and W = H V; Rayleigh-Ritz on G = V^T W; residual
    r = W s - theta V s; stop when |r|^2 <= tol or after max_iter products with H;
    correction t = r / (D - theta) (denominators below 1e-8 in size set to 1e-8),
    orthogonalised twice against V; a full subspace restarts from the Ritz vector.
    Returns (theta, unit vector, number of products, |r|^2)."""
    shape = x0.shape
    d = diag.ravel()
    v = x0.ravel() / np.linalg.norm(x0)
    V = [v]
    Wl = [matvec(v.reshape(shape)).ravel()]
    nmv = 1
    while True:
        Vm, Wm = np.array(V).T, np.array(Wl).T
        G = Vm.T @ Wm
        G = 0.5 * (G + G.T)
        evals, evecs = np.linalg.eigh(G)
        theta, s = float(evals[0]), evecs[:, 0]
        u, hu = Vm @ s, Wm @ s
        r = hu - theta * u
        rn2 = float(r @ r)
        if rn2 <= tol or nmv >= max_iter:
            break
        den = d - theta
        den = np.where(np.abs(den) < 1e-8, 1e-8, den)
        t = r / den
        if len(V) >= max_sub:
            V, Wl = [u], [hu]
        for _ in range(2):
            for vv in V:
                t = t - (vv @ t) * vv
        tn = np.linalg.norm(t)
        if tn < 1e-14:
            break
        t = t / tn
        V.append(t)
        Wl.append(matvec(t.reshape(shape)).ravel())
        nmv += 1
    u = u / np.linalg.norm(u)
    return theta, u.reshape(shape), nmv, rn2


# ------------------------------------------------------------------ perturbative noise
# The MPO factorises exactly across the bond being split (channels w of that bond):
#   H = sum_w S_w (x) E_w,  S_w = sum_a (-1)^{p(a) N(l)} L_a (x) W_left[a, w] diag((-1)^{p(w) n(s)}),
#                           E_w = sum_b W_right[w, b] diag((-1)^{p(b) n(s)}) (x) R_b,
# (the two-site H_eff's signs regrouped: the sign of moving the right part of w past the
# left site is (-1)^{p(w) n(s1)}).  The perturbative noise of White (2005) adds to the
# density matrix of the kept part the weight that the system-side operators move psi into:
# N = sum_w P_w P_w^T with P_w = S_w psi (forward split, kept part (l, s)) or E_w psi
# (backward split, kept part (s, r)); sign factors on the other side's indices cancel in
# P_w P_w^T.  The split then diagonalises rho + noise * N / tr N (N restricted to the
# sectors the new bond can hold), so the noise adds total weight `noise` (Sec. 2.1.6 names
# perturbative noise; the normalisation is this build's choice).
def system_left(X3, L, W, par_l, pa, pw):
    """{w: P_w = S_w psi} for X3 = psi as (M_l, 4, cols), rows (l, s) the kept part.  W: the
    MPO tensor of the kept site, channels (a on the left bond, w on the cut bond); pw: the
    parities of the cut bond's channels."""
    ml, _, nc = X3.shape
    sgn = np.where(ops.SITE_N % 2 == 1, -1.0, 1.0)
    P = {}
    for (a, w), m in W.items():
        La = L[a] * par_l[None, :] if pa[a] else L[a]
        mw = m * sgn[None, :] if pw[w] else m
        t = (La @ X3.reshape(ml, 4 * nc)).reshape(ml, 4, nc)       # L_a psi
        t = np.einsum("uv,xvc->xuc", mw, t)                        # site operator on s
        P[w] = P[w] + t if w in P else t
    return P


def system_right(X3, R, W, pb):
    """{w: P_w = E_w psi} for X3 = psi as (rows of the other part, 4, M_r), (s, r) the kept
    part.  W: the MPO tensor of the kept site (channels w on the cut bond, b on the right
    bond); pb: the parities of the right bond's channels."""
    sgn = np.where(ops.SITE_N % 2 == 1, -1.0, 1.0)
    P = {}
    for (w, b), m in W.items():
        mb = m * sgn[None, :] if pb[b] else m
        t = np.einsum("uv,evr->eur", mb, X3) @ R[b].T              # (ne, 4, M_r')
        P[w] = P[w] + t if w in P else t
    return P


def noise_left(X3, L, W, par_l, pa, pw):
    """N = sum_w P_w P_w^T over rows (l, s), P_w from system_left."""
    ml, _, nc = X3.shape
    N = np.zeros((ml * 4, ml * 4))
    for t in system_left(X3, L, W, par_l, pa, pw).values():
        t2 = t.reshape(ml * 4, nc)
        N += t2 @ t2.T
    return N


def noise_right(X3, R, W, pb):
    """N = sum_w P_w^T P_w over rows (s, r), P_w from system_right."""
    ne, _, mr = X3.shape
    N = np.zeros((4 * mr, 4 * mr))
    for t in system_right(X3, R, W, pb).values():
        t2 = t.reshape(ne, 4 * mr)
        N += t2.T @ t2
    return N


def _add_noise(X_rows, row_lab, allowed, N, noise):
    """Density matrix rho = X X^T (+ noise * N / tr N on the allowed sectors' rows).  Rows of
    a label outside `allowed` are zero in X and get no noise."""
    rho = X_rows @ X_rows.T
    if noise > 0 and N is not None:
        ok = np.array([tuple(q) in allowed for q in row_lab])
        Nm = N * ok[:, None] * ok[None, :]
        tr = float(np.trace(Nm))
        if tr > 0:
            rho = rho + (noise / tr) * Nm
    return rho


def davidson_roots(matvec, diag, X0, tol=1e-10, max_iter=100, max_sub=40, allowed=None):
    """The k lowest eigenpairs by the block form of the Davidson method (Davidson 1975 with
    several roots, Liu 1978).

    Guesses X0 (k arrays) are orthonormalised in order (twice Gram-Schmidt); one whose
    remainder has norm <= 1e-8 is replaced by the unit vector at the smallest diagonal
    element not used yet (ties by index) among the `allowed` entries (boolean mask of the
    quantum-number-allowed elements; default all).  Subspace V (orthonormal), W = H V; Rayleigh-Ritz
    on G = V^T W; the k lowest Ritz pairs (theta_j, u_j); r_j = W s_j - theta_j u_j.  Stop
    when every |r_j|^2 <= tol or after max_iter products.  Otherwise the corrections
    t_j = r_j / (D - theta_j) (denominators below 1e-8 in size set to 1e-8) of the roots with
    |r_j|^2 > tol, in root order, are each orthogonalised twice against V (and the
    corrections added before), normalised and added unless their norm is <= 1e-14.  When the
    subspace cannot take them (size + count > max_sub) it restarts from the k Ritz vectors.
    Returns (thetas, unit vectors, number of products, max |r_j|^2)."""
    k = len(X0)
    shape = X0[0].shape
    d = diag.ravel()
    V = []
    used = set()
    order = np.argsort(d, kind="stable")
    if allowed is not None:
        order = [j for j in order if allowed.ravel()[j]]
    for x in X0:
        v = x.ravel().astype(float).copy()
        for _ in range(2):
            for vv in V:
                v = v - (vv @ v) * vv
        nv = np.linalg.norm(v)
        if nv <= 1e-8:
            for idx in order:
                if idx in used:
                    continue
                e = np.zeros(len(d))
                e[idx] = 1.0
                for _ in range(2):
                    for vv in V:
                        e = e - (vv @ e) * vv
                if np.linalg.norm(e) > 1e-8:
                    used.add(idx)
                    v, nv = e, np.linalg.norm(e)
                    break
        V.append(v / nv)
    Wl = [matvec(v.reshape(shape)).ravel() for v in V]
    nmv = k
    while True:
        Vm, Wm = np.array(V).T, np.array(Wl).T
        G = Vm.T @ Wm
        G = 0.5 * (G + G.T)
        evals, evecs = np.linalg.eigh(G)
        thetas = evals[:k]
        U, HU = Vm @ evecs[:, :k], Wm @ evecs[:, :k]
        R = HU - U * thetas[None, :]
        rn2 = np.sum(R * R, axis=0)
        if np.all(rn2 <= tol) or nmv >= max_iter:
            break
        todo = [j for j in range(k) if rn2[j] > tol]
        if len(V) + len(todo) > max_sub:
            V = [U[:, j] / np.linalg.norm(U[:, j]) for j in range(k)]
            Wl = [HU[:, j] / np.linalg.norm(U[:, j]) for j in range(k)]
        added = 0
        for j in todo:
            den = d - thetas[j]
            den = np.where(np.abs(den) < 1e-8, 1e-8, den)
            t = R[:, j] / den
            for _ in range(2):
                for vv in V:
                    t = t - (vv @ t) * vv
            tn = np.linalg.norm(t)
            if tn <= 1e-14:
                continue
            t = t / tn
            V.append(t)
            Wl.append(matvec(t.reshape(shape)).ravel())
            nmv += 1
            added += 1
        if added == 0:
            break
    out = [(U[:, j] / np.linalg.norm(U[:, j])).reshape(shape) for j in range(k)]
    return [float(x) for x in thetas], out, nmv, float(rn2.max())


def krylov_exp(matvec, x, t, tol=1e-12, max_k=40):
    """exp(-t H) x by the Krylov (Lanczos) method: orthonormal basis V of span{x, Hx, ...}
    (each new vector orthogonalised twice against all previous ones), T = V^T H V, and
    y = |x| V exp(-t T) e_1.  With c = exp(-t (T - lambda_min)) e_1 (shifted against
    overflow), it stops when the next vector's weight |beta_k| |c_k| is <= tol |c|, when the
    space is exhausted (beta <= 1e-14 max(1, |lambda|)) or at max_k vectors."""
    shape = x.shape
    nx = np.linalg.norm(x)
    V = [x.ravel() / nx]
    HV = []
    while True:
        w = matvec(V[-1].reshape(shape)).ravel()
        HV.append(w)
        k = len(V)
        T = np.array(V) @ np.array(HV).T
        T = 0.5 * (T + T.T)
        lam, U = np.linalg.eigh(T)
        c = U @ (np.exp(-t * (lam - lam[0])) * U[0, :])      # exp(-t (T - lam_0)) e_1
        for _ in range(2):
            for v in V:
                w = w - (v @ w) * v
        beta = np.linalg.norm(w)
        if beta * abs(c[-1]) <= tol * np.linalg.norm(c) \
                or beta <= 1e-14 * max(1.0, np.abs(lam).max()) or k >= max_k:
            break
        V.append(w / beta)
    y = nx * np.exp(-t * lam[0]) * (np.array(V).T @ c)
    return y.reshape(shape)


# ---------------------------------------------------------------------------- truncation
def _select(evals_by_sector, M, cutoff):
    """Keep the M largest eigenvalues over all sectors.  Eigenvalues <= cutoff * max are
    dropped.  Ties (|difference| <= 1e-14 * max) are broken by (sector index, index in
    sector), both ascending.  Returns the kept count per sector."""
    cand = []
    for j, w in enumerate(evals_by_sector):
        for t, lam in enumerate(w):
            cand.append((float(lam), j, t))
    if not cand:
        return [0] * len(evals_by_sector)
    lmax = max(c[0] for c in cand)
    cand.sort(key=lambda c: -c[0])
    # chain near-equal neighbours into groups, then order each group by (sector, index)
    ordered, group = [], [cand[0]]
    for c in cand[1:]:
        if group[-1][0] - c[0] <= 1e-14 * lmax:
            group.append(c)
        else:
            ordered.extend(sorted(group, key=lambda g: (g[1], g[2])))
            group = [c]
    ordered.extend(sorted(group, key=lambda g: (g[1], g[2])))
    kept = [0] * len(evals_by_sector)
    for lam, j, t in ordered[:M]:
        if lam > cutoff * lmax:
            kept[j] += 1
    return kept


def _sector_eigs(X, labels, rho=None):
    """Per sector q (sorted): eigenvalues (descending) and eigenvectors of X_q X_q^T,
    X_q the rows of X labelled q (or of the given rho's diagonal block q)."""
    secs = sorted({tuple(q) for q in labels})
    out = []
    for q in secs:
        rows = np.nonzero((labels[:, 0] == q[0]) & (labels[:, 1] == q[1]))[0]
        if rho is None:
            xq = X[rows]
            w, u = np.linalg.eigh(xq @ xq.T)
        else:
            w, u = np.linalg.eigh(rho[np.ix_(rows, rows)])
        out.append((q, rows, w[::-1], u[:, ::-1]))
    return out


def left_split(psi, lab_l, M, cutoff=1e-14, N=None, noise=0.0, lab_r=None):
    """psi (l s1, s2 r) -> A (l, s1, new) with A^T A = 1, C = A^T psi, new bond labels,
    discarded weight (of the density matrix, noise included).  N, noise, lab_r: the
    perturbative noise matrix over rows (l, s1), its weight and the right bond's labels."""
    ml, _, _, mr = psi.shape
    X = psi.reshape(ml * 4, 4 * mr)
    row_lab = (lab_l[:, None, :] + SITE_Q[None, :, :]).reshape(-1, 2)
    rho = None
    if noise > 0:
        allowed = {tuple(q) for q in (lab_r[None, :, :] - SITE_Q[:, None, :]).reshape(-1, 2)}
        rho = _add_noise(X, row_lab, allowed, N, noise)
    eig = _sector_eigs(X, row_lab, rho)
    kept = _select([e[2] for e in eig], M, cutoff)
    cols, lab = [], []
    for (q, rows, w, u), kq in zip(eig, kept):
        for t in range(kq):
            c = np.zeros(ml * 4)
            c[rows] = u[:, t]
            cols.append(c)
            lab.append(q)
    A = np.array(cols).T.reshape(ml, 4, len(cols))
    C = (A.reshape(ml * 4, -1).T @ X).reshape(-1, 4, mr)
    total = sum(float(np.sum(e[2])) for e in eig)
    keptw = sum(float(np.sum(e[2][:kq])) for e, kq in zip(eig, kept))
    return A, C, np.array(lab, dtype=np.int64).reshape(-1, 2), total - keptw


def right_split(psi, lab_r, M, cutoff=1e-14, N=None, noise=0.0, lab_l=None):
    """psi (l s1, s2 r) -> B (new, s2, r) with B B^T = 1, C = psi B^T, new bond labels
    (left-block quantum numbers of the new bond), discarded weight.  N: noise matrix over
    rows (s2, r)."""
    ml, _, _, mr = psi.shape
    X = psi.reshape(ml * 4, 4 * mr)
    col_lab = (lab_r[None, :, :] - SITE_Q[:, None, :]).reshape(-1, 2)
    rho = None
    if noise > 0:
        allowed = {tuple(q) for q in (lab_l[:, None, :] + SITE_Q[None, :, :]).reshape(-1, 2)}
        rho = _add_noise(X.T, col_lab, allowed, N, noise)
    eig = _sector_eigs(X.T, col_lab, rho)
    kept = _select([e[2] for e in eig], M, cutoff)
    rows_out, lab = [], []
    for (q, cidx, w, u), kq in zip(eig, kept):
        for t in range(kq):
            r = np.zeros(4 * mr)
            r[cidx] = u[:, t]
            rows_out.append(r)
            lab.append(q)
    B = np.array(rows_out).reshape(len(rows_out), 4, mr)
    C = (X @ B.reshape(len(rows_out), -1).T).reshape(ml, 4, -1)
    total = sum(float(np.sum(e[2])) for e in eig)
    keptw = sum(float(np.sum(e[2][:kq])) for e, kq in zip(eig, kept))
    return B, C, np.array(lab, dtype=np.int64).reshape(-1, 2), total - keptw


def left_split1(psi, lab_l, M, cutoff=1e-14, N=None, noise=0.0, lab_r=None):
    """One-site psi (l s, r) -> A (l, s, new) with A^T A = 1, C = A^T psi (new, r), new
    bond labels, discarded weight (the density matrix of the left part, as left_split)."""
    ml, _, mr = psi.shape
    X = psi.reshape(ml * 4, mr)
    row_lab = (lab_l[:, None, :] + SITE_Q[None, :, :]).reshape(-1, 2)
    rho = None
    if noise > 0:
        rho = _add_noise(X, row_lab, {tuple(q) for q in lab_r}, N, noise)
    eig = _sector_eigs(X, row_lab, rho)
    kept = _select([e[2] for e in eig], M, cutoff)
    cols, lab = [], []
    for (q, rows, w, u), kq in zip(eig, kept):
        for t in range(kq):
            c = np.zeros(ml * 4)
            c[rows] = u[:, t]
            cols.append(c)
            lab.append(q)
    U = np.array(cols).T
    total = sum(float(np.sum(e[2])) for e in eig)
    keptw = sum(float(np.sum(e[2][:kq])) for e, kq in zip(eig, kept))
    return (U.reshape(ml, 4, -1), U.T @ X, np.array(lab, dtype=np.int64).reshape(-1, 2),
            total - keptw)


def right_split1(psi, lab_r, M, cutoff=1e-14, N=None, noise=0.0, lab_l=None):
    """One-site psi (l, s r) -> B (new, s, r) with B B^T = 1, C = psi B^T (l, new), new
    bond labels (left-block quantum numbers), discarded weight."""
    ml, _, mr = psi.shape
    X = psi.reshape(ml, 4 * mr)
    col_lab = (lab_r[None, :, :] - SITE_Q[:, None, :]).reshape(-1, 2)
    rho = None
    if noise > 0:
        rho = _add_noise(X.T, col_lab, {tuple(q) for q in lab_l}, N, noise)
    eig = _sector_eigs(X.T, col_lab, rho)
    kept = _select([e[2] for e in eig], M, cutoff)
    rows_out, lab = [], []
    for (q, cidx, w, u), kq in zip(eig, kept):
        for t in range(kq):
            r = np.zeros(4 * mr)
            r[cidx] = u[:, t]
            rows_out.append(r)
            lab.append(q)
    Bm = np.array(rows_out)
    total = sum(float(np.sum(e[2])) for e in eig)
    keptw = sum(float(np.sum(e[2][:kq])) for e, kq in zip(eig, kept))
    return (Bm.reshape(-1, 4, mr), X @ Bm.T, np.array(lab, dtype=np.int64).reshape(-1, 2),
            total - keptw)


# --------------------------------------------------------------------------------- sweep
class DMRG:
    """Two-site DMRG driver.  Sweep = forward half over windows 0..n-2 followed by a
    backward half over windows n-2..0.  After optimising window i the forward half splits
    psi into A_i (left-canonical) and moves right (unless i = n-2); the backward half
    splits into B_{i+1} (right-canonical) and moves left (unless i = 0).  The guess for the
    next window is the split remainder contracted with the next site tensor."""

    def __init__(self, mpo, bonds, sites, center=0):
        self.mpo = mpo
        self.n = mpo.n
        self.lab, self.A = blocks_to_dense(bonds, sites)
        n = self.n
        self.L = [None] * (n + 1)
        self.R = [None] * (n + 1)
        self.L[0] = left_boundary()
        self.R[n] = right_boundary()
        for k in range(center):
            self.L[k + 1] = left_env_update(self.L[k], self.A[k], mpo.W[k], self.lab[k],
                                            len(mpo.chans[k + 1]))
        for k in range(n - 1, center + 1, -1):
            self.R[k] = right_env_update(self.R[k + 1], self.A[k], mpo.W[k],
                                         mpo.parity[k + 1], len(mpo.chans[k]))
        self.psi = np.einsum("asb,btc->astc", self.A[center], self.A[center + 1])
        self.stats = []

    def heff(self, i):
        return Heff(self.mpo, i, self.L[i], self.R[i + 2], self.lab[i])

    def optimise(self, i, tol, max_iter, max_sub):
        h = self.heff(i)
        e, psi, nmv, rn2 = davidson(h.apply, h.diag(), self.psi, tol, max_iter, max_sub)
        self.psi = psi
        self.stats.append({"window": i, "energy": e, "n_matvec": nmv, "resid2": rn2})
        return e

    def move_right(self, i, M, cutoff, noise=0.0):
        N = None
        if noise > 0:
            m = self.mpo
            N = noise_left(self.psi.reshape(self.psi.shape[0], 4, -1), self.L[i], m.W[i],
                           parity_of(self.lab[i]), m.parity[i], m.parity[i + 1])
        A, C, lab, dw = left_split(self.psi, self.lab[i], M, cutoff, N, noise, self.lab[i + 2])
        self.A[i] = A
        self.lab[i + 1] = lab
        self.L[i + 1] = left_env_update(self.L[i], A, self.mpo.W[i], self.lab[i],
                                        len(self.mpo.chans[i + 1]))
        self.psi = np.einsum("asb,btc->astc", C, self.A[i + 2])
        return dw

    def move_left(self, i, M, cutoff, noise=0.0):
        N = None
        if noise > 0:
            m = self.mpo
            N = noise_right(self.psi.reshape(-1, 4, self.psi.shape[3]), self.R[i + 2], m.W[i + 1],
                            m.parity[i + 2])
        B, C, lab, dw = right_split(self.psi, self.lab[i + 2], M, cutoff, N, noise, self.lab[i])
        self.A[i + 1] = B
        self.lab[i + 1] = lab
        self.R[i + 1] = right_env_update(self.R[i + 2], B, self.mpo.W[i + 1],
                                         self.mpo.parity[i + 2], len(self.mpo.chans[i + 1]))
        self.psi = np.einsum("asb,btc->astc", self.A[i - 1], C)
        return dw

    def sweep(self, M, tol=1e-10, max_iter=30, max_sub=30, cutoff=1e-14, noise=0.0):
        n = self.n
        dws = []
        for i in range(0, n - 1):
            self.optimise(i, tol, max_iter, max_sub)
            if i < n - 2:
                dws.append(self.move_right(i, M, cutoff, noise))
        for i in range(n - 2, -1, -1):
            e = self.optimise(i, tol, max_iter, max_sub)
            if i > 0:
                dws.append(self.move_left(i, M, cutoff, noise))
        return e, max(dws) if dws else 0.0

    def run(self, bond_dims, tol=1e-10, max_iter=30, max_sub=30, cutoff=1e-14, dots=None,
            noise=None):
        """Sweeps with bond dimension bond_dims[k]; dots[k] = 1 makes sweep k a one-site
        sweep (default: all two-site).  Mixing the two (Sec. 2.1.2) switches between the
        two-site and the one-site wavefunction at the start of a sweep.  noise[k]: weight of
        the perturbative noise in sweep k's splits (default none)."""
        energies = []
        for k, M in enumerate(bond_dims):
            nz = 0.0 if noise is None else noise[k]
            if dots is not None and dots[k] == 1:
                e, _ = self.sweep1(M, tol, max_iter, max_sub, cutoff, nz)
            else:
                self.to_two_site()
                e, _ = self.sweep(M, tol, max_iter, max_sub, cutoff, nz)
            energies.append(e)
        return energies

    # ------------------------------------------------------------ one-site algorithm
    # Between sweeps the centre is at the left end: either the two-site psi of window
    # (0, 1) (after a two-site sweep; R_2 exists) or the one-site psi of site 0 (after a
    # one-site sweep or at the start; R_1 exists once needed).
    def heff1(self, i):
        return Heff1(self.mpo, i, self.L[i], self.R[i + 1], self.lab[i])

    def to_one_site(self, M, cutoff):
        """Two-site psi of window (0, 1) -> one-site psi of site 0 by the backward split
        (B_1 right-orthonormal, R_1 from it), truncated like any split to M states.  At the
        start (no sweep yet) the centre tensor A_0 itself is the one-site psi."""
        if self.psi.ndim == 3:
            return
        if not self.stats:
            self.psi = self.A[0].copy()
        else:
            B, C, lab, _ = right_split(self.psi, self.lab[2], M, cutoff)
            self.A[1] = B
            self.lab[1] = lab
            self.psi = C.reshape(C.shape[0], 4, -1)
        self.R[1] = right_env_update(self.R[2], self.A[1], self.mpo.W[1], self.mpo.parity[2],
                                     len(self.mpo.chans[1]))

    def to_two_site(self):
        """One-site psi of site 0 -> two-site psi of window (0, 1): psi . A_1."""
        if self.psi.ndim == 3:
            self.psi = np.einsum("asb,btc->astc", self.psi, self.A[1])

    def optimise1(self, i, tol, max_iter, max_sub):
        h = self.heff1(i)
        e, psi, nmv, rn2 = davidson(h.apply, h.diag(), self.psi, tol, max_iter, max_sub)
        self.psi = psi
        self.stats.append({"window": i, "energy": e, "n_matvec": nmv, "resid2": rn2, "dot": 1})
        return e

    def move_right1(self, i, M, cutoff, noise=0.0):
        N = None
        if noise > 0:
            m = self.mpo
            N = noise_left(self.psi, self.L[i], m.W[i], parity_of(self.lab[i]), m.parity[i],
                           m.parity[i + 1])
        A, C, lab, dw = left_split1(self.psi, self.lab[i], M, cutoff, N, noise, self.lab[i + 1])
        self.A[i] = A
        self.lab[i + 1] = lab
        self.L[i + 1] = left_env_update(self.L[i], A, self.mpo.W[i], self.lab[i],
                                        len(self.mpo.chans[i + 1]))
        self.psi = np.einsum("ab,bsc->asc", C, self.A[i + 1])
        return dw

    def move_left1(self, i, M, cutoff, noise=0.0):
        N = None
        if noise > 0:
            m = self.mpo
            N = noise_right(self.psi, self.R[i + 1], m.W[i], m.parity[i + 1])
        B, C, lab, dw = right_split1(self.psi, self.lab[i + 1], M, cutoff, N, noise, self.lab[i])
        self.A[i] = B
        self.lab[i] = lab
        self.R[i] = right_env_update(self.R[i + 1], B, self.mpo.W[i], self.mpo.parity[i + 1],
                                     len(self.mpo.chans[i]))
        self.psi = np.einsum("asb,bc->asc", self.A[i - 1], C)
        return dw

    def sweep1(self, M, tol=1e-10, max_iter=30, max_sub=30, cutoff=1e-14, noise=0.0):
        """One-site sweep: forward over sites 0..n-1 (left split and move right after each
        site but the last), backward over sites n-1..0 (right split and move left after
        each site but site 0).  Without noise a split can keep at most the rank of psi's
        matricisation, so bond dimensions never grow; the perturbative noise lets them grow
        up to M."""
        n = self.n
        self.to_one_site(M, cutoff)
        dws = []
        for i in range(0, n):
            self.optimise1(i, tol, max_iter, max_sub)
            if i < n - 1:
                dws.append(self.move_right1(i, M, cutoff, noise))
        for i in range(n - 1, -1, -1):
            e = self.optimise1(i, tol, max_iter, max_sub)
            if i > 0:
                dws.append(self.move_left1(i, M, cutoff, noise))
        return e, max(dws) if dws else 0.0


class StateAveragedDMRG(DMRG):
    """State-averaged two-site DMRG (Sec. 2.1.3 (i)): one set of site tensors for k states,
    the centre carrying one wavefunction per state.  Each window solves for the k lowest
    eigenpairs (davidson_roots) and splits with the averaged density matrix
    rho = sum_j w_j psi_j psi_j^T (equal weights w_j = 1/k), every state then projected
    onto the kept basis.  The average is an ordinary split of the k states stacked along the
    discarded side, each scaled by sqrt(w_j): rows (l, s1) see X = [sqrt(w_j) X_j]_j.  The
    states beyond the first start from the MPS's own psi completed by davidson_roots' rule.
    Two-site sweeps only (the one-site schedule of the base class is not offered here)."""

    def __init__(self, mpo, bonds, sites, n_roots, center=0):
        super().__init__(mpo, bonds, sites, center)
        self.k = n_roots
        self.psis = [self.psi] + [np.zeros_like(self.psi) for _ in range(n_roots - 1)]

    def optimise(self, i, tol, max_iter, max_sub):
        h = self.heff(i)
        ql = self.lab[i][:, None, None, None, :] + SITE_Q[None, :, None, None, :] + \
            SITE_Q[None, None, :, None, :]
        allowed = np.all(ql == self.lab[i + 2][None, None, None, :, :], axis=-1)
        es, psis, nmv, rn2 = davidson_roots(h.apply, h.diag(), self.psis, tol, max_iter, max_sub,
                                            allowed)
        self.psis = psis
        self.stats.append({"window": i, "energies": es, "energy": es[0], "n_matvec": nmv,
                           "resid2": rn2})
        return es

    def sweep(self, M, tol=1e-10, max_iter=100, max_sub=40, cutoff=1e-14, noise=0.0):
        n = self.n
        dws = []
        for i in range(0, n - 1):
            es = self.optimise(i, tol, max_iter, max_sub)
            if i < n - 2:
                dws.append(self._split(i, M, cutoff, noise, forward=True))
        for i in range(n - 2, -1, -1):
            es = self.optimise(i, tol, max_iter, max_sub)
            if i > 0:
                dws.append(self._split(i, M, cutoff, noise, forward=False))
        return es, max(dws) if dws else 0.0

    def _split(self, i, M, cutoff, noise, forward):
        """Averaged split of window i and the next guesses of every state."""
        k, w = self.k, np.sqrt(1.0 / self.k)
        ml, _, _, mr = self.psis[0].shape
        m = self.mpo
        if forward:
            X = np.concatenate([w * p for p in self.psis], axis=3)        # (ml, 4, 4, k mr)
            lab_stack = np.concatenate([self.lab[i + 2]] * k)
            N = None
            if noise > 0:
                N = noise_left(X.reshape(ml, 4, -1), self.L[i], m.W[i], parity_of(self.lab[i]),
                               m.parity[i], m.parity[i + 1])
            A, C, lab, dw = left_split(X, self.lab[i], M, cutoff, N, noise, lab_stack)
            self.A[i] = A
            self.lab[i + 1] = lab
            self.L[i + 1] = left_env_update(self.L[i], A, m.W[i], self.lab[i], len(m.chans[i + 1]))
            self.psis = [np.einsum("asb,btc->astc", C[:, :, j * mr:(j + 1) * mr] / w, self.A[i + 2])
                         for j in range(k)]
        else:
            X = np.concatenate([w * p for p in self.psis], axis=0)        # (k ml, 4, 4, mr)
            lab_stack = np.concatenate([self.lab[i]] * k)
            N = None
            if noise > 0:
                N = noise_right(X.reshape(-1, 4, mr), self.R[i + 2], m.W[i + 1], m.parity[i + 2])
            B, C, lab, dw = right_split(X, self.lab[i + 2], M, cutoff, N, noise, lab_stack)
            self.A[i + 1] = B
            self.lab[i + 1] = lab
            self.R[i + 1] = right_env_update(self.R[i + 2], B, m.W[i + 1], m.parity[i + 2],
                                             len(m.chans[i + 1]))
            self.psis = [np.einsum("asb,btc->astc", self.A[i - 1], C[j * ml:(j + 1) * ml] / w)
                         for j in range(k)]
        self.psi = self.psis[0]
        return dw

    def run(self, bond_dims, tol=1e-10, max_iter=100, max_sub=40, cutoff=1e-14, noise=None):
        out = []
        for k_, M in enumerate(bond_dims):
            es, _ = self.sweep(M, tol, max_iter, max_sub, cutoff,
                               0.0 if noise is None else noise[k_])
            out.append(es)
        return out


# ------------------------------------------------------------------------------------ TDVP
def tdvp_step(d, tau, M, cutoff=1e-14, tol=1e-12, max_k=40):
    """One second-order step of imaginary-time two-site TDVP (the projector-splitting
    integrator, Haegeman et al. 2016; Sec. 2.7.3 lists TDVP among the paper's dynamics
    methods, its H_eff product reused inside a Krylov exponential) on the two-site DMRG
    state d (centre: the two-site psi of window (0, 1)): psi(tau) ~ exp(-tau H) psi(0).

    Forward half (tau/2): for windows i = 0..n-2, psi <- exp(-tau/2 H2_i) psi; unless i is
    the last window, split it (A_i left-orthonormal, truncated to M like a sweep split),
    evolve the one-site remainder at site i+1 backwards, C <- exp(+tau/2 H1_{i+1}) C, and
    contract it with A_{i+2} for the next window.  Backward half (tau/2): windows n-2..0
    mirrored (B_{i+1}, C at site i evolved backwards, A_{i-1} . C).  Every local result is
    normalised (imaginary time does not keep the norm; only the direction is wanted).
    Returns the energy <psi|H|psi> at window 0 after the step and the largest discarded
    weight."""
    n = d.n
    m = d.mpo
    unit = lambda x: x / np.linalg.norm(x)
    dws = []
    for i in range(0, n - 1):
        h = d.heff(i)
        d.psi = unit(krylov_exp(h.apply, d.psi, 0.5 * tau, tol, max_k))
        if i < n - 2:
            A, C, lab, dw = left_split(d.psi, d.lab[i], M, cutoff)
            dws.append(dw)
            d.A[i] = A
            d.lab[i + 1] = lab
            d.L[i + 1] = left_env_update(d.L[i], A, m.W[i], d.lab[i], len(m.chans[i + 1]))
            h1 = Heff1(m, i + 1, d.L[i + 1], d.R[i + 2], d.lab[i + 1])
            C = unit(krylov_exp(h1.apply, C, -0.5 * tau, tol, max_k))
            d.psi = np.einsum("asb,btc->astc", C, d.A[i + 2])
    for i in range(n - 2, -1, -1):
        h = d.heff(i)
        d.psi = unit(krylov_exp(h.apply, d.psi, 0.5 * tau, tol, max_k))
        if i > 0:
            B, C, lab, dw = right_split(d.psi, d.lab[i + 2], M, cutoff)
            dws.append(dw)
            d.A[i + 1] = B
            d.lab[i + 1] = lab
            d.R[i + 1] = right_env_update(d.R[i + 2], B, m.W[i + 1], m.parity[i + 2],
                                          len(m.chans[i + 1]))
            h1 = Heff1(m, i, d.L[i], d.R[i + 1], d.lab[i])
            C = unit(krylov_exp(h1.apply, C, -0.5 * tau, tol, max_k))
            d.psi = np.einsum("asb,btc->astc", d.A[i - 1], C)
    e = float(np.vdot(d.psi, d.heff(0).apply(d.psi)))
    return e, max(dws) if dws else 0.0
