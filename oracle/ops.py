"""Local Fock space of one spatial orbital (test infrastructure only).

Basis order and operator matrices are the ones of the paper's Listing 1, Part A:
states [|0>, |alpha>, |beta>, |alpha beta>] with quantum numbers (N, 2Sz) =
(0,0), (1,1), (1,-1), (2,0), and |alpha beta> = a+_alpha a+_beta |0>, so that
a+_beta |alpha> = -|alpha beta>.  Matrices act on column vectors (row = output state).

Globally, spin orbitals are ordered site-major with alpha before beta (mode 2p + sigma);
a product state |s_0 s_1 ... > is the ordered product of the local creation strings.
"""
import numpy as np

SITE_Q = ((0, 0), (1, 1), (1, -1), (2, 0))
SITE_N = np.array([0, 1, 1, 2])
SITE_PARITY = SITE_N % 2

# Listing 1: "c" = alpha+, "d" = alpha, "C" = beta+, "D" = beta
CRE_A = np.array([[0, 0, 0, 0], [1, 0, 0, 0], [0, 0, 0, 0], [0, 0, 1, 0]], dtype=float)
ANN_A = np.array([[0, 1, 0, 0], [0, 0, 0, 0], [0, 0, 0, 1], [0, 0, 0, 0]], dtype=float)
CRE_B = np.array([[0, 0, 0, 0], [0, 0, 0, 0], [1, 0, 0, 0], [0, -1, 0, 0]], dtype=float)
ANN_B = np.array([[0, 0, 1, 0], [0, 0, 0, -1], [0, 0, 0, 0], [0, 0, 0, 0]], dtype=float)
IDENT = np.eye(4)
# fermion parity (-1)^N of a local state
PARITY = np.diag([1.0, -1.0, -1.0, 1.0])


def elementary(sigma, dagger):
    """4x4 matrix of a+_sigma (dagger=True) or a_sigma on one site; sigma 0 = alpha, 1 = beta."""
    if sigma == 0:
        return CRE_A if dagger else ANN_A
    return CRE_B if dagger else ANN_B


def op_key(mat):
    """Hashable key of a local operator matrix whose entries are small integers."""
    r = np.rint(mat)
    assert np.array_equal(r, mat), "local operators here have integer entries"
    return tuple(int(v) for v in r.ravel())


def key_matrix(key):
    return np.array(key, dtype=float).reshape(4, 4)


def op_parity(mat):
    """Fermion parity (0 even, 1 odd) of a local operator with definite parity."""
    nz = np.argwhere(mat != 0)
    if len(nz) == 0:
        return 0
    pars = {(SITE_N[i] + SITE_N[j]) % 2 for i, j in nz}
    assert len(pars) == 1, "operator without definite parity"
    return pars.pop()


def op_dq(mat):
    """Quantum-number change (dN, d2Sz) of a local operator with definite change."""
    nz = np.argwhere(mat != 0)
    if len(nz) == 0:
        return (0, 0)
    dqs = {(SITE_Q[i][0] - SITE_Q[j][0], SITE_Q[i][1] - SITE_Q[j][1]) for i, j in nz}
    assert len(dqs) == 1, "operator without definite quantum-number change"
    return dqs.pop()
