"""The library's MPO (b2_build_mpo, host work) and its compression (b2_mpo_compress,
Sec. 2.3), checked on the CPU: the exported tensors contracted to the Fock-space Hamiltonian
equal the oracle's exact MPO; compression with tol = 0 is exact; lossy compression shrinks
the bonds and moves the ground-state energy by a controlled amount."""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as sla

from oracle import mpo as ompo
from synth import ab_initio_integrals, hubbard_integrals

b2 = pytest.importorskip("paper_2310_03920_gb300.b2")

P = np.diag([1.0, -1.0, -1.0, 1.0])


def contract(ex):
    """Fock-space matrix of an exported MPO (site 0 most significant)."""
    T = {0: sp.csr_matrix(np.ones((1, 1)))}
    for k, site in enumerate(ex["entries"]):
        new = {}
        for w, w2, m in site:
            if w not in T:
                continue
            mp = m @ P if ex["parity"][k + 1][w2] else m
            t = sp.kron(T[w], sp.csr_matrix(mp), format="csr")
            new[w2] = new[w2] + t if w2 in new else t
        T = new
    assert list(T) == [0]
    return T[0]


def sector(H, n, n_elec):
    """Rows/columns of product states with n_elec electrons and S_z = 0."""
    occ = [(0, 0), (1, 0), (0, 1), (1, 1)]
    idx = []
    for x in range(4 ** n):
        na = nb = 0
        r = x
        for _ in range(n):
            a, b = occ[r % 4]
            na += a
            nb += b
            r //= 4
        if na + nb == n_elec and na == nb:
            idx.append(x)
    idx = np.array(idx)
    return H[idx][:, idx]


def lowest(H):
    return float(sla.eigsh(H, k=1, which="SA", tol=1e-12)[0][0])


def test_library_mpo_equals_oracle_hamiltonian():
    for n, seed in ((4, 3), (6, 4)):
        h, eri = ab_initio_integrals(n, seed=seed)
        m = b2.b2_build_mpo(None, h, eri, 0.0, n, 0)
        H = contract(b2.b2_mpo_export(m))
        ref = ompo.MPO(h, eri, kind="trie").dense()
        assert abs(H - sp.csr_matrix(ref)).max() < 1e-12 * np.abs(ref).max()
        b2.b2_free_mpo(m)


def test_exact_compression_keeps_the_hamiltonian():
    n = 6
    h, eri = ab_initio_integrals(n, seed=4)
    m = b2.b2_build_mpo(None, h, eri, 0.0, n, 0)
    d0 = b2.b2_mpo_info(m)
    H0 = contract(b2.b2_mpo_export(m))
    disc = b2.b2_mpo_compress(m, 0.0)
    d1 = b2.b2_mpo_info(m)
    ex = b2.b2_mpo_export(m)
    H1 = contract(ex)
    assert all(a <= b for a, b in zip(d1, d0)) and d1[0] == 1 and d1[-1] == 1
    assert disc < 1e-7
    assert abs(H1 - H0).max() < 1e-11 * abs(H0).max()
    # compressed channels keep one parity and one quantum-number shift each: every entry
    # changes N and 2Sz by the difference of its channels' shifts
    q = {0: (0, 0), 1: (1, 1), 2: (1, -1), 3: (2, 0)}
    for k, site in enumerate(ex["entries"]):
        for w, w2, op in site:
            for so, si in zip(*np.nonzero(op)):
                dn = q[so][0] - q[si][0] + ex["dq"][k][w][0]
                dz = q[so][1] - q[si][1] + ex["dq"][k][w][1]
                assert (dn, dz) == tuple(ex["dq"][k + 1][w2])
    b2.b2_free_mpo(m)


@pytest.mark.parametrize("kind", ["ab_initio", "hubbard"])
def test_lossy_compression_shrinks_bonds_with_small_energy_error(kind):
    """tol = 1e-8 removes only numerically dependent channels (energy unchanged to 1e-10);
    tol = 1e-2 removes more (ab initio: every truncated bond no larger, fewer channels in
    total) at an energy error of the order of the discarded weight."""
    n = 6
    if kind == "hubbard":
        h, eri = hubbard_integrals(n, 1.0, 4.0)
    else:
        h, eri = ab_initio_integrals(n, seed=2, n_chol=4, decay=6.0)
    m = b2.b2_build_mpo(None, h, eri, 0.0, n, 0)
    d0 = b2.b2_mpo_info(m)
    e0 = lowest(sector(contract(b2.b2_mpo_export(m)), n, n))
    res = {}
    for tol in (1e-8, 1e-2):
        mc = b2.b2_build_mpo(None, h, eri, 0.0, n, 0)
        disc = b2.b2_mpo_compress(mc, tol)
        dc = b2.b2_mpo_info(mc)
        e = lowest(sector(contract(b2.b2_mpo_export(mc)), n, n))
        res[tol] = (dc, abs(e - e0), disc)
        b2.b2_free_mpo(mc)
    assert res[1e-8][1] < 1e-10 and res[1e-8][2] < 1e-7
    assert all(a <= b for a, b in zip(res[1e-2][0], res[1e-8][0]))
    assert all(a <= b for a, b in zip(res[1e-8][0], d0))
    assert res[1e-2][1] < 10 * res[1e-2][2] * abs(e0) + 1e-12
    if kind == "ab_initio":
        assert int(res[1e-2][0].sum()) < int(res[1e-8][0].sum())
    b2.b2_free_mpo(m)


def test_bad_tolerance_rejected():
    h, eri = ab_initio_integrals(4, seed=1)
    m = b2.b2_build_mpo(None, h, eri, 0.0, 4, 0)
    for tol in (-1.0, 1.0, float("nan")):
        with pytest.raises(b2.B2Error) as e:
            b2.b2_mpo_compress(m, tol)
        assert e.value.code == b2.B2_EINVAL
    b2.b2_free_mpo(m)
