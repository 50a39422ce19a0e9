"""Pins of the oracle's Krylov exponential and imaginary-time two-site TDVP against dense
matrix exponentials of the Fock-space Hamiltonian."""
import numpy as np
import scipy.linalg as sla

from oracle import dmrg, fci, mpo
from synth import ab_initio_integrals, hubbard_integrals, occupancies, random_mps, sector_sizes


def test_krylov_exp_matches_expm():
    rng = np.random.default_rng(0)
    for n, t in ((30, 0.3), (200, 0.05), (200, 2.0), (5, 1.0)):
        a = rng.standard_normal((n, n))
        H = a + a.T + np.diag(np.linspace(-5, 5, n))
        x = rng.standard_normal(n)
        y = dmrg.krylov_exp(lambda v: H @ v, x, t, 1e-13, 80)
        ref = sla.expm(-t * H) @ x
        assert np.linalg.norm(y - ref) <= 1e-10 * np.linalg.norm(ref)
    # an invariant subspace of dimension 3 ends the iteration exactly
    H = np.diag([1.0, 2.0, 3.0] + [7.0] * 20)
    x = np.zeros(23)
    x[:3] = 1.0
    y = dmrg.krylov_exp(lambda v: H @ v, x, 0.7, 1e-13, 40)
    assert np.linalg.norm(y - sla.expm(-0.7 * H) @ x) < 1e-13


def _fock_state(d):
    """The state of the two-site centre psi of window (0, 1) and sites 2.. in the Fock
    space (site 0 most significant; the two-site index s1 s2 is 4 s1 + s2)."""
    v = np.ones((1, 1))
    for A in [d.psi.reshape(d.psi.shape[0], 16, -1)] + d.A[2:]:
        v = np.einsum("fl,lsr->fsr", v, A).reshape(-1, A.shape[2])
    return v[:, 0]


def test_tdvp_full_bonds_is_exact_evolution():
    """With complete bond spaces nothing is truncated and the projector-splitting
    integrator reproduces exp(-tau H) psi(0) exactly (up to the Krylov tolerance)."""
    n = 4
    h, eri = ab_initio_integrals(n, seed=13)
    bonds = sector_sizes(n, n, 0, 64, occupancies(n, n, "ab_initio"))
    sites = random_mps(bonds, seed=113)
    d = dmrg.DMRG(mpo.MPO(h, eri), bonds, sites)
    Hd = mpo.MPO(h, eri, kind="trie").dense()
    v0 = _fock_state(d)
    tau = 0.2
    for step in range(3):
        e, dw = dmrg.tdvp_step(d, tau, 64)
        ref = sla.expm(-(step + 1) * tau * Hd) @ v0
        ref /= np.linalg.norm(ref)
        v = _fock_state(d)
        assert min(np.linalg.norm(v - ref), np.linalg.norm(v + ref)) < 1e-9
        assert abs(e - ref @ Hd @ ref) < 1e-9


def test_tdvp_long_imaginary_time_reaches_ground_state():
    n = 6
    h, eri = hubbard_integrals(n, 1.0, 4.0)
    bonds = sector_sizes(n, n, 0, 64, occupancies(n, n, "hubbard"))
    sites = random_mps(bonds, seed=7)
    e0 = fci.fci_ground_state(h, eri, n, 0)[0]
    _, H = fci.fci_hamiltonian(h, eri, n, 0)
    lam = np.linalg.eigvalsh(H.toarray())
    d = dmrg.DMRG(mpo.MPO(h, eri), bonds, sites)
    tau = 1.0
    es = [dmrg.tdvp_step(d, tau, 64)[0] for _ in range(25)]
    assert all(b <= a + 1e-9 for a, b in zip(es, es[1:]))     # imaginary time lowers E
    assert abs(es[-1] - e0) < 1e-8
    # the excited-state admixture decays as exp(-2 (E1 - E0) tau) per step
    err = np.array(es) - e0
    ratio = err[12] / err[11]
    assert abs(ratio - np.exp(-2 * (lam[1] - lam[0]) * tau)) < 0.05
