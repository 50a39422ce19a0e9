"""Pins of the oracle's one-site algorithm (Sec. 2.1.2: the d = 4 window of one site, and
sweeps that mix one-site and two-site windows) against the dense Fock-space Hamiltonian,
exact diagonalisation and the variational principle."""
import numpy as np

from oracle import dmrg, fci, mpo
from synth import ab_initio_integrals, hubbard_integrals, occupancies, random_mps, sector_sizes


def _problem(n, M, seed, n_elec=None, kind="ab_initio"):
    n_elec = n if n_elec is None else n_elec
    if kind == "ab_initio":
        h, eri = ab_initio_integrals(n, seed=seed)
    else:
        h, eri = hubbard_integrals(n, 1.0, 4.0)
    bonds = sector_sizes(n, n_elec, 0, M, occupancies(n, n_elec, kind))
    sites = random_mps(bonds, seed=seed + 100)
    return h, eri, bonds, sites


def _basis(As, side):
    if side == "left":
        v = np.ones((1, 1))
        for A in As:
            v = np.einsum("fl,lsr->fsr", v, A).reshape(-1, A.shape[2])
        return v
    v = np.ones((1, 1))
    for A in reversed(As):
        v = np.einsum("lsr,rf->lsf", A, v).reshape(A.shape[0], -1)
    return v


def _mps_energy(d, Hd):
    """<Psi|H|Psi> / <Psi|Psi> of the full MPS with the one-site centre psi at site 0."""
    v = _basis([d.psi] + d.A[1:], "left")[:, 0]
    return float(v @ (Hd @ v)) / float(v @ v)


def test_heff1_matches_projected_hamiltonian():
    """Y = P^T H P psi, P = (left block states) (x) 1_4 (x) (right block states) in the
    full Fock space with the dense FCI Hamiltonian: the definition of the one-site H_eff."""
    n = 6
    h, eri, bonds, sites = _problem(n, 16, 21)
    d = dmrg.DMRG(mpo.MPO(h, eri), bonds, sites)
    d.to_one_site(16, 1e-14)
    for i in range(2):
        d.optimise1(i, 1e-10, 30, 30)
        d.move_right1(i, 16, 1e-14)
    i = 2
    Lv = _basis(d.A[:i], "left")
    Rv = _basis(d.A[i + 1:], "right")
    Hd = mpo.MPO(h, eri, kind="trie").dense()
    rng = np.random.default_rng(4)
    psi = rng.standard_normal(d.psi.shape) * (d.psi != 0)
    P = np.einsum("fl,st,rg->fsgltr", Lv, np.eye(4), Rv).reshape(4 ** n, -1)
    y_ref = P.T @ (Hd @ (P @ psi.reshape(-1)))
    y = d.heff1(i).apply(psi).reshape(-1)
    assert np.abs(y - y_ref).max() < 1e-12 * max(1.0, np.abs(y_ref).max())
    # with a fermion-odd left block: site 3 sits right of an odd number of electrons in
    # some left states, so the parity signs of Heff1 are exercised
    assert (d.lab[i][:, 0] % 2 == 1).any()


def test_heff1_hermitian_and_diagonal():
    h, eri, bonds, sites = _problem(7, 24, 31, n_elec=6)
    d = dmrg.DMRG(mpo.MPO(h, eri), bonds, sites)
    d.to_one_site(24, 1e-14)
    for i in range(3):
        d.optimise1(i, 1e-10, 30, 30)
        d.move_right1(i, 24, 1e-14)
    H = d.heff1(3)
    rng = np.random.default_rng(1)
    mask = d.psi != 0
    x = rng.standard_normal(mask.shape) * mask
    yv = rng.standard_normal(mask.shape) * mask
    hx, hy = H.apply(x), H.apply(yv)
    assert abs(np.vdot(yv, hx) - np.vdot(hy, x)) < 1e-13 * np.linalg.norm(hx) * np.linalg.norm(yv)
    dg = H.diag()
    idx = np.argwhere(mask)
    for k in rng.choice(len(idx), 20, replace=False):
        e = np.zeros(mask.shape)
        e[tuple(idx[k])] = 1.0
        assert abs(H.apply(e)[tuple(idx[k])] - dg[tuple(idx[k])]) < 1e-12
    # the one-site H_eff is the two-site one restricted to psi = C . A_{i+1}: for the same
    # environments, <x|H1|y> = <x A|H2|y A> with A the (right-orthonormal) next site
    A = d.A[4]
    H2 = dmrg.Heff(d.mpo, 3, d.L[3], d.R[5], d.lab[3])
    x2 = np.einsum("asb,btc->astc", x, A)
    y2 = np.einsum("asb,btc->astc", yv, A)
    assert abs(np.vdot(x2, H2.apply(y2)) - np.vdot(x, H.apply(yv))) < 1e-12 * np.abs(hx).max()


def test_one_site_sweep_holds_exact_state():
    """At the exact bond dimension a two-site sweep reaches FCI; switching to one-site
    sweeps (split of the window-(0, 1) psi, then one-site windows) must keep it there, and
    the MPS they leave is the FCI state (its Fock-space energy)."""
    n = 6
    h, eri, bonds, sites = _problem(n, 64, 51)
    e_fci, _, _ = fci.fci_ground_state(h, eri, n, 0)
    d = dmrg.DMRG(mpo.MPO(h, eri), bonds, sites)
    es = d.run([64, 64, 64], dots=[2, 1, 1])
    assert abs(es[0] - e_fci) < 1e-9
    assert all(abs(e - e_fci) < 1e-9 for e in es[1:])
    assert all(abs(s["energy"] - e_fci) < 1e-9 for s in d.stats if s.get("dot") == 1)
    Hd = mpo.MPO(h, eri, kind="trie").dense()
    assert abs(_mps_energy(d, Hd) - e_fci) < 1e-9


def test_one_site_sweeps_variational_monotone_no_growth():
    """Truncated: every one-site sweep lowers the energy (its splits only rotate psi, no
    state with weight is dropped), stays above FCI, keeps every bond's dimension, and the
    reported energy is the expectation value of the whole MPS in the Fock space."""
    n = 6
    h, eri, bonds, sites = _problem(n, 8, 52)
    e_fci, _, _ = fci.fci_ground_state(h, eri, n, 0)
    Hd = mpo.MPO(h, eri, kind="trie").dense()
    d = dmrg.DMRG(mpo.MPO(h, eri), bonds, sites)
    dims0 = [len(l) for l in d.lab]
    es = []
    for _ in range(4):
        e, dw = d.sweep1(8)
        es.append(e)
        assert dw < 1e-12
        assert all(len(a) <= b for a, b in zip(d.lab, dims0))
        assert abs(_mps_energy(d, Hd) - e) < 1e-10
    assert all(len(a) <= b for a, b in zip(d.lab, dims0))
    assert es[-1] >= e_fci - 1e-10
    assert all(b <= a + 1e-10 for a, b in zip(es, es[1:]))


def test_mixed_two_then_one_site():
    """Two-site sweeps grow and rotate the bonds; the switch splits the window-(0, 1) psi
    with truncation to M; one-site sweeps then lower the energy at fixed bonds (their
    energies are those of the whole MPS) and the run switches back.  A two-site energy is
    that of the untruncated window, so no order holds across a switch."""
    n = 6
    h, eri, bonds, sites = _problem(n, 4, 61, kind="hubbard")
    e_fci, _, _ = fci.fci_ground_state(h, eri, n, 0)
    Hd = mpo.MPO(h, eri, kind="trie").dense()
    d = dmrg.DMRG(mpo.MPO(h, eri), bonds, sites)
    es = d.run([8, 8], dots=[2, 2])
    dims = [len(l) for l in d.lab]
    one = []
    for _ in range(2):
        e, dw = d.sweep1(8)
        one.append(e)
        assert dw < 1e-12
        assert abs(_mps_energy(d, Hd) - e) < 1e-10
        assert max(len(l) for l in d.lab) <= 8
    assert all(len(a) <= b for a, b in zip(d.lab, dims))   # one-site sweeps never grow
    assert one[1] <= one[0] + 1e-10
    es += one + d.run([8], dots=[2])
    assert min(es) >= e_fci - 1e-10
    assert d.stats[-1].get("dot") is None and sum(s.get("dot") == 1 for s in d.stats) == 4 * n
