"""Pins of the oracle's perturbative noise (Sec. 2.1.6 names it; White 2005): the
system/environment factorisation it is built on, its normalisation and its effect on the
bond dimension and the energy."""
import numpy as np

from oracle import dmrg, fci, mpo
from synth import ab_initio_integrals, hubbard_integrals, occupancies, random_mps, sector_sizes


def _state(n, M, seed, kind="ab_initio", moves=2):
    if kind == "ab_initio":
        h, eri = ab_initio_integrals(n, seed=seed)
    else:
        h, eri = hubbard_integrals(n, 1.0, 4.0)
    bonds = sector_sizes(n, n, 0, M, occupancies(n, n, kind))
    sites = random_mps(bonds, seed=seed + 100)
    d = dmrg.DMRG(mpo.MPO(h, eri), bonds, sites)
    for i in range(moves):
        d.optimise(i, 1e-10, 30, 30)
        d.move_right(i, M, 1e-14)
    return h, eri, d


def test_cut_factorisation_reproduces_heff():
    """H_eff psi = sum_w E_w (S_w psi) with the cut at the window's middle bond: the
    regrouped signs of S_w and E_w are those of the (independently pinned) H_eff."""
    h, eri, d = _state(8, 24, 11)
    i = 2
    m = d.mpo
    psi = np.random.default_rng(2).standard_normal(d.psi.shape) * (d.psi != 0)
    ml, _, _, mr = psi.shape
    S = dmrg.system_left(psi.reshape(ml, 4, 4 * mr), d.L[i], m.W[i], dmrg.parity_of(d.lab[i]),
                         m.parity[i], m.parity[i + 1])
    y = np.zeros(psi.shape)
    for w, t in S.items():
        Ww = {k: v for k, v in m.W[i + 1].items() if k[0] == w}
        E = dmrg.system_right(t.reshape(ml * 4, 4, mr), d.R[i + 2], Ww, m.parity[i + 2])
        y += E[w].reshape(psi.shape)
    ref = d.heff(i).apply(psi)
    assert np.abs(y - ref).max() < 1e-12 * np.abs(ref).max()
    # and at the one-site window's right bond: sum_w P_w(S) contracted with R_w
    R1 = dmrg.right_env_update(d.R[i + 2], d.A[i + 1], m.W[i + 1], m.parity[i + 2],
                               len(m.chans[i + 1]))
    # one-site window of site i on bonds (i, i+1): a psi on those bonds
    mr1 = R1[0].shape[0]
    psi1 = np.random.default_rng(4).standard_normal((ml, 4, mr1))
    mask = (d.lab[i][:, None, None, :] + dmrg.SITE_Q[None, :, None, :])
    lab1 = d.lab[i + 1]
    ok = np.all(mask[:, :, 0, None, :] == lab1[None, None, :, :], axis=-1)
    psi1 = psi1 * ok
    S1 = dmrg.system_left(psi1, d.L[i], m.W[i], dmrg.parity_of(d.lab[i]), m.parity[i],
                          m.parity[i + 1])
    y1 = sum(t @ R1[w].T for w, t in S1.items())
    ref1 = dmrg.Heff1(m, i, d.L[i], R1, d.lab[i]).apply(psi1)
    assert np.abs(y1 - ref1).max() < 1e-12 * np.abs(ref1).max()


def test_noise_matrix_is_gram_and_normalised():
    h, eri, d = _state(6, 16, 12)
    i = 2
    m = d.mpo
    ml, _, _, mr = d.psi.shape
    N = dmrg.noise_left(d.psi.reshape(ml, 4, 4 * mr), d.L[i], m.W[i], dmrg.parity_of(d.lab[i]),
                        m.parity[i], m.parity[i + 1])
    assert np.allclose(N, N.T, atol=1e-12 * np.abs(N).max())
    assert np.linalg.eigvalsh(N).min() > -1e-10 * np.abs(N).max()
    X = d.psi.reshape(ml * 4, 4 * mr)
    row_lab = (d.lab[i][:, None, :] + dmrg.SITE_Q[None, :, :]).reshape(-1, 2)
    allowed = {tuple(q) for q in (d.lab[i + 2][None, :, :] - dmrg.SITE_Q[:, None, :]).reshape(-1, 2)}
    rho = dmrg._add_noise(X, row_lab, allowed, N, 1e-3)
    assert abs(np.trace(rho) - (np.sum(X * X) + 1e-3)) < 1e-12
    # rows whose sector the bond cannot hold get nothing
    bad = np.array([tuple(q) not in allowed for q in row_lab])
    if bad.any():
        assert not rho[bad].any()


def test_noise_grows_one_site_bonds_and_lowers_energy():
    """One-site sweeps from a small-bond MPS: without noise the bonds stay put; with noise
    they grow towards M and the energy drops below the noiseless one; every energy is
    variational (above FCI)."""
    n = 6
    h, eri = hubbard_integrals(n, 1.0, 4.0)
    bonds = sector_sizes(n, n, 0, 3, occupancies(n, n, "hubbard"))
    sites = random_mps(bonds, seed=7)
    e_fci = fci.fci_ground_state(h, eri, n, 0)[0]
    d0 = dmrg.DMRG(mpo.MPO(h, eri), bonds, sites)
    e0 = d0.run([16] * 3, dots=[1] * 3)
    d1 = dmrg.DMRG(mpo.MPO(h, eri), bonds, sites)
    e1 = d1.run([16] * 4, dots=[1] * 4, noise=[1e-3, 1e-4, 1e-5, 0.0])
    dims0 = [len(l) for l in d0.lab]
    dims1 = [len(l) for l in d1.lab]
    assert dims0 == [sum(b[2] for b in bb) for bb in bonds]
    assert max(dims1) > max(dims0) and max(dims1) <= 16
    assert e1[-1] < e0[-1] - 1e-6
    assert min(e0 + e1) >= e_fci - 1e-10


def test_two_site_noise_then_clean_reaches_fci():
    """Noise in the early sweeps of an exact-M two-site run does not spoil the end: the
    noiseless final sweeps reach FCI."""
    n = 6
    h, eri = ab_initio_integrals(n, seed=51)
    bonds = sector_sizes(n, n, 0, 8, occupancies(n, n, "ab_initio"))
    sites = random_mps(bonds, seed=151)
    e_fci = fci.fci_ground_state(h, eri, n, 0)[0]
    d = dmrg.DMRG(mpo.MPO(h, eri), bonds, sites)
    es = d.run([64] * 4, noise=[1e-2, 1e-4, 0.0, 0.0])
    assert abs(es[-1] - e_fci) < 1e-9
