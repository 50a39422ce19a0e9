"""GPU integral gradient (b2_rdm_grad) and the autograd Function: against closed forms,
the oracle's density matrices of the same MPS, finite differences of the DMRG energy and
identities that hold at any size."""
import itertools

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from oracle import fci, rdm  # noqa: E402
from paper_2310_03920_gb300 import b2  # noqa: E402
from paper_2310_03920_gb300.autograd import DMRGSolver, dmrg_energy  # noqa: E402
from synth import ab_initio_integrals, hubbard_integrals  # noqa: E402

DEV = torch.device("cuda", 0)


@pytest.fixture(scope="module")
def ctx():
    c = b2.Context(0)
    yield c
    c.close()


def _product_state(occ):
    """Bond-dimension-1 MPS of the determinant with site occupations occ[k] in {0..3}."""
    q = [(0, 0), (1, 1), (1, -1), (2, 0)]
    bonds, N, tsz = [[(0, 0, 1)]], 0, 0
    for s in occ:
        N, tsz = N + q[s][0], tsz + q[s][1]
        bonds.append([(N, tsz, 1)])
    sites = [{(0, s, 0): np.ones((1, 1))} for s in occ]
    return bonds, sites, N, tsz


def test_grad_product_state_closed_form(ctx):
    occ = [3, 1, 0, 2, 3, 0, 1]
    n = len(occ)
    bonds, sites, N, tsz = _product_state(occ)
    h, eri = ab_initio_integrals(n, seed=1)
    m = b2.b2_build_mpo(ctx, h, eri, 0.0, N, tsz)
    s = b2.b2_mps_import(ctx, bonds, sites, N, tsz, center=0)
    g1, g2 = b2.b2_rdm_grad(ctx, m, s, n)
    # spin-orbital occupations: local states |0>, |a>, |b>, |ab>
    nso = np.array([[1.0 if x in (1, 3) else 0.0, 1.0 if x in (2, 3) else 0.0] for x in occ])
    eye = np.eye(n)
    ref2 = np.zeros((n, n, n, n))
    for a, b in itertools.product(range(2), repeat=2):
        ref2 += np.einsum("p,r,pq,rs->pqrs", nso[:, a], nso[:, b], eye, eye)
        if a == b:
            ref2 -= np.einsum("p,r,ps,rq->pqrs", nso[:, a], nso[:, b], eye, eye)
    assert np.abs(g1 - np.diag(nso.sum(1))).max() < 1e-14
    assert np.abs(g2 - 0.5 * ref2).max() < 1e-14
    b2.b2_free_mps(s)
    b2.b2_free_mpo(m)


@pytest.mark.parametrize("kind,n,n_elec,two_sz,M,seed", [
    ("ab_initio", 6, 6, 0, 12, 31),
    ("ab_initio", 7, 5, 1, 16, 32),
    ("hubbard", 8, 8, 0, 20, 33),
])
def test_grad_random_mps_matches_oracle(ctx, kind, n, n_elec, two_sz, M, seed):
    if kind == "hubbard":
        h, eri = hubbard_integrals(n, 1.0, 4.0)
    else:
        h, eri = ab_initio_integrals(n, seed=seed)
    m = b2.b2_build_mpo(ctx, h, eri, 0.0, n_elec, two_sz)
    s = b2.b2_mps_random(ctx, m, M, seed=seed)
    g1, g2 = b2.b2_rdm_grad(ctx, m, s, n)
    bonds, sites, center = b2.b2_mps_export(ctx, s)
    assert center == 0
    gamma, Gamma = rdm.mps_rdm12(bonds, sites, n_elec, two_sz)
    assert np.abs(g1 - gamma).max() < 1e-12
    assert np.abs(g2 - 0.5 * Gamma).max() < 1e-12
    b2.b2_free_mps(s)
    b2.b2_free_mpo(m)


def test_grad_dmrg_state_matches_oracle_and_energy(ctx):
    # n = 8 ab initio, M = 64 (a truncated MPS): the gradient is that of the MPS, and the
    # energy expression e_core + h.gamma + (1/2) eri.Gamma reproduces the sweep energy
    n = 8
    h, eri = ab_initio_integrals(n, seed=0)
    e_core = 1.25
    m = b2.b2_build_mpo(ctx, h, eri, e_core, n, 0)
    s = b2.b2_mps_random(ctx, m, 64, seed=100)
    env = b2.b2_env_init(ctx, m, s, 0)
    res = b2.b2_sweep(ctx, m, s, env, [64] * 4, conv_tol=1e-14, dav_max_iter=200, max_subspace=40)
    g1, g2 = b2.b2_rdm_grad(ctx, m, s, n)
    e_expr = e_core + np.sum(h * g1) + np.sum(eri * g2)
    assert abs(e_expr - res[-1]["energy"]) < 1e-9
    bonds, sites, _ = b2.b2_mps_export(ctx, s)
    gamma, Gamma = rdm.mps_rdm12(bonds, sites, n, 0)
    assert np.abs(g1 - gamma).max() < 1e-11
    assert np.abs(g2 - 0.5 * Gamma).max() < 1e-11
    b2.b2_free_env(env)
    b2.b2_free_mps(s)
    b2.b2_free_mpo(m)


def _sym_eri_direction(rng, n):
    x = rng.standard_normal((n, n, n, n))
    x = x + x.transpose(1, 0, 2, 3)
    x = x + x.transpose(0, 1, 3, 2)
    x = x + x.transpose(2, 3, 0, 1)
    return x / 8.0


def test_autograd_energy_gradient_fd_and_fci(ctx):
    # exact bond dimension (n = 6: 64 >= 4^3): DMRG = FCI, so the gradient is the FCI
    # density matrices and matches central differences of the forward energy
    n, n_elec = 6, 6
    h0, eri0 = ab_initio_integrals(n, seed=41)
    solver = DMRGSolver(ctx, n_elec, 0, [64] * 4, seed=5, conv_tol=1e-22, dav_max_iter=400,
                        max_subspace=40)
    h = torch.tensor(h0, requires_grad=True)
    eri = torch.tensor(eri0, requires_grad=True)
    e_core = torch.tensor(0.3, dtype=torch.float64, requires_grad=True)
    E = dmrg_energy(h, eri, e_core, solver)
    E.backward()
    e_fci, c, dets = fci.fci_ground_state(h0, eri0, n_elec, 0, 0.3)
    assert abs(E.item() - e_fci) < 1e-10
    gamma, Gamma = rdm.rdm12(dets, c, n)
    assert np.abs(h.grad.numpy() - gamma).max() < 1e-8
    assert np.abs(eri.grad.numpy() - 0.5 * Gamma).max() < 1e-8
    assert e_core.grad.item() == 1.0
    # central differences (step 1e-5) along a random symmetric direction
    rng = np.random.default_rng(7)
    dh = rng.standard_normal((n, n))
    dh = 0.5 * (dh + dh.T)
    de = _sym_eri_direction(rng, n)
    eps = 1e-5

    def energy(sign):
        return dmrg_energy(torch.tensor(h0 + sign * eps * dh), torch.tensor(eri0 + sign * eps * de),
                           0.3, solver).item()

    fd = (energy(+1) - energy(-1)) / (2 * eps)
    an = float(np.sum(h.grad.numpy() * dh) + np.sum(eri.grad.numpy() * de))
    assert abs(fd - an) < 1e-6 * max(1.0, abs(an))


def test_grad_full_size_identities(ctx):
    # n = 24 orbitals, 24 electrons, M = 500: identities that hold for any state with
    # N electrons, and E = <psi|H|psi> evaluated independently through the environments
    # and H_eff of window 0 equals e_core + h.gamma + (1/2) eri.Gamma
    n, N, M = 24, 24, 500
    h, eri = ab_initio_integrals(n, seed=24)
    e_core = 0.5
    m = b2.b2_build_mpo(ctx, h, eri, e_core, N, 0)
    s = b2.b2_mps_random(ctx, m, M, seed=124)
    g1, g2 = b2.b2_rdm_grad(ctx, m, s, n)
    Gamma = 2.0 * g2
    assert abs(np.trace(g1) - N) < 1e-9
    assert abs(np.einsum("pprr->", Gamma) - N * (N - 1)) < 1e-7
    assert np.abs(np.einsum("pqrr->pq", Gamma) - (N - 1) * g1).max() < 1e-9
    assert np.abs(g1 - g1.T).max() < 1e-11
    assert np.abs(Gamma - Gamma.transpose(2, 3, 0, 1)).max() < 1e-11
    assert np.abs(Gamma - Gamma.transpose(1, 0, 3, 2)).max() < 1e-11
    env = b2.b2_env_init(ctx, m, s, 0)
    nel, _ = b2.b2_psi_layout(ctx, env, 0)
    psi = torch.zeros(nel, dtype=torch.float64, device=DEV)
    out = torch.zeros_like(psi)
    b2.b2_psi_from_mps(ctx, env, 0, psi)
    b2.b2_heff_apply(ctx, env, 0, psi, out)
    torch.cuda.synchronize()
    e_env = float(torch.dot(psi, out) / torch.dot(psi, psi))
    e_expr = e_core + np.sum(h * g1) + np.sum(eri * g2)
    assert abs(e_env - e_expr) < 1e-9 * max(1.0, abs(e_env))
    b2.b2_free_env(env)
    b2.b2_free_mps(s)
    b2.b2_free_mpo(m)


def test_grad_n24_M500_against_oracle_transfer_matrices(ctx):
    # the gradient workload's size (n = 24, N = 24, M = 500, integrals of seed 4): the full
    # gamma and 160 elements of Gamma / 2 from b2_rdm_grad against the oracle's single-string
    # transfer-matrix contractions of the same seeded MPS (Sec. 2.5.1 definitions)
    from oracle import rdm as ordm
    from synth import config_integrals, occupancies, random_mps, sector_sizes
    h, eri, N, tsz, kind = config_integrals("abinitio_n24")
    n, M = 24, 500
    bonds = sector_sizes(n, N, tsz, M, occupancies(n, N, kind))
    sites = random_mps(bonds, seed=104, center=0)
    m = b2.b2_build_mpo(ctx, h, eri, 0.0, N, tsz)
    s = b2.b2_mps_import(ctx, bonds, sites, N, tsz, center=0)
    g1, g2 = b2.b2_rdm_grad(ctx, m, s, n)
    pairs = [(p, q) for p in range(n) for q in range(n)]
    rng = np.random.default_rng(24)
    quads = [tuple(int(v) for v in rng.integers(0, n, 4)) for _ in range(140)]
    # coinciding indices and the ends of the chain
    quads += [(0, 0, 23, 23), (23, 0, 0, 23), (5, 5, 5, 5), (11, 12, 12, 11), (3, 9, 9, 3),
              (0, 23, 23, 0), (12, 12, 13, 13), (7, 8, 9, 10), (22, 1, 2, 21), (4, 4, 4, 17),
              (17, 4, 4, 4), (1, 1, 1, 1), (20, 2, 20, 2), (2, 20, 2, 20), (10, 10, 10, 9),
              (9, 10, 10, 10), (6, 19, 13, 0), (0, 13, 19, 6), (15, 15, 16, 16), (16, 15, 15, 16)]
    g_ref, G_ref = ordm.rdm_elements_mps(bonds, sites, pairs, quads)
    assert np.abs(g1.ravel() - g_ref).max() <= 1e-11
    G_gpu = np.array([2.0 * g2[q4] for q4 in quads])
    assert np.abs(G_gpu - G_ref).max() <= 1e-11
    # the comparison is not vacuous: many sampled elements are far above the tolerance
    assert np.sum(np.abs(G_ref) > 1e-4) > 40 and np.sum(np.abs(g_ref) > 1e-2) > 24
    b2.b2_free_mps(s)
    b2.b2_free_mpo(m)
