"""State-averaged two-site sweeps (b2_sweep_opts.n_roots, Sec. 2.1.3 (i)) against the
oracle's StateAveragedDMRG and the FCI spectrum.

Both sides converge every root of every window (|r_j|^2 <= 1e-10 within the product
limit), so the roots do not depend on start vectors or iteration paths; per-sweep root
energies agree to 1e-8 (the same bound as the oracle's own exact-M pin)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from oracle import dmrg, fci, mpo  # noqa: E402
from paper_2310_03920_gb300 import b2  # noqa: E402
from synth import (ab_initio_integrals, hubbard_integrals, occupancies, random_mps,  # noqa: E402
                   sector_sizes)


@pytest.fixture(scope="module")
def ctx():
    c = b2.Context(0)
    yield c
    c.close()


def _case(kind, n, M0, seed):
    h, eri = hubbard_integrals(n, 1.0, 4.0) if kind == "hubbard" else ab_initio_integrals(n, seed=seed)
    bonds = sector_sizes(n, n, 0, M0, occupancies(n, n, kind))
    sites = random_mps(bonds, seed=seed + 100)
    return h, eri, bonds, sites


def _fci_lowest(h, eri, n, k):
    """The k lowest FCI eigenvalues of the (N = n, S_z = 0) sector (sparse Lanczos above a
    few thousand determinants)."""
    import scipy.sparse.linalg as sla
    _, H = fci.fci_hamiltonian(h, eri, n, 0)
    if H.shape[0] <= 6000:
        return np.linalg.eigvalsh(H.toarray())[:k]
    return np.sort(sla.eigsh(H, k=k, which="SA", tol=1e-12)[0])


def _run(ctx, h, eri, n, bonds, sites, Ms, k, noise=None):
    m = b2.b2_build_mpo(ctx, h, eri, 0.0, n, 0)
    s = b2.b2_mps_import(ctx, bonds, sites, n, 0, center=0)
    env = b2.b2_env_init(ctx, m, s, center=0)
    res = b2.b2_sweep(ctx, m, s, env, Ms, dav_max_iter=400, max_subspace=40, n_roots=k, noise=noise)
    bonds2, _, _ = b2.b2_mps_export(ctx, s)
    b2.b2_free_env(env)
    b2.b2_free_mps(s)
    b2.b2_free_mpo(m)
    return res, bonds2


@pytest.mark.parametrize("kind,n,M0,seed,k,Ms", [
    ("ab_initio", 8, 8, 95, 3, [16, 16, 24]),
    ("hubbard", 10, 6, 96, 4, [20, 20]),
], ids=["abinitio_n8_k3", "hubbard_L10_k4"])
def test_state_averaged_sweeps_vs_oracle(ctx, kind, n, M0, seed, k, Ms):
    h, eri, bonds, sites = _case(kind, n, M0, seed)
    ref = dmrg.StateAveragedDMRG(mpo.MPO(h, eri), bonds, sites, k)
    es_ref = ref.run(Ms, max_iter=400, max_sub=40)
    res, bonds2 = _run(ctx, h, eri, n, bonds, sites, Ms, k)
    es = [r["root_energy"] for r in res]
    assert np.abs(np.array(es) - np.array(es_ref)).max() < 1e-8, (es, es_ref)
    assert [sum(x[2] for x in b) for b in bonds2][2:] == [len(l) for l in ref.lab][2:]
    lam = _fci_lowest(h, eri, n, k)
    assert all(e >= l - 1e-10 for e, l in zip(es[-1], lam))   # Poincare upper bounds


def test_state_averaged_exact_bonds_give_fci_spectrum(ctx):
    n, k = 6, 3
    h, eri, bonds, sites = _case("ab_initio", n, 64, 51)
    res, _ = _run(ctx, h, eri, n, bonds, sites, [64] * 3, k)
    lam = _fci_lowest(h, eri, n, k)
    assert np.abs(np.array(res[-1]["root_energy"]) - lam).max() < 1e-8


def test_state_averaged_with_noise_vs_oracle(ctx):
    h, eri, bonds, sites = _case("hubbard", 8, 4, 97)
    Ms, noise, k = [16, 16, 16], [1e-4, 1e-6, 0.0], 2
    ref = dmrg.StateAveragedDMRG(mpo.MPO(h, eri), bonds, sites, k)
    es_ref = ref.run(Ms, max_iter=400, max_sub=40, noise=noise)
    res, _ = _run(ctx, h, eri, 8, bonds, sites, Ms, k, noise=noise)
    es = [r["root_energy"] for r in res]
    assert np.abs(np.array(es) - np.array(es_ref)).max() < 1e-8, (es, es_ref)


def test_state_averaging_rejects_unsupported(ctx):
    h, eri, bonds, sites = _case("ab_initio", 6, 8, 98)
    m = b2.b2_build_mpo(ctx, h, eri, 0.0, 6, 0)
    s = b2.b2_mps_import(ctx, bonds, sites, 6, 0)
    env = b2.b2_env_init(ctx, m, s)
    for kw, code in (({"n_roots": 2, "prec": b2.B2_BF16X3}, b2.B2_EUNSUPPORTED),
                     ({"n_roots": 2, "dots": [1]}, b2.B2_EUNSUPPORTED),
                     ({"n_roots": 17}, b2.B2_EINVAL)):
        with pytest.raises(b2.B2Error) as ei:
            b2.b2_sweep(ctx, m, s, env, [8], **kw)
        assert ei.value.code == code
    b2.b2_free_env(env)
    b2.b2_free_mps(s)
    b2.b2_free_mpo(m)
