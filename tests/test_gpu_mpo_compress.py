"""A compressed MPO (b2_mpo_compress, Sec. 2.3) on the GPU path: H_eff and sweeps against
the oracle's exact MPO, within the compression's tolerance."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from oracle import dmrg, mpo  # noqa: E402
from paper_2310_03920_gb300 import b2  # noqa: E402
from synth import ab_initio_integrals, occupancies, random_mps, sector_sizes  # noqa: E402
from tests.helpers import dense_to_layout, layout_to_dense  # noqa: E402

DEV = torch.device("cuda", 0)


@pytest.fixture(scope="module")
def ctx():
    c = b2.Context(0)
    yield c
    c.close()


def _case(n=8, M=32, seed=5):
    h, eri = ab_initio_integrals(n, seed=seed, n_chol=4, decay=6.0)
    bonds = sector_sizes(n, n, 0, M, occupancies(n, n, "ab_initio"))
    return h, eri, bonds


@pytest.mark.parametrize("tol,bound", [(1e-10, 1e-9), (1e-2, 5e-2)], ids=["tol1e-10", "tol1e-2"])
def test_compressed_heff_vs_exact_oracle(ctx, tol, bound):
    n, c = 8, 3
    h, eri, bonds = _case()
    sites = random_mps(bonds, seed=77, center=c)
    ref = dmrg.DMRG(mpo.MPO(h, eri), bonds, sites, center=c)
    H = ref.heff(c)
    m = b2.b2_build_mpo(ctx, h, eri, 0.0, n, 0)
    d0 = b2.b2_mpo_info(m)
    b2.b2_mpo_compress(m, tol, ctx)
    assert all(a <= b for a, b in zip(b2.b2_mpo_info(m), d0))
    s = b2.b2_mps_import(ctx, bonds, sites, n, 0, center=c)
    env = b2.b2_env_init(ctx, m, s, center=c)
    table = b2.b2_psi_blocks(ctx, env, c)
    n_elem, _ = b2.b2_psi_layout(ctx, env, c)
    x = np.random.default_rng(1).standard_normal(n_elem)
    y_ref = dense_to_layout(H.apply(layout_to_dense(x, table, bonds[c], bonds[c + 2])), table,
                            bonds[c], bonds[c + 2])
    xt = torch.tensor(x, device=DEV)
    for prec, extra in ((b2.B2_FP64, 0.0), (b2.B2_BF16X3, 2e-4)):
        y = torch.empty_like(xt)
        b2.b2_heff_apply(ctx, env, c, xt, y, prec=prec)
        err = np.linalg.norm(y.cpu().numpy() - y_ref) / np.linalg.norm(y_ref)
        assert err < bound + extra, (prec, err)
    with pytest.raises(b2.B2Error) as e:       # no coefficient Jacobian after compression
        b2.b2_rdm_grad(ctx, m, s, n)
    assert e.value.code == b2.B2_EUNSUPPORTED
    b2.b2_free_env(env)
    b2.b2_free_mps(s)
    b2.b2_free_mpo(m)


def test_compressed_sweeps_reach_exact_energies(ctx):
    n = 8
    h, eri, bonds = _case(M=16)
    sites = random_mps(bonds, seed=78)
    es_ref = dmrg.DMRG(mpo.MPO(h, eri), bonds, sites).run([32] * 3)
    m = b2.b2_build_mpo(ctx, h, eri, 0.0, n, 0)
    b2.b2_mpo_compress(m, 1e-10, ctx)
    s = b2.b2_mps_import(ctx, bonds, sites, n, 0, center=0)
    env = b2.b2_env_init(ctx, m, s, center=0)
    res = b2.b2_sweep(ctx, m, s, env, [32] * 3)
    es = [r["energy"] for r in res]
    assert np.abs(np.array(es) - np.array(es_ref)).max() < 1e-8, (es, es_ref)
    b2.b2_free_env(env)
    b2.b2_free_mps(s)
    b2.b2_free_mpo(m)
