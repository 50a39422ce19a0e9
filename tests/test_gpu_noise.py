"""Perturbative noise in the sweeps' splits (b2_sweep_opts.noise) against the oracle.

Same schedules on both sides; the noise changes which states a split keeps, so matching
energies (1e-9 per sweep) and bond dimensions show that the noise density matrix is the
oracle's."""
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


SCHEDULES = [
    ("two_site", [2, 2, 2], [24, 24, 24], [1e-3, 1e-5, 0.0]),
    ("one_site_growth", [1, 1, 1, 1], [20, 20, 20, 20], [1e-3, 1e-4, 1e-5, 0.0]),
    ("mixed", [2, 1, 1, 2], [20, 20, 20, 20], [1e-4, 1e-4, 0.0, 0.0]),
]


@pytest.mark.parametrize("name,dots,Ms,noise", SCHEDULES, ids=[x[0] for x in SCHEDULES])
@pytest.mark.parametrize("kind,n,M0,seed", [("ab_initio", 8, 6, 91), ("hubbard", 10, 4, 92)],
                         ids=["abinitio_n8", "hubbard_L10"])
def test_noise_sweeps_vs_oracle(ctx, name, dots, Ms, noise, kind, n, M0, seed):
    h, eri, bonds, sites = _case(kind, n, M0, seed)
    ref = dmrg.DMRG(mpo.MPO(h, eri), bonds, sites)
    es_ref = ref.run(Ms, dots=dots, noise=noise)
    m = b2.b2_build_mpo(ctx, h, eri, 0.0, n, 0)
    s = b2.b2_mps_import(ctx, bonds, sites, n, 0, center=0)
    env = b2.b2_env_init(ctx, m, s, center=0)
    res = b2.b2_sweep(ctx, m, s, env, Ms, dots=dots, noise=noise)
    es = [r["energy"] for r in res]
    assert np.abs(np.array(es) - np.array(es_ref)).max() < 1e-9, (es, es_ref)
    bonds2, sites2, center = b2.b2_mps_export(ctx, s)
    assert [sum(x[2] for x in b) for b in bonds2] == [len(l) for l in ref.lab]
    if name == "one_site_growth":       # the noise grew the bonds of one-site sweeps
        assert max(len(l) for l in ref.lab) > max(sum(x[2] for x in b) for b in bonds)
    assert min(es) >= fci.fci_ground_state(h, eri, n, 0)[0] - 1e-10
    b2.b2_free_env(env)
    b2.b2_free_mps(s)
    b2.b2_free_mpo(m)


def test_noise_rejected_where_unsupported(ctx):
    h, eri, bonds, sites = _case("ab_initio", 6, 8, 93)
    m = b2.b2_build_mpo(ctx, h, eri, 0.0, 6, 0)
    s = b2.b2_mps_import(ctx, bonds, sites, 6, 0)
    env = b2.b2_env_init(ctx, m, s)
    with pytest.raises(b2.B2Error) as ei:
        b2.b2_sweep(ctx, m, s, env, [8], noise=[-1.0])
    assert ei.value.code == b2.B2_EINVAL
    b2.b2_free_env(env)
    b2.b2_free_mps(s)
    b2.b2_free_mpo(m)
