"""Imaginary-time two-site TDVP (b2_tdvp, Sec. 2.7.3) against the oracle's tdvp_step.

Same seeded MPS, same steps: the per-step energies agree to 1e-9 and the bond dimensions
exactly (the Krylov exponentials are converged to 1e-12 on both sides, so the states do not
depend on the Krylov paths); with complete bonds the oracle step is exact evolution
(pinned on the CPU against expm of the Fock-space Hamiltonian)."""
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


@pytest.mark.parametrize("kind,n,M0,M,tau,steps", [
    ("ab_initio", 4, 64, 64, 0.2, 3),
    ("ab_initio", 8, 12, 16, 0.1, 3),
    ("hubbard", 10, 8, 24, 0.25, 3),
], ids=["abinitio_n4_complete", "abinitio_n8_M16", "hubbard_L10_M24"])
def test_tdvp_vs_oracle(ctx, kind, n, M0, M, tau, steps):
    h, eri, bonds, sites = _case(kind, n, M0, 21 + n)
    ref = dmrg.DMRG(mpo.MPO(h, eri), bonds, sites)
    es_ref = [dmrg.tdvp_step(ref, tau, M)[0] for _ in range(steps)]
    m = b2.b2_build_mpo(ctx, h, eri, 0.0, n, 0)
    s = b2.b2_mps_import(ctx, bonds, sites, n, 0, center=0)
    env = b2.b2_env_init(ctx, m, s, center=0)
    res = b2.b2_tdvp(ctx, m, s, env, steps, tau, M)
    es = [r["energy"] for r in res]
    assert np.abs(np.array(es) - np.array(es_ref)).max() < 1e-9, (es, es_ref)
    assert all(r["n_matvec"] > 0 and r["matvec_flops"] > 0 for r in res)
    bonds2, sites2, center = b2.b2_mps_export(ctx, s)
    assert center == 0
    assert [sum(x[2] for x in b) for b in bonds2][2:] == [len(l) for l in ref.lab][2:]
    # the exported MPS is the evolved state: its energy is the last step's
    ref2 = dmrg.DMRG(mpo.MPO(h, eri), bonds2, sites2, center=0)
    e_state = float(np.vdot(ref2.psi, ref2.heff(0).apply(ref2.psi)) / np.vdot(ref2.psi, ref2.psi))
    assert abs(e_state - es[-1]) < 1e-9
    # imaginary time lowers the energy towards the ground state
    assert es[-1] < es[0] and es[-1] >= fci.fci_ground_state(h, eri, n, 0)[0] - 1e-10
    b2.b2_free_env(env)
    b2.b2_free_mps(s)
    b2.b2_free_mpo(m)


def test_tdvp_rejects_bad_options(ctx):
    h, eri, bonds, sites = _case("ab_initio", 6, 8, 33)
    m = b2.b2_build_mpo(ctx, h, eri, 0.0, 6, 0)
    s = b2.b2_mps_import(ctx, bonds, sites, 6, 0)
    env = b2.b2_env_init(ctx, m, s)
    for tau, M in ((0.0, 8), (-0.1, 8), (0.1, 0)):
        with pytest.raises(b2.B2Error) as ei:
            b2.b2_tdvp(ctx, m, s, env, 1, tau, M)
        assert ei.value.code == b2.B2_EINVAL
    b2.b2_free_env(env)
    b2.b2_free_mps(s)
    b2.b2_free_mpo(m)
