"""Failure paths of the C-ABI, made on the host: an allocator that refuses, non-finite
integrals, and shortened device-side limits (b2_debug_limits) that run out.  Nothing here
faults, traps or hangs the GPU; after each failure the same context must keep working."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2310_03920_gb300 import b2  # noqa: E402
from synth import ab_initio_integrals, occupancies, random_mps, sector_sizes  # noqa: E402

DEV = torch.device("cuda", 0)


def _small(n=6, M=16, seed=2, center=0):
    h, eri = ab_initio_integrals(n, seed=seed)
    bonds = sector_sizes(n, n, 0, M, occupancies(n, n, "ab_initio"))
    sites = random_mps(bonds, seed=100 + seed, center=center)
    return h, eri, bonds, sites


def test_allocator_failure_returns_enomem_and_the_context_recovers():
    state = {"fail": False, "refused": 0}
    stream = torch.cuda.current_stream(0)

    def alloc(size):
        if state["fail"]:
            state["refused"] += 1
            return 0
        return torch.cuda.caching_allocator_alloc(size, 0, stream)

    def free(p):
        torch.cuda.caching_allocator_delete(p)

    ctx = b2.Context(0, alloc=alloc, free=free)
    h, eri, bonds, sites = _small()
    m = b2.b2_build_mpo(ctx, h, eri, 0.0, 6, 0)      # host work only
    state["fail"] = True
    with pytest.raises(b2.B2Error) as e:
        b2.b2_mps_import(ctx, bonds, sites, 6, 0)
    assert e.value.code == b2.B2_ENOMEM
    assert "allocator callback failed" in str(e.value)
    assert state["refused"] >= 1
    state["fail"] = False
    s = b2.b2_mps_import(ctx, bonds, sites, 6, 0)
    env = b2.b2_env_init(ctx, m, s)
    n_elem, _ = b2.b2_psi_layout(ctx, env, 0)
    x = torch.ones(n_elem, dtype=torch.float64, device=DEV)
    y = torch.empty_like(x)
    b2.b2_heff_apply(ctx, env, 0, x, y)
    torch.cuda.synchronize()
    assert torch.isfinite(y).all() and float(y.abs().sum()) > 0
    # a failure in the middle of a call that already holds memory: environments of a
    # larger centre need several allocations; refuse them, then succeed again
    state["fail"] = True
    with pytest.raises(b2.B2Error) as e:
        b2.b2_env_init(ctx, m, s, center=0)
    assert e.value.code == b2.B2_ENOMEM
    state["fail"] = False
    env2 = b2.b2_env_init(ctx, m, s, center=0)
    b2.b2_heff_apply(ctx, env2, 0, x, y)
    torch.cuda.synchronize()
    for handle, f in ((env2, b2.b2_free_env), (env, b2.b2_free_env), (s, b2.b2_free_mps),
                      (m, b2.b2_free_mpo)):
        f(handle)
    ctx.close()


@pytest.mark.parametrize("where", ["h_nan", "h_inf", "eri_nan", "eri_inf"])
def test_non_finite_integrals_are_rejected(where):
    ctx = b2.Context(0)
    h, eri = ab_initio_integrals(5, seed=1)
    bad = {"h_nan": np.nan, "h_inf": np.inf, "eri_nan": np.nan, "eri_inf": -np.inf}[where]
    if where.startswith("h"):
        h = h.copy()
        h[1, 3] = bad
    else:
        eri = eri.copy()
        eri[0, 2, 4, 1] = bad
    with pytest.raises(b2.B2Error) as e:
        b2.b2_build_mpo(ctx, h, eri, 0.0, 5, 1)
    assert e.value.code == b2.B2_EINVAL
    # the context is untouched: the clean integrals still build
    h2, eri2 = ab_initio_integrals(5, seed=1)
    b2.b2_free_mpo(b2.b2_build_mpo(ctx, h2, eri2, 0.0, 5, 1))
    ctx.close()


def test_eigensolver_sweep_limit_reports_enoconv():
    ctx = b2.Context(0)
    h, eri, bonds, sites = _small(n=6, M=24, seed=5)
    m = b2.b2_build_mpo(ctx, h, eri, 0.0, 6, 0)
    s = b2.b2_mps_import(ctx, bonds, sites, 6, 0)
    env = b2.b2_env_init(ctx, m, s)
    b2.b2_debug_limits(ctx, 0, 1)   # one Jacobi sweep: a sector of dim >= 2 cannot confirm
    with pytest.raises(b2.B2Error) as e:
        b2.b2_sweep(ctx, m, s, env, [24])
    assert e.value.code == b2.B2_ENOCONV
    assert "sweep limit" in str(e.value)
    # the MPS may be left mid-sweep: start again from the file with the default limit
    b2.b2_free_env(env)
    b2.b2_free_mps(s)
    b2.b2_debug_limits(ctx, 0, 0)
    s = b2.b2_mps_import(ctx, bonds, sites, 6, 0)
    env = b2.b2_env_init(ctx, m, s)
    r = b2.b2_sweep(ctx, m, s, env, [24, 24])
    # at a truncated bond dimension a sweep may raise the energy by about the discarded weight
    assert np.isfinite(r[-1]["energy"]) and r[-1]["energy"] <= r[0]["energy"] + 1e-6
    b2.b2_free_env(env)
    b2.b2_free_mps(s)
    b2.b2_free_mpo(m)
    ctx.close()


def test_debug_limits_reject_negative_values():
    ctx = b2.Context(0)
    with pytest.raises(b2.B2Error) as e:
        b2.b2_debug_limits(ctx, -1, 0)
    assert e.value.code == b2.B2_EINVAL
    ctx.close()


@pytest.mark.parametrize("prec", [b2.B2_BF16X3, b2.B2_TF32X3], ids=["bf16x3", "tf32x3"])
def test_tensor_core_wait_that_runs_out_reports_etimeout(prec):
    # every CTA of the contraction first waits on a barrier that nothing arrives on; the
    # bounded wait runs out, the CTA drains its copies and MMAs, frees tensor memory and
    # returns; b2_sync reports B2_ETIMEOUT and the next products are correct again
    ctx = b2.Context(0)
    h, eri, bonds, sites = _small(n=8, M=48, seed=6, center=3)
    m = b2.b2_build_mpo(ctx, h, eri, 0.0, 8, 0)
    s = b2.b2_mps_import(ctx, bonds, sites, 8, 0, center=3)
    env = b2.b2_env_init(ctx, m, s, center=3)
    n_elem, _ = b2.b2_psi_layout(ctx, env, 3)
    x = torch.randn(n_elem, dtype=torch.float64, device=DEV,
                    generator=torch.Generator(device=DEV).manual_seed(3))
    y64, ys = torch.empty_like(x), torch.empty_like(x)
    b2.b2_heff_apply(ctx, env, 3, x, y64)
    b2.b2_sync(ctx)
    b2.b2_debug_limits(ctx, 2000, 0)
    b2.b2_heff_apply(ctx, env, 3, x, ys, prec=prec)
    with pytest.raises(b2.B2Error) as e:
        b2.b2_sync(ctx)
    assert e.value.code == b2.B2_ETIMEOUT
    # the same through Davidson, which checks the status after its products
    p = x.clone()
    with pytest.raises(b2.B2Error) as e:
        b2.b2_davidson(ctx, env, 3, p, max_iter=4, prec=prec)
    assert e.value.code == b2.B2_ETIMEOUT
    b2.b2_debug_limits(ctx, 0, 0)
    b2.b2_sync(ctx)
    b2.b2_heff_apply(ctx, env, 3, x, ys, prec=prec)
    b2.b2_sync(ctx)
    assert float((ys - y64).norm() / y64.norm()) < 2e-4
    b2.b2_free_env(env)
    b2.b2_free_mps(s)
    b2.b2_free_mpo(m)
    ctx.close()
