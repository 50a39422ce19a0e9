"""Batched many-problem execution: one grouped H_eff launch over several independent
problems per Davidson iteration.  Per problem, the grouped path runs the same kernels with
the same arguments in the same order as the single-problem path, so the results must be
identical (bitwise), and the single-problem path is itself checked against the oracle."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2310_03920_gb300 import b2  # noqa: E402
from synth import (ab_initio_integrals, hubbard_integrals, occupancies, random_mps,  # noqa: E402
                   sector_sizes)

DEV = torch.device("cuda", 0)

# (integrals, electrons, kind, M, MPS seed, window): uneven sizes and both Hamiltonians
PROBLEMS = [
    (lambda: hubbard_integrals(10, 1.0, 3.0), 10, "hubbard", 40, 301, 4),
    (lambda: ab_initio_integrals(8, seed=11), 8, "ab_initio", 40, 302, 3),
    (lambda: ab_initio_integrals(9, seed=12), 8, "ab_initio", 64, 303, 0),
    (lambda: hubbard_integrals(16, 1.0, 6.0), 16, "hubbard", 120, 304, 7),
    (lambda: ab_initio_integrals(10, seed=13), 10, "ab_initio", 96, 305, 8),
]


@pytest.fixture(scope="module")
def ctx():
    c = b2.Context(0)
    yield c
    c.close()


def _make(ctx, spec, center):
    ints, n_elec, kind, M, seed, _ = spec
    h, eri = ints()
    n = h.shape[0]
    bonds = sector_sizes(n, n_elec, 0, M, occupancies(n, n_elec, kind))
    sites = random_mps(bonds, seed=seed, center=center)
    m = b2.b2_build_mpo(ctx, h, eri, 0.0, n_elec, 0)
    s = b2.b2_mps_import(ctx, bonds, sites, n_elec, 0, center=center)
    env = b2.b2_env_init(ctx, m, s, center=center)
    return m, s, env


def _free(objs):
    for m, s, env in objs:
        b2.b2_free_env(env)
        b2.b2_free_mps(s)
        b2.b2_free_mpo(m)


def _psi(ctx, env, w):
    n, _ = b2.b2_psi_layout(ctx, env, w)
    psi = torch.empty(n, dtype=torch.float64, device=DEV)
    b2.b2_psi_from_mps(ctx, env, w, psi)
    return psi


@pytest.mark.parametrize("prec", [b2.B2_FP64, b2.B2_BF16X3, b2.B2_TF32X3])
def test_grouped_heff_equals_single_problem_launches(ctx, prec):
    objs = [_make(ctx, p, p[5]) for p in PROBLEMS]
    envs = [o[2] for o in objs]
    sites = [p[5] for p in PROBLEMS]
    psis = [_psi(ctx, e, w) for e, w in zip(envs, sites)]
    single = []
    fl_single = 0.0
    for e, w, x in zip(envs, sites, psis):
        out = torch.empty_like(x)
        fl_single += b2.b2_heff_apply(ctx, e, w, x, out, prec=prec)
        single.append(out)
    outs = [torch.full_like(x, np.nan) for x in psis]
    fl = b2.b2_heff_apply_batched(ctx, envs, sites, psis, outs, prec=prec)
    torch.cuda.synchronize()
    assert fl == fl_single
    for a, b in zip(single, outs):
        assert torch.equal(a, b)
    _free(objs)


def test_grouped_davidson_equals_single_problem(ctx):
    objs = [_make(ctx, p, p[5]) for p in PROBLEMS]
    envs = [o[2] for o in objs]
    sites = [p[5] for p in PROBLEMS]
    psis = [_psi(ctx, e, w) for e, w in zip(envs, sites)]
    ref = []
    for e, w, x in zip(envs, sites, psis):
        y = x.clone()
        ref.append((b2.b2_davidson(ctx, e, w, y, max_iter=60, max_subspace=20, conv_tol=1e-12), y))
    ys = [x.clone() for x in psis]
    en, nmv, r2 = b2.b2_davidson_batched(ctx, envs, sites, ys, max_iter=60, max_subspace=20,
                                         conv_tol=1e-12)
    torch.cuda.synchronize()
    for i, ((e1, n1, r1), y1) in enumerate(ref):
        assert en[i] == e1 and nmv[i] == n1 and r2[i] == r1
        assert torch.equal(ys[i], y1)
    _free(objs)


@pytest.mark.parametrize("prec", [b2.B2_FP64, b2.B2_BF16X3, b2.B2_TF32X3])
def test_grouped_sweeps_equal_single_problem_sweeps(ctx, prec):
    # one bond-dimension schedule for the whole batch (the call takes one)
    specs = PROBLEMS[:4]
    kw = dict(conv_tol=1e-12, dav_max_iter=60, max_subspace=30, prec=prec)
    M = [60, 80]
    single = []
    for p in specs:
        m, s, env = _make(ctx, p, 0)
        res = b2.b2_sweep(ctx, m, s, env, M, **kw)
        single.append((res, b2.b2_mps_export(ctx, s)))
        _free([(m, s, env)])
    objs = [_make(ctx, p, 0) for p in specs]
    res_b = b2.b2_sweep_batched(ctx, [o[2] for o in objs], M, **kw)
    for i, (res, (bonds, sites, center)) in enumerate(single):
        for a, b in zip(res, res_b[i]):
            assert a["energy"] == b["energy"]
            assert a["n_matvec"] == b["n_matvec"]
            assert a["discarded_weight"] == b["discarded_weight"]
        bonds_b, sites_b, center_b = b2.b2_mps_export(ctx, objs[i][1])
        assert center_b == center == 0
        assert bonds_b == bonds
        for k in range(len(sites)):
            assert sites[k].keys() == sites_b[k].keys()
            for key in sites[k]:
                assert np.array_equal(sites[k][key], sites_b[k][key])
    _free(objs)
