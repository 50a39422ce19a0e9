"""Split-precision (hi/lo x3 on tcgen05 tensor cores) H_eff and the refined Davidson.

Tolerance of one split product.  bf16 x3: each FP64 operand a is stored as bf16 hi + lo,
leaving |a - hi - lo| <= 2^-16 |a| (two 8-bit mantissas), and the dropped lo*lo product is
of the same size; FP32 accumulation adds 2^-24 per addition.  The chained L.psi.R^T product
rounds its intermediate once more, so a block product carries a relative error of a few
2^-16 (~3e-5 * the sum of the magnitudes of its terms): the test bounds the normwise error
of H_eff.psi by 2e-4 relative.  tf32 x3: two 11-bit mantissas leave 2^-22 per operand, and
the FP32 accumulation (2^-24 per addition, thousands of additions per output) dominates:
bound 2e-5.  The refined Davidson must reproduce the FP64 energy to 1e-6 Eh in both modes.
"""
import json
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from oracle import dmrg, mpo  # noqa: E402
from paper_2310_03920_gb300 import b2  # noqa: E402
from synth import (ab_initio_integrals, hubbard_integrals, occupancies, random_mps,  # noqa: E402
                   sector_sizes)
from tests.helpers import dense_to_layout, layout_to_dense  # noqa: E402

DEV = torch.device("cuda", 0)
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def ctx():
    c = b2.Context(0)
    yield c
    c.close()


def _setup(ctx, h, eri, n_elec, kind, M, seed, center):
    n = h.shape[0]
    bonds = sector_sizes(n, n_elec, 0, M, occupancies(n, n_elec, kind))
    sites = random_mps(bonds, seed=seed, center=center)
    m = b2.b2_build_mpo(ctx, h, eri, 0.0, n_elec, 0)
    s = b2.b2_mps_import(ctx, bonds, sites, n_elec, 0, center=center)
    env = b2.b2_env_init(ctx, m, s, center=center)
    return bonds, sites, m, s, env


CASES = [
    ("abinitio_n8_M40_w3", lambda: ab_initio_integrals(8, seed=0), 8, "ab_initio", 40, 200, 3),
    ("abinitio_n10_M160_w4", lambda: ab_initio_integrals(10, seed=6), 10, "ab_initio", 160, 211, 4),
    ("hubbard_L16_M200_w7", lambda: hubbard_integrals(16, 1.0, 4.0), 16, "hubbard", 200, 204, 7),
]


BOUND = {b2.B2_BF16X3: 2e-4, b2.B2_TF32X3: 2e-5}


@pytest.mark.parametrize("prec", [b2.B2_BF16X3, b2.B2_TF32X3], ids=["bf16x3", "tf32x3"])
@pytest.mark.parametrize("name,ints,n_elec,kind,M,seed,w", CASES, ids=[c[0] for c in CASES])
def test_split_matvec_vs_oracle(ctx, name, ints, n_elec, kind, M, seed, w, prec):
    h, eri = ints()
    bonds, sites, m, s, env = _setup(ctx, h, eri, n_elec, kind, M, seed, w)
    ref = dmrg.DMRG(mpo.MPO(h, eri), bonds, sites, center=w)
    H = ref.heff(w)
    table = b2.b2_psi_blocks(ctx, env, w)
    n_elem, _ = b2.b2_psi_layout(ctx, env, w)
    x = np.random.default_rng(seed).standard_normal(n_elem)
    xt = torch.tensor(x, device=DEV)
    y64, y16 = torch.empty_like(xt), torch.empty_like(xt)
    f64 = b2.b2_heff_apply(ctx, env, w, xt, y64, prec=b2.B2_FP64)
    f16 = b2.b2_heff_apply(ctx, env, w, xt, y16, prec=prec)
    assert f64 == f16
    y_ref = dense_to_layout(H.apply(layout_to_dense(x, table, bonds[w], bonds[w + 2])), table,
                            bonds[w], bonds[w + 2])
    err = np.linalg.norm(y16.cpu().numpy() - y_ref) / np.linalg.norm(y_ref)
    assert err < BOUND[prec], err
    assert err > 1e-10         # the split path really ran in reduced precision
    # deterministic: the same call twice gives the same bits
    y16b = torch.empty_like(xt)
    b2.b2_heff_apply(ctx, env, w, xt, y16b, prec=prec)
    assert torch.equal(y16, y16b)
    for o in (env, s):
        (b2.b2_free_env if o is env else b2.b2_free_mps)(o)
    b2.b2_free_mpo(m)


@pytest.mark.parametrize("prec", [b2.B2_BF16X3, b2.B2_TF32X3], ids=["bf16x3", "tf32x3"])
@pytest.mark.parametrize("w", [3, 5])
def test_refined_davidson_reaches_fp64_energy(ctx, w, prec):
    h, eri = ab_initio_integrals(10, seed=6)
    bonds, sites, m, s, env = _setup(ctx, h, eri, 10, "ab_initio", 120, 500 + w, w)
    n_elem, _ = b2.b2_psi_layout(ctx, env, w)
    p64 = torch.empty(n_elem, dtype=torch.float64, device=DEV)
    b2.b2_psi_from_mps(ctx, env, w, p64)
    p16 = p64.clone()
    e64, n64, r64 = b2.b2_davidson(ctx, env, w, p64, max_iter=300, max_subspace=40)
    e16, n16, r16 = b2.b2_davidson(ctx, env, w, p16, max_iter=300, max_subspace=40,
                                   prec=prec, refine_max=30)
    assert r64 <= 1e-10 and r16 <= 1e-10
    assert abs(e16 - e64) <= 1e-6
    assert abs(abs(float(torch.dot(p16, p64))) - 1.0) < 1e-6
    b2.b2_free_env(env)
    b2.b2_free_mps(s)
    b2.b2_free_mpo(m)


def test_mixed_sweep_matches_fp64_energy(ctx):
    from tests.golden.make_golden import case_inputs
    h, eri, N, tsz, bonds, sites, c = case_inputs("abinitio_n8_M64")
    with open(os.path.join(GOLDEN, "dmrg_oracle.json")) as f:
        gold = json.load(f)["cases"]["abinitio_n8_M64"]["sweep_energies"]
    m = b2.b2_build_mpo(ctx, h, eri, 0.0, N, tsz)
    s = b2.b2_mps_import(ctx, bonds, sites, N, tsz, center=0)
    env = b2.b2_env_init(ctx, m, s, center=0)
    res = b2.b2_sweep(ctx, m, s, env, [c["M"]] * c["sweeps"], conv_tol=c["tol"], dav_max_iter=c["max_iter"],
                      max_subspace=c["max_sub"], prec=b2.B2_BF16X3)
    assert abs(res[-1]["energy"] - gold[-1]) <= 1e-6
    b2.b2_free_env(env)
    b2.b2_free_mps(s)
    b2.b2_free_mpo(m)
