"""GPU parity at the workload sizes: the middle window of the L = 32, M = 500 Hubbard
chain, sector blocks larger than one 128 x 128 tensor-core tile in both directions, the
decaying-integral ab initio family of the n = 36 workload at an oracle-sized n, every
problem of a grouped (batched) launch, and -- where the CPU oracle cannot follow (the
n = 36 middle window at M = 1000: the oracle's plain MPO construction alone takes most of
an hour) -- properties that hold at any size.

Tolerances: FP64 products <= 1e-12 relative (normwise), split-precision products within
the bound of their mode (bf16 x3: 2e-4, tf32 x3: 2e-5, see test_gpu_mixed)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from oracle import dmrg, mpo  # noqa: E402
from paper_2310_03920_gb300 import b2  # noqa: E402
from synth import (ab_initio_integrals, config_integrals, hubbard_integrals,  # noqa: E402
                   occupancies, random_mps, sector_sizes)
from tests.helpers import dense_to_layout, layout_to_dense  # noqa: E402

DEV = torch.device("cuda", 0)
SPLIT_BOUND = {b2.B2_BF16X3: 2e-4, b2.B2_TF32X3: 2e-5}


@pytest.fixture(scope="module")
def ctx():
    c = b2.Context(0)
    yield c
    c.close()


def _gpu(ctx, h, eri, n_elec, bonds, sites, w):
    m = b2.b2_build_mpo(ctx, h, eri, 0.0, n_elec, 0)
    s = b2.b2_mps_import(ctx, bonds, sites, n_elec, 0, center=w)
    env = b2.b2_env_init(ctx, m, s, center=w)
    return m, s, env


def _free(m, s, env):
    b2.b2_free_env(env)
    b2.b2_free_mps(s)
    b2.b2_free_mpo(m)


def _compare(ctx, env, w, H, bonds, x, check_diag=True):
    """GPU products (FP64 and every split mode) and diagonal against the oracle H_eff."""
    table = b2.b2_psi_blocks(ctx, env, w)
    xd = layout_to_dense(x, table, bonds[w], bonds[w + 2])
    y_ref = dense_to_layout(H.apply(xd), table, bonds[w], bonds[w + 2])
    xt = torch.tensor(x, device=DEV)
    yt = torch.empty_like(xt)
    b2.b2_heff_apply(ctx, env, w, xt, yt)
    err = np.linalg.norm(yt.cpu().numpy() - y_ref) / np.linalg.norm(y_ref)
    assert err <= 1e-12, err
    for prec, bound in SPLIT_BOUND.items():
        b2.b2_heff_apply(ctx, env, w, xt, yt, prec=prec)
        e = np.linalg.norm(yt.cpu().numpy() - y_ref) / np.linalg.norm(y_ref)
        assert 1e-10 < e <= bound, (prec, e)
    if check_diag:
        b2.b2_heff_diag(ctx, env, w, yt)
        d_ref = dense_to_layout(H.diag(), table, bonds[w], bonds[w + 2])
        assert np.abs(yt.cpu().numpy() - d_ref).max() <= 1e-12 * max(1.0, np.abs(d_ref).max())
    return table


def test_blocks_larger_than_one_tensor_core_tile(ctx):
    # L = 14 Hubbard chain with alternating occupancies 0.85 / 0.15: at M = 800 the middle
    # window has psi blocks of 185 x 139 (two row tiles and two column tiles of 128) next to
    # small ones, so every tile position of the contraction runs
    L, w, M = 14, 6, 800
    h, eri = hubbard_integrals(L, 1.0, 4.0)
    f = np.array([0.85 if p % 2 == 0 else 0.15 for p in range(L)])
    bonds = sector_sizes(L, L, 0, M, f)
    sites = random_mps(bonds, seed=77, center=w)
    ref = dmrg.DMRG(mpo.MPO(h, eri), bonds, sites, center=w)
    m, s, env = _gpu(ctx, h, eri, L, bonds, sites, w)
    x = np.random.default_rng(14).standard_normal(b2.b2_psi_layout(ctx, env, w)[0])
    table = _compare(ctx, env, w, ref.heff(w), bonds, x)
    ml = np.array([bonds[w][jl][2] for jl in table[:, 0]])
    mr = np.array([bonds[w + 2][jr][2] for jr in table[:, 3]])
    assert np.any((ml > 128) & (mr > 128))
    _free(m, s, env)


def test_hubbard_L32_M500_middle_window(ctx):
    # the sweep workload's bond dimension and chain: window (15, 16) of a random MPS with
    # the M = 500 sector sizes, centred there
    L, M, w = 32, 500, 15
    h, eri = hubbard_integrals(L, 1.0, 4.0)
    bonds = sector_sizes(L, L, 0, M, occupancies(L, L, "hubbard"))
    sites = random_mps(bonds, seed=1132, center=w)
    ref = dmrg.DMRG(mpo.MPO(h, eri), bonds, sites, center=w)
    m, s, env = _gpu(ctx, h, eri, L, bonds, sites, w)
    x = np.random.default_rng(32).standard_normal(b2.b2_psi_layout(ctx, env, w)[0])
    _compare(ctx, env, w, ref.heff(w), bonds, x)
    # psi of the MPS itself, and its energy <psi|H|psi>
    psi = torch.empty(len(x), dtype=torch.float64, device=DEV)
    b2.b2_psi_from_mps(ctx, env, w, psi)
    hp = torch.empty_like(psi)
    b2.b2_heff_apply(ctx, env, w, psi, hp)
    table = b2.b2_psi_blocks(ctx, env, w)
    e_ref = float(np.sum(ref.psi * ref.heff(w).apply(ref.psi)) / np.sum(ref.psi ** 2))
    e_gpu = float(torch.dot(psi, hp) / torch.dot(psi, psi))
    assert abs(e_gpu - e_ref) <= 1e-11 * max(1.0, abs(e_ref))
    assert np.abs(psi.cpu().numpy() - dense_to_layout(ref.psi, table, bonds[w], bonds[w + 2])).max() <= 1e-13
    _free(m, s, env)


def test_decaying_integral_family_window(ctx):
    # the n = 36 workload's integral recipe (60 Cholesky vectors damped by exp(-|p-q|/6),
    # seed 2) at n = 14, middle window, M = 64
    n, w, M = 14, 6, 64
    h, eri = ab_initio_integrals(n, seed=2, n_chol=60, decay=6.0)
    bonds = sector_sizes(n, n, 0, M, occupancies(n, n, "ab_initio"))
    sites = random_mps(bonds, seed=102, center=w)
    ref = dmrg.DMRG(mpo.MPO(h, eri), bonds, sites, center=w)
    m, s, env = _gpu(ctx, h, eri, n, bonds, sites, w)
    x = np.random.default_rng(36).standard_normal(b2.b2_psi_layout(ctx, env, w)[0])
    _compare(ctx, env, w, ref.heff(w), bonds, x)
    _free(m, s, env)


def test_n36_M1000_middle_window_properties(ctx):
    # beyond the oracle: symmetry of H_eff, diagonal = <e_i|H|e_i> on sampled unit vectors
    # (two different kernels), split products within their bound of the FP64 product, and
    # the energy <psi|H|psi> of the MPS the same through windows (16, 17) and (17, 18)
    h, eri, N, tsz, kind = config_integrals("abinitio_n36")
    n, M, w = 36, 1000, 17
    bonds = sector_sizes(n, N, tsz, M, occupancies(n, N, kind))
    sites = random_mps(bonds, seed=102, center=w)
    m, s, env = _gpu(ctx, h, eri, N, bonds, sites, w)
    n_elem, _ = b2.b2_psi_layout(ctx, env, w)
    g = torch.Generator(device="cpu").manual_seed(36)
    x = torch.randn(n_elem, dtype=torch.float64, generator=g).to(DEV)
    y = torch.randn(n_elem, dtype=torch.float64, generator=g).to(DEV)
    hx, hy = torch.empty_like(x), torch.empty_like(y)
    b2.b2_heff_apply(ctx, env, w, x, hx)
    b2.b2_heff_apply(ctx, env, w, y, hy)
    a, c = float(torch.dot(y, hx)), float(torch.dot(hy, x))
    assert abs(a - c) <= 1e-13 * float(hx.norm() * y.norm())
    for prec, bound in SPLIT_BOUND.items():
        hs = torch.empty_like(x)
        b2.b2_heff_apply(ctx, env, w, x, hs, prec=prec)
        assert float((hs - hx).norm() / hx.norm()) <= bound
    d = torch.empty_like(x)
    b2.b2_heff_diag(ctx, env, w, d)
    rng = np.random.default_rng(5)
    e = torch.zeros_like(x)
    for i in rng.choice(n_elem, 6, replace=False):
        e.zero_()
        e[int(i)] = 1.0
        b2.b2_heff_apply(ctx, env, w, e, hx)
        assert abs(float(hx[int(i)]) - float(d[int(i)])) <= 1e-12 * max(1.0, abs(float(d[int(i)])))
    # energy of the MPS through two windows: move the centre one site left
    psi = torch.empty(n_elem, dtype=torch.float64, device=DEV)
    b2.b2_psi_from_mps(ctx, env, w, psi)
    b2.b2_heff_apply(ctx, env, w, psi, hx)
    e1 = float(torch.dot(psi, hx) / torch.dot(psi, psi))
    _free(m, s, env)
    sites2 = random_mps(bonds, seed=102, center=w - 1)
    m, s, env = _gpu(ctx, h, eri, N, bonds, sites2, w - 1)
    n2, _ = b2.b2_psi_layout(ctx, env, w - 1)
    psi2 = torch.empty(n2, dtype=torch.float64, device=DEV)
    b2.b2_psi_from_mps(ctx, env, w - 1, psi2)
    h2 = torch.empty_like(psi2)
    b2.b2_heff_apply(ctx, env, w - 1, psi2, h2)
    e2 = float(torch.dot(psi2, h2) / torch.dot(psi2, psi2))
    # the same state (same random tensors, other gauge): same energy
    assert abs(e1 - e2) <= 1e-9 * max(1.0, abs(e1))
    _free(m, s, env)


# grouped launch: every problem's product against the oracle (not only against the
# single-problem path)
BATCH = [
    (lambda: hubbard_integrals(10, 1.0, 3.0), 10, "hubbard", 40, 301, 4),
    (lambda: ab_initio_integrals(8, seed=11), 8, "ab_initio", 40, 302, 3),
    (lambda: ab_initio_integrals(9, seed=12), 8, "ab_initio", 64, 303, 0),
    (lambda: hubbard_integrals(16, 1.0, 6.0), 16, "hubbard", 120, 304, 7),
    (lambda: ab_initio_integrals(10, seed=13), 10, "ab_initio", 96, 305, 8),
    (lambda: hubbard_integrals(14, 1.0, 2.0), 14, "hubbard", 300, 306, 6),
]


@pytest.mark.parametrize("prec", [b2.B2_FP64] + list(SPLIT_BOUND))
def test_grouped_products_against_oracle(ctx, prec):
    probs, refs = [], []
    for ints, n_elec, kind, M, seed, w in BATCH:
        h, eri = ints()
        n = h.shape[0]
        bonds = sector_sizes(n, n_elec, 0, M, occupancies(n, n_elec, kind))
        sites = random_mps(bonds, seed=seed, center=w)
        refs.append(dmrg.DMRG(mpo.MPO(h, eri), bonds, sites, center=w).heff(w))
        m, s, env = _gpu(ctx, h, eri, n_elec, bonds, sites, w)
        n_elem, _ = b2.b2_psi_layout(ctx, env, w)
        x = np.random.default_rng(seed).standard_normal(n_elem)
        probs.append((m, s, env, w, bonds, x))
    xs = [torch.tensor(p[5], device=DEV) for p in probs]
    ys = [torch.empty_like(x) for x in xs]
    b2.b2_heff_apply_batched(ctx, [p[2] for p in probs], [p[3] for p in probs], xs, ys, prec=prec)
    bound = 1e-12 if prec == b2.B2_FP64 else SPLIT_BOUND[prec]
    for (m, s, env, w, bonds, x), H, y in zip(probs, refs, ys):
        table = b2.b2_psi_blocks(ctx, env, w)
        y_ref = dense_to_layout(H.apply(layout_to_dense(x, table, bonds[w], bonds[w + 2])), table,
                                bonds[w], bonds[w + 2])
        err = np.linalg.norm(y.cpu().numpy() - y_ref) / np.linalg.norm(y_ref)
        assert err <= bound, err
    for m, s, env, *_ in probs:
        _free(m, s, env)
