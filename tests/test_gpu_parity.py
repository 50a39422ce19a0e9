"""GPU parity: the C-ABI library against the CPU oracle on the same seeded inputs."""
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
from synth import (ab_initio_integrals, hubbard_integrals,  # noqa: E402
                   occupancies, random_mps, sector_sizes)
from tests.helpers import dense_to_layout, layout_mask, layout_to_dense  # noqa: E402

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


def _free(m, s, env):
    b2.b2_free_env(env)
    b2.b2_free_mps(s)
    b2.b2_free_mpo(m)


CASES = [
    # name, integrals, n_elec, kind, M, MPS seed, window
    ("abinitio_n8_M40_w3", lambda: ab_initio_integrals(8, seed=0), 8, "ab_initio", 40, 200, 3),
    ("abinitio_n10_M96_w4", lambda: ab_initio_integrals(10, seed=6), 10, "ab_initio", 96, 201, 4),
    ("abinitio_n9_N8_M64_w0", lambda: ab_initio_integrals(9, seed=7), 8, "ab_initio", 64, 202, 0),
    ("abinitio_n9_N8_M64_w7", lambda: ab_initio_integrals(9, seed=7), 8, "ab_initio", 64, 203, 7),
    ("hubbard_L16_M120_w7", lambda: hubbard_integrals(16, 1.0, 4.0), 16, "hubbard", 120, 204, 7),
]


@pytest.mark.parametrize("name,ints,n_elec,kind,M,seed,w", CASES, ids=[c[0] for c in CASES])
def test_heff_matvec_and_diag_parity(ctx, name, ints, n_elec, kind, M, seed, w):
    h, eri = ints()
    bonds, sites, m, s, env = _setup(ctx, h, eri, n_elec, kind, M, seed, w)
    ref = dmrg.DMRG(mpo.MPO(h, eri), bonds, sites, center=w)
    H = ref.heff(w)
    table = b2.b2_psi_blocks(ctx, env, w)
    n_elem, n_blocks = b2.b2_psi_layout(ctx, env, w)
    assert n_blocks == len(table) and n_elem == int(table[:, 5].sum())
    # every quantum-number-allowed entry is in the layout, nothing else
    mask = layout_mask(table, bonds[w], bonds[w + 2])
    lab_l, lab_r = ref.lab[w], ref.lab[w + 2]
    q = np.array([[0, 0], [1, 1], [1, -1], [2, 0]])
    allowed = np.all((lab_l[:, None, None, None, :] + q[None, :, None, None, :]
                      + q[None, None, :, None, :]) == lab_r[None, None, None, :, :], axis=-1)
    assert np.array_equal(mask, allowed)
    # psi from the MPS
    psi_t = torch.empty(n_elem, dtype=torch.float64, device=DEV)
    b2.b2_psi_from_mps(ctx, env, w, psi_t)
    np.testing.assert_allclose(psi_t.cpu().numpy(), dense_to_layout(ref.psi, table, bonds[w], bonds[w + 2]),
                               atol=1e-13)
    # H_eff psi on a random vector, the diagonal, and the shifted product
    rng = np.random.default_rng(seed)
    x = rng.standard_normal(n_elem)
    xt = torch.tensor(x, device=DEV)
    yt = torch.empty_like(xt)
    flops = b2.b2_heff_apply(ctx, env, w, xt, yt)
    y_ref = dense_to_layout(H.apply(layout_to_dense(x, table, bonds[w], bonds[w + 2])), table,
                            bonds[w], bonds[w + 2])
    y = yt.cpu().numpy()
    assert np.linalg.norm(y - y_ref) <= 1e-12 * np.linalg.norm(y_ref)
    assert flops > 0
    dt = torch.empty_like(xt)
    b2.b2_heff_diag(ctx, env, w, dt)
    d_ref = dense_to_layout(H.diag(), table, bonds[w], bonds[w + 2])
    assert np.abs(dt.cpu().numpy() - d_ref).max() <= 1e-12 * max(1.0, np.abs(d_ref).max())
    b2.b2_heff_apply(ctx, env, w, xt, yt, e_shift=1.75)
    np.testing.assert_allclose(yt.cpu().numpy(), y_ref - 1.75 * x, atol=1e-12 * np.abs(y_ref).max())
    _free(m, s, env)


def test_heff_hermitian_on_gpu(ctx):
    h, eri = ab_initio_integrals(10, seed=9)
    bonds, sites, m, s, env = _setup(ctx, h, eri, 10, "ab_initio", 80, 300, 4)
    n_elem, _ = b2.b2_psi_layout(ctx, env, 4)
    g = torch.Generator(device="cpu").manual_seed(1)
    x = torch.randn(n_elem, dtype=torch.float64, generator=g).to(DEV)
    y = torch.randn(n_elem, dtype=torch.float64, generator=g).to(DEV)
    hx, hy = torch.empty_like(x), torch.empty_like(y)
    b2.b2_heff_apply(ctx, env, 4, x, hx)
    b2.b2_heff_apply(ctx, env, 4, y, hy)
    a, bb = float(torch.dot(y, hx)), float(torch.dot(hy, x))
    assert abs(a - bb) <= 1e-13 * float(hx.norm() * y.norm())
    _free(m, s, env)


def test_heff_rejects_overlap_and_bad_window(ctx):
    h, eri = ab_initio_integrals(6, seed=2)
    bonds, sites, m, s, env = _setup(ctx, h, eri, 6, "ab_initio", 16, 301, 0)
    n_elem, _ = b2.b2_psi_layout(ctx, env, 0)
    x = torch.zeros(2 * n_elem, dtype=torch.float64, device=DEV)
    with pytest.raises(b2.B2Error) as e:
        b2.b2_heff_apply(ctx, env, 0, x[:n_elem], x[1:n_elem + 1])
    assert e.value.code == b2.B2_EINVAL
    with pytest.raises(b2.B2Error):
        b2.b2_heff_apply(ctx, env, 2, x[:n_elem], x[n_elem:])   # R_{4} of centre 0 exists, L_2 not
    _free(m, s, env)


@pytest.mark.parametrize("w", [0, 3, 6])
def test_davidson_parity(ctx, w):
    h, eri = ab_initio_integrals(8, seed=0)
    bonds, sites, m, s, env = _setup(ctx, h, eri, 8, "ab_initio", 48, 400 + w, w)
    ref = dmrg.DMRG(mpo.MPO(h, eri), bonds, sites, center=w)
    H = ref.heff(w)
    # a random-MPS window is a poor guess: allow enough products for both to converge
    # (unconverged Davidson iterates amplify rounding differences and are not comparable)
    e_ref, v_ref, nmv_ref, r2_ref = dmrg.davidson(H.apply, H.diag(), ref.psi, 1e-10, 300, 40)
    assert r2_ref <= 1e-10
    n_elem, _ = b2.b2_psi_layout(ctx, env, w)
    psi = torch.empty(n_elem, dtype=torch.float64, device=DEV)
    b2.b2_psi_from_mps(ctx, env, w, psi)
    e, nmv, r2 = b2.b2_davidson(ctx, env, w, psi, max_iter=300, max_subspace=40)
    assert r2 <= 1e-10
    assert abs(e - e_ref) < 1e-9
    table = b2.b2_psi_blocks(ctx, env, w)
    v = dense_to_layout(v_ref, table, bonds[w], bonds[w + 2])
    assert abs(abs(float(np.dot(psi.cpu().numpy(), v))) - 1.0) < 1e-8
    _free(m, s, env)


def test_eigh_batched_vs_numpy(ctx):
    dims = [1, 2, 3, 7, 16, 33, 64, 100, 104, 105, 160, 257]
    rng = np.random.default_rng(5)
    mats = []
    for d in dims:
        x = rng.standard_normal((d, max(1, d // 2)))
        a = x @ x.T + (1e-3 * np.diag(rng.random(d)) if d % 2 else 0.0)   # PSD, some rank deficient
        mats.append(a)
    a_t = torch.tensor(np.concatenate([a.ravel() for a in mats]), device=DEV)
    ev = torch.empty(sum(dims), dtype=torch.float64, device=DEV)
    vec = torch.empty(sum(d * d for d in dims), dtype=torch.float64, device=DEV)
    b2.b2_eigh_batched(ctx, dims, a_t, ev, vec)
    ev, vec = ev.cpu().numpy(), vec.cpu().numpy()
    eo = vo = 0
    for d, a in zip(dims, mats):
        w = ev[eo:eo + d]
        u = vec[vo:vo + d * d].reshape(d, d)
        wr = np.linalg.eigvalsh(a)[::-1]
        scale = np.linalg.norm(a)
        assert np.all(np.diff(w) <= 0)
        assert np.abs(w - wr).max() <= 1e-13 * scale
        assert np.abs(u.T @ u - np.eye(d)).max() <= 1e-13 * d
        assert np.abs(u @ np.diag(w) @ u.T - a).max() <= 1e-13 * scale * np.sqrt(d)
        eo += d
        vo += d * d


def test_eigh_batched_edge_cases(ctx):
    # zero, diagonal, identity, identity + rank one (a degenerate eigenvalue), scales near
    # the ends of the FP64 range (the kernels scale by a power of two on entry), and graded
    # density-matrix-like inputs; the one-CTA entry point must agree bitwise
    from synth import graded_density_matrices
    rng = np.random.default_rng(17)
    mats = [np.zeros((5, 5)), np.diag(rng.standard_normal(9)), np.eye(70)]
    u = rng.standard_normal(66)
    mats.append(np.eye(66) + np.outer(u, u))
    x = rng.standard_normal((40, 40))
    mats.append(1e200 * (x + x.T))
    mats.append(1e-200 * (x + x.T))
    mats += graded_density_matrices([96, 31, 130], seed=9)
    dims = [a.shape[0] for a in mats]
    a_t = torch.tensor(np.concatenate([a.ravel() for a in mats]), device=DEV)
    out = []
    for fn in (b2.b2_eigh_batched, b2.b2_eigh_batched_static):
        ev = torch.empty(sum(dims), dtype=torch.float64, device=DEV)
        vec = torch.empty(sum(d * d for d in dims), dtype=torch.float64, device=DEV)
        fn(ctx, dims, a_t, ev, vec)
        torch.cuda.synchronize()
        out.append((ev.cpu().numpy(), vec.cpu().numpy()))
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])
    ev, vec = out[0]
    eo = vo = 0
    for d, a in zip(dims, mats):
        w = ev[eo:eo + d]
        v = vec[vo:vo + d * d].reshape(d, d)
        scale = max(np.abs(a).max(), np.finfo(float).tiny)
        assert np.all(np.diff(w) <= 0)
        assert np.abs(w - np.linalg.eigvalsh(a)[::-1]).max() <= 1e-13 * scale * d
        assert np.abs(v.T @ v - np.eye(d)).max() <= 1e-13 * d
        assert np.abs((a / scale) @ v - v * (w / scale)).max() <= 1e-13 * d
        if not np.any(a - np.diag(np.diag(a))):   # diagonal input: nothing to rotate
            assert np.array_equal(np.sort(w), np.sort(np.diag(a)))
        eo += d
        vo += d * d


def _golden():
    with open(os.path.join(GOLDEN, "dmrg_oracle.json")) as f:
        return json.load(f)["cases"]


@pytest.mark.parametrize("case", ["abinitio_n8_M64", "hubbard_L12_M48"])
def test_sweep_energies_match_oracle(ctx, case):
    from tests.golden.make_golden import CASES, case_inputs
    h, eri, N, tsz, bonds, sites, c = case_inputs(case)
    gold = _golden()[case]
    m = b2.b2_build_mpo(ctx, h, eri, 0.0, N, tsz)
    s = b2.b2_mps_import(ctx, bonds, sites, N, tsz, center=0)
    env = b2.b2_env_init(ctx, m, s, center=0)
    res = b2.b2_sweep(ctx, m, s, env, [c["M"]] * c["sweeps"], conv_tol=c["tol"], dav_max_iter=c["max_iter"],
                      max_subspace=c["max_sub"])
    es = [r["energy"] for r in res]
    for e, g in zip(es, gold["sweep_energies"]):
        assert abs(e - g) < 1e-9, (es, gold["sweep_energies"])
    if "fci" in gold:
        assert es[-1] >= gold["fci"] - 1e-10
    # the returned MPS is canonical with centre 0 and reproduces the energy
    bonds2, sites2, center = b2.b2_mps_export(ctx, s)
    assert center == 0
    ref = dmrg.DMRG(mpo.MPO(h, eri), bonds2, sites2, center=0)
    Hh = ref.heff(0)
    e_state = float(np.vdot(ref.psi, Hh.apply(ref.psi)))
    assert abs(e_state - es[-1]) < 1e-9
    _free(m, s, env)


def test_sweep_exact_bond_dimension_reaches_fci(ctx):
    from oracle import fci
    n = 6
    h, eri = ab_initio_integrals(n, seed=51)
    M = 64
    bonds = sector_sizes(n, n, 0, M, occupancies(n, n, "ab_initio"))
    sites = random_mps(bonds, seed=151)
    e_fci = fci.fci_ground_state(h, eri, n, 0)[0]
    m = b2.b2_build_mpo(ctx, h, eri, 0.0, n, 0)
    s = b2.b2_mps_import(ctx, bonds, sites, n, 0)
    env = b2.b2_env_init(ctx, m, s)
    res = b2.b2_sweep(ctx, m, s, env, [M] * 3)
    assert abs(res[-1]["energy"] - e_fci) < 1e-9
    _free(m, s, env)


@pytest.mark.parametrize("kind", ["ab_initio", "hubbard"])
def test_mps_random_is_right_canonical_with_generator_sectors(ctx, kind):
    n, M = 10, 60
    if kind == "hubbard":
        h, eri = hubbard_integrals(n, 1.0, 4.0)
        occ = np.full(n, 0.5)
    else:
        h, eri = ab_initio_integrals(n, seed=3)
        occ = None
    m = b2.b2_build_mpo(ctx, h, eri, 0.0, n, 0)
    s = b2.b2_mps_random(ctx, m, M, occ=occ, seed=7)
    bonds, sites, center = b2.b2_mps_export(ctx, s)
    assert center == 0
    # same sector sizes as the seeded generator's recipe
    assert bonds == sector_sizes(n, n, 0, M, occupancies(n, n, kind))
    lab, A = dmrg.blocks_to_dense(bonds, sites)
    for k in range(1, n):
        B = A[k].reshape(A[k].shape[0], -1)
        assert np.abs(B @ B.T - np.eye(B.shape[0])).max() < 1e-10
    assert abs(np.sum(A[0] ** 2) - 1.0) < 1e-12
    # the state is usable: environments and a sweep run from it
    env = b2.b2_env_init(ctx, m, s, center=0)
    res = b2.b2_sweep(ctx, m, s, env, [M], dav_max_iter=60, max_subspace=40)
    assert np.isfinite(res[0]["energy"])
    _free(m, s, env)
