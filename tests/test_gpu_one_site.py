"""One-site windows and one-site / mixed sweeps (Sec. 2.1.2) on the GPU against the oracle.

A one-site window is addressed as site | B2_ONE_SITE; its psi has the blocks (jl, s, 0, jr).
Tolerances: FP64 products element-wise 1e-12 (relative to the largest element); split
precision at the bounds of the two-site tests (a one-site window has fewer, smaller terms);
sweep energies 1e-9 as for the two-site sweep."""
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

DEV = torch.device("cuda", 0)
ONE = b2.B2_ONE_SITE


@pytest.fixture(scope="module")
def ctx():
    c = b2.Context(0)
    yield c
    c.close()


def _offsets(bond):
    return np.cumsum([0] + [m for (_, _, m) in bond])


def to_dense1(x, table, bl, br):
    ol, orr = _offsets(bl), _offsets(br)
    d = np.zeros((ol[-1], 4, orr[-1]))
    for jl, s1, s2, jr, off, size in table:
        assert s2 == 0
        ml, mr = bl[jl][2], br[jr][2]
        d[ol[jl]:ol[jl] + ml, s1, orr[jr]:orr[jr] + mr] = x[off:off + size].reshape(ml, mr)
    return d


def to_layout1(d, table, bl, br):
    ol, orr = _offsets(bl), _offsets(br)
    x = np.zeros(int(sum(t[5] for t in table)))
    for jl, s1, s2, jr, off, size in table:
        ml, mr = bl[jl][2], br[jr][2]
        x[off:off + size] = d[ol[jl]:ol[jl] + ml, s1, orr[jr]:orr[jr] + mr].ravel()
    return x


CASES = [
    ("abinitio_n8_M40_s3", lambda: ab_initio_integrals(8, seed=0), 8, "ab_initio", 40, 300, 3),
    ("abinitio_n10_M160_s4", lambda: ab_initio_integrals(10, seed=6), 10, "ab_initio", 160, 311, 4),
    ("abinitio_n10_M160_s0", lambda: ab_initio_integrals(10, seed=6), 10, "ab_initio", 160, 312, 0),
    ("abinitio_n10_M160_s9", lambda: ab_initio_integrals(10, seed=6), 10, "ab_initio", 160, 313, 9),
    ("hubbard_L16_M200_s7", lambda: hubbard_integrals(16, 1.0, 4.0), 16, "hubbard", 200, 304, 7),
]


def _window(ctx, ints, n_elec, kind, M, seed, c):
    h, eri = ints()
    n = h.shape[0]
    bonds = sector_sizes(n, n_elec, 0, M, occupancies(n, n_elec, kind))
    ce = min(c, n - 2)                                  # environments' centre (two-site rule)
    sites = random_mps(bonds, seed=seed, center=ce)
    m = b2.b2_build_mpo(ctx, h, eri, 0.0, n_elec, 0)
    s = b2.b2_mps_import(ctx, bonds, sites, n_elec, 0, center=ce)
    env = b2.b2_env_init(ctx, m, s, center=ce)
    ref = dmrg.DMRG(mpo.MPO(h, eri), bonds, sites, center=ce)
    if c + 1 < n:
        b2.b2_env_update(ctx, env, c + 1, -1)          # R_{c+1} from R_{c+2} and site c+1
        ref.R[c + 1] = dmrg.right_env_update(ref.R[c + 2], ref.A[c + 1], ref.mpo.W[c + 1],
                                             ref.mpo.parity[c + 2], len(ref.mpo.chans[c + 1]))
    else:                                               # last site: L_{n-1} from site n-2
        b2.b2_env_update(ctx, env, c - 1, 1)
        ref.L[c] = dmrg.left_env_update(ref.L[c - 1], ref.A[c - 1], ref.mpo.W[c - 1],
                                        ref.lab[c - 1], len(ref.mpo.chans[c]))
    H = dmrg.Heff1(ref.mpo, c, ref.L[c], ref.R[c + 1], ref.lab[c])
    return bonds, m, s, env, ref, H


def _free(m, s, env):
    b2.b2_free_env(env)
    b2.b2_free_mps(s)
    b2.b2_free_mpo(m)


@pytest.mark.parametrize("name,ints,n_elec,kind,M,seed,c", CASES, ids=[x[0] for x in CASES])
def test_one_site_heff_and_diag_vs_oracle(ctx, name, ints, n_elec, kind, M, seed, c):
    bonds, m, s, env, ref, H = _window(ctx, ints, n_elec, kind, M, seed, c)
    w = c | ONE
    n_elem, n_blk = b2.b2_psi_layout(ctx, env, w)
    table = b2.b2_psi_blocks(ctx, env, w)
    bl, br = bonds[c], bonds[c + 1]
    # the one-site psi of the MPS is its site tensor
    p = torch.empty(n_elem, dtype=torch.float64, device=DEV)
    b2.b2_psi_from_mps(ctx, env, w, p)
    assert np.array_equal(to_dense1(p.cpu().numpy(), table, bl, br), ref.A[c])
    x = np.random.default_rng(seed).standard_normal(n_elem)
    xt = torch.tensor(x, device=DEV)
    y = torch.empty_like(xt)
    fl = b2.b2_heff_apply(ctx, env, w, xt, y)
    assert fl > 0
    y_ref = H.apply(to_dense1(x, table, bl, br))
    y_gpu = to_dense1(y.cpu().numpy(), table, bl, br)
    scale = np.abs(y_ref).max()
    assert np.abs(y_gpu - y_ref).max() <= 1e-12 * scale
    d = torch.empty_like(xt)
    b2.b2_heff_diag(ctx, env, w, d)
    mask = to_dense1(np.ones(n_elem), table, bl, br) != 0
    d_ref = H.diag() * mask
    assert np.abs(to_dense1(d.cpu().numpy(), table, bl, br) - d_ref).max() <= 1e-12 * scale
    for prec, bound in ((b2.B2_BF16X3, 2e-4), (b2.B2_TF32X3, 2e-5)):
        y16 = torch.empty_like(xt)
        b2.b2_heff_apply(ctx, env, w, xt, y16, prec=prec)
        err = np.linalg.norm(to_dense1(y16.cpu().numpy(), table, bl, br) - y_ref) / np.linalg.norm(y_ref)
        assert 1e-12 < err < bound, (prec, err)
    _free(m, s, env)


def test_one_site_davidson_vs_oracle(ctx):
    name, ints, n_elec, kind, M, seed, c = CASES[1]
    bonds, m, s, env, ref, H = _window(ctx, ints, n_elec, kind, M, seed, c)
    w = c | ONE
    n_elem, _ = b2.b2_psi_layout(ctx, env, w)
    p = torch.empty(n_elem, dtype=torch.float64, device=DEV)
    b2.b2_psi_from_mps(ctx, env, w, p)
    e, nmv, r2 = b2.b2_davidson(ctx, env, w, p, max_iter=200, max_subspace=40)
    e_ref, _, _, _ = dmrg.davidson(H.apply, H.diag(), ref.A[c], 1e-12, 200, 40)
    assert r2 <= 1e-10 and abs(e - e_ref) < 1e-9
    _free(m, s, env)


def _sweep_case(n, M, seed, kind):
    if kind == "hubbard":
        h, eri = hubbard_integrals(n, 1.0, 4.0)
    else:
        h, eri = ab_initio_integrals(n, seed=seed)
    bonds = sector_sizes(n, n, 0, M, occupancies(n, n, kind))
    sites = random_mps(bonds, seed=seed + 100)
    return h, eri, bonds, sites


@pytest.mark.parametrize("dots,Ms", [([1, 1, 1], [24, 24, 24]),
                                     ([2, 2, 1, 1, 2], [32, 32, 32, 32, 32])],
                         ids=["one_site", "mixed_2_2_1_1_2"])
@pytest.mark.parametrize("kind,n,M0,seed", [("ab_initio", 8, 16, 71), ("hubbard", 10, 12, 72)],
                         ids=["abinitio_n8", "hubbard_L10"])
def test_sweeps_vs_oracle(ctx, dots, Ms, kind, n, M0, seed):
    h, eri, bonds, sites = _sweep_case(n, M0, seed, kind)
    ref = dmrg.DMRG(mpo.MPO(h, eri), bonds, sites)
    es_ref = ref.run(Ms, dots=dots)
    m = b2.b2_build_mpo(ctx, h, eri, 0.0, n, 0)
    s = b2.b2_mps_import(ctx, bonds, sites, n, 0, center=0)
    env = b2.b2_env_init(ctx, m, s, center=0)
    res = b2.b2_sweep(ctx, m, s, env, Ms, dots=dots)
    es = [r["energy"] for r in res]
    assert np.abs(np.array(es) - np.array(es_ref)).max() < 1e-9, (es, es_ref)
    for r, d in zip(res, dots):
        if d == 1:
            assert r["discarded_weight"] < 1e-12
    # bond dimensions agree with the oracle's and the returned MPS reproduces the energy
    bonds2, sites2, center = b2.b2_mps_export(ctx, s)
    assert center == 0
    assert [sum(x[2] for x in b) for b in bonds2] == [len(l) for l in ref.lab]
    ref2 = dmrg.DMRG(mpo.MPO(h, eri), bonds2, sites2, center=0)
    e_state = float(np.vdot(ref2.psi, ref2.heff(0).apply(ref2.psi)))
    assert abs(e_state - es[-1]) < 1e-9
    _free(m, s, env)


def test_one_site_sweep_holds_fci(ctx):
    n = 6
    h, eri, bonds, sites = _sweep_case(n, 64, 51, "ab_initio")
    e_fci = fci.fci_ground_state(h, eri, n, 0)[0]
    m = b2.b2_build_mpo(ctx, h, eri, 0.0, n, 0)
    s = b2.b2_mps_import(ctx, bonds, sites, n, 0)
    env = b2.b2_env_init(ctx, m, s)
    res = b2.b2_sweep(ctx, m, s, env, [64, 64, 64], dots=[2, 1, 1])
    assert all(abs(r["energy"] - e_fci) < 1e-9 for r in res)
    _free(m, s, env)


def test_bad_dots_and_window_ids_rejected(ctx):
    h, eri, bonds, sites = _sweep_case(6, 8, 81, "ab_initio")
    m = b2.b2_build_mpo(ctx, h, eri, 0.0, 6, 0)
    s = b2.b2_mps_import(ctx, bonds, sites, 6, 0)
    env = b2.b2_env_init(ctx, m, s)
    with pytest.raises(b2.B2Error) as ei:
        b2.b2_sweep(ctx, m, s, env, [8], dots=[3])
    assert ei.value.code == b2.B2_EINVAL
    with pytest.raises(b2.B2Error) as ei:
        b2.b2_psi_layout(ctx, env, 5 | ONE)              # R_6 = right boundary exists, L_5 not
    assert ei.value.code == b2.B2_EINVAL
    with pytest.raises(b2.B2Error) as ei:
        b2.b2_psi_layout(ctx, env, 0 | (1 << 25))        # unknown window bits
    assert ei.value.code == b2.B2_EINVAL
    _free(m, s, env)
