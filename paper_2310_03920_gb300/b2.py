"""Thin ctypes binding of libb2 (include/b2.h).  Argument marshalling only: every step of
the computation runs in the library's CUDA kernels.  PyTorch supplies device memory (the
library's allocations go through torch's caching allocator) and the stream.

Importing this module loads ``libb2.so`` from this directory and raises if it is missing:
there is no fallback path.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libb2.so")

B2_OK, B2_EINVAL, B2_ENOMEM, B2_ECUDA, B2_ENOCONV, B2_ETIMEOUT, B2_EUNSUPPORTED = 0, -1, -2, -3, -4, -5, -6
B2_FP64, B2_BF16X3, B2_TF32X3 = 0, 1, 2
PRECISIONS = {"fp64": B2_FP64, "bf16x3": B2_BF16X3, "tf32x3": B2_TF32X3}
B2_ONE_SITE = 1 << 24   # window id flag: site | B2_ONE_SITE is the one-site window of site
_ERRNAMES = {-1: "B2_EINVAL", -2: "B2_ENOMEM", -3: "B2_ECUDA", -4: "B2_ENOCONV",
             -5: "B2_ETIMEOUT", -6: "B2_EUNSUPPORTED"}

if not os.path.exists(LIB_PATH):
    raise ImportError("libb2.so not built (%s); run __graft_entry__.build()" % LIB_PATH)
lib = ctypes.CDLL(LIB_PATH)

_vp, _i, _d, _i64, _u64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_int64, ctypes.c_uint64
_ALLOC = ctypes.CFUNCTYPE(_vp, ctypes.c_size_t, _vp)
_FREE = ctypes.CFUNCTYPE(None, _vp, _vp)


class DavOpts(ctypes.Structure):
    _fields_ = [("max_iter", _i), ("max_subspace", _i), ("conv_tol", _d), ("prec", _i),
                ("refine_max", _i)]


class SweepOpts(ctypes.Structure):
    _fields_ = [("n_sweeps", _i), ("bond_dims", ctypes.POINTER(_i)), ("conv_tol", _d),
                ("dav_max_iter", _i), ("max_subspace", _i), ("prec", _i), ("trunc_cutoff", _d),
                ("dots", ctypes.POINTER(_i)), ("n_roots", _i), ("noise", ctypes.POINTER(_d))]


class TdvpOpts(ctypes.Structure):
    _fields_ = [("n_steps", _i), ("tau", _d), ("bond_dim", _i), ("trunc_cutoff", _d),
                ("krylov_tol", _d), ("krylov_max", _i)]


class TdvpResult(ctypes.Structure):
    _fields_ = [("energy", _d), ("discarded_weight", _d), ("seconds", _d), ("matvec_flops", _d),
                ("n_matvec", _i), ("max_bond", _i)]


class SweepResult(ctypes.Structure):
    _fields_ = [("energy", _d), ("discarded_weight", _d), ("seconds", _d), ("matvec_flops", _d),
                ("other_flops", _d), ("n_matvec", _i), ("max_bond", _i), ("t_davidson", _d),
                ("t_split", _d), ("root_energy", _d * 16)]


class ProfileData(ctypes.Structure):
    _fields_ = [("launches", _i64), ("heff_launches", _i64), ("heff_ms", _d), ("heff_flops", _d),
                ("eig_launches", _i64), ("eig_ms", _d), ("eig_flops", _d),
                ("rr_launches", _i64), ("rr_ms", _d)]


_sig = {
    "b2_create": (_i, [ctypes.POINTER(_vp), _i, _vp, _ALLOC, _FREE, _vp]),
    "b2_destroy": (None, [_vp]),
    "b2_last_error": (ctypes.c_char_p, [_vp]),
    "b2_build_mpo": (_i, [_vp, _i, _vp, _vp, _d, _i, _i, _d, ctypes.POINTER(_vp)]),
    "b2_mpo_info": (_i, [_vp, ctypes.POINTER(_i), _vp]),
    "b2_mpo_compress": (_i, [_vp, _vp, _d, ctypes.POINTER(_d)]),
    "b2_mpo_export": (_i, [_vp, _vp, _vp, _vp, _vp]),
    "b2_mps_import": (_i, [_vp, _i, _i, _i, _vp, _vp, _vp, _i, ctypes.POINTER(_vp)]),
    "b2_mps_size": (_i, [_vp, ctypes.POINTER(_i64), ctypes.POINTER(_i64), ctypes.POINTER(_i)]),
    "b2_mps_export": (_i, [_vp, _vp, _vp, _vp, _vp]),
    "b2_mps_random": (_i, [_vp, _vp, _i, _vp, _u64, ctypes.POINTER(_vp)]),
    "b2_env_init": (_i, [_vp, _vp, _vp, _i, ctypes.POINTER(_vp)]),
    "b2_env_update": (_i, [_vp, _vp, _i, _i]),
    "b2_psi_layout": (_i, [_vp, _vp, _i, ctypes.POINTER(_i64), ctypes.POINTER(_i64)]),
    "b2_psi_blocks": (_i, [_vp, _vp, _i, _vp]),
    "b2_psi_from_mps": (_i, [_vp, _vp, _i, _vp]),
    "b2_heff_apply": (_i, [_vp, _vp, _i, _vp, _vp, _i, _d, ctypes.POINTER(_d)]),
    "b2_heff_diag": (_i, [_vp, _vp, _i, _vp]),
    "b2_davidson": (_i, [_vp, _vp, _i, _vp, ctypes.POINTER(DavOpts), ctypes.POINTER(_d),
                         ctypes.POINTER(_i), ctypes.POINTER(_d)]),
    "b2_sweep": (_i, [_vp, _vp, _vp, _vp, ctypes.POINTER(SweepOpts), ctypes.POINTER(SweepResult)]),
    "b2_tdvp": (_i, [_vp, _vp, _vp, _vp, ctypes.POINTER(TdvpOpts), ctypes.POINTER(TdvpResult)]),
    "b2_eigh_batched": (_i, [_vp, _i, _vp, _vp, _vp, _vp]),
    "b2_eigh_batched_static": (_i, [_vp, _i, _vp, _vp, _vp, _vp]),
    "b2_rdm_grad": (_i, [_vp, _vp, _vp, _vp, _vp]),
    "b2_heff_apply_batched": (_i, [_vp, _i, _vp, _vp, _vp, _vp, _i, ctypes.POINTER(_d)]),
    "b2_davidson_batched": (_i, [_vp, _i, _vp, _vp, _vp, ctypes.POINTER(DavOpts), _vp, _vp, _vp]),
    "b2_sweep_batched": (_i, [_vp, _i, _vp, ctypes.POINTER(SweepOpts), _vp]),
    "b2_sweep_batched_dims": (_i, [_vp, _i, _vp, ctypes.POINTER(SweepOpts), _vp, _vp]),
    "b2_debug_limits": (_i, [_vp, _i, _i]),
    "b2_sync": (_i, [_vp]),
    "b2_profile": (_i, [_vp, _i]),
    "b2_profile_read": (_i, [_vp, ctypes.POINTER(ProfileData)]),
    "b2_free_mpo": (None, [_vp]),
    "b2_free_mps": (None, [_vp]),
    "b2_free_env": (None, [_vp]),
}
for _name, (_res, _args) in _sig.items():
    _f = getattr(lib, _name)
    _f.restype = _res
    _f.argtypes = _args

EXPORTED = sorted(_sig)


class B2Error(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s: %s" % (_ERRNAMES.get(code, code), msg))
        self.code = code


def _check(ctx, code):
    if code != B2_OK:
        raise B2Error(code, lib.b2_last_error(ctx).decode())


def _ptr(t):
    """Device pointer of a contiguous CUDA float64 tensor."""
    import torch
    assert t.is_cuda and t.dtype == torch.float64 and t.is_contiguous(), "need contiguous cuda float64"
    return ctypes.c_void_p(t.data_ptr())


class Context:
    """A libb2 context on a CUDA device and stream.  Device memory comes from torch's
    caching allocator, or from the given alloc(size) -> pointer (0 = failure) and free(ptr)
    callables."""

    def __init__(self, device=0, stream=None, alloc=None, free=None):
        import torch
        self.torch = torch
        self.device = device
        self.stream = stream if stream is not None else torch.cuda.current_stream(device)
        dev, st = device, self.stream
        if (alloc is None) != (free is None):
            raise ValueError("give both alloc and free, or neither")

        if alloc is None:
            def _alloc(size, user):
                return torch.cuda.caching_allocator_alloc(int(size), dev, st)

            def _free(p, user):
                torch.cuda.caching_allocator_delete(p)
        else:
            def _alloc(size, user):
                return alloc(int(size)) or None

            def _free(p, user):
                free(p)

        self._cb = (_ALLOC(_alloc), _FREE(_free))
        h = _vp()
        _check(None, lib.b2_create(ctypes.byref(h), device, ctypes.c_void_p(self.stream.cuda_stream),
                                   self._cb[0], self._cb[1], None))
        self.h = h

    def close(self):
        if self.h:
            lib.b2_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def b2_build_mpo(ctx, h1, eri, e_core, n_elec, two_sz, cutoff=0.0):
    """ctx may be None (host work)."""
    h1 = np.ascontiguousarray(h1, dtype=np.float64)
    eri = np.ascontiguousarray(eri, dtype=np.float64)
    out = _vp()
    h = ctx.h if ctx is not None else None
    _check(h, lib.b2_build_mpo(h, h1.shape[0], h1.ctypes.data, eri.ctypes.data, e_core,
                               n_elec, two_sz, cutoff, ctypes.byref(out)))
    return out


def b2_mpo_compress(mpo, tol, ctx=None):
    """Compresses the MPO in place; returns the largest relative discarded weight."""
    d = _d()
    h = ctx.h if ctx is not None else None
    _check(h, lib.b2_mpo_compress(h, mpo, tol, ctypes.byref(d)))
    return d.value


def b2_mpo_export(mpo):
    """{"bond_dims", "entries": per site a list of (w, w2, 4x4 op), "parity", "dq"}."""
    dims = b2_mpo_info(mpo)
    n = len(dims) - 1
    cnt = np.zeros(n, dtype=np.int64)
    _check(None, lib.b2_mpo_export(mpo, cnt.ctypes.data, None, None, None))
    tot = int(cnt.sum())
    chan = np.zeros(2 * max(tot, 1), dtype=np.int32)
    ops = np.zeros(16 * max(tot, 1))
    info = np.zeros(3 * int(dims.sum()), dtype=np.int32)
    _check(None, lib.b2_mpo_export(mpo, cnt.ctypes.data, chan.ctypes.data, ops.ctypes.data,
                                   info.ctypes.data))
    entries, e = [], 0
    for k in range(n):
        site = []
        for _ in range(int(cnt[k])):
            site.append((int(chan[2 * e]), int(chan[2 * e + 1]), ops[16 * e:16 * e + 16].reshape(4, 4)))
            e += 1
        entries.append(site)
    parity, dq, c = [], [], 0
    for k in range(n + 1):
        parity.append([int(info[3 * (c + w)]) for w in range(dims[k])])
        dq.append([(int(info[3 * (c + w) + 1]), int(info[3 * (c + w) + 2])) for w in range(dims[k])])
        c += int(dims[k])
    return {"bond_dims": dims, "entries": entries, "parity": parity, "dq": dq}


def b2_mpo_info(mpo):
    n = _i()
    _check(None, lib.b2_mpo_info(mpo, ctypes.byref(n), None))
    dims = np.zeros(n.value + 1, dtype=np.int32)
    _check(None, lib.b2_mpo_info(mpo, ctypes.byref(n), dims.ctypes.data))
    return dims


def b2_mps_import(ctx, bonds, sites, n_elec, two_sz, center=0):
    """bonds / sites in the ``synth.mps_gen`` format (lists of (N, 2Sz, m) and dicts of
    blocks keyed (jl, s, jr))."""
    n = len(sites)
    ns = np.array([len(b) for b in bonds], dtype=np.int32)
    sec = np.array([x for b in bonds for x in b], dtype=np.int32).reshape(-1)
    data = np.concatenate([np.concatenate([blocks[k].ravel() for k in sorted(blocks)])
                           for blocks in sites]).astype(np.float64)
    out = _vp()
    _check(ctx.h, lib.b2_mps_import(ctx.h, n, n_elec, two_sz, ns.ctypes.data, sec.ctypes.data,
                                    data.ctypes.data, center, ctypes.byref(out)))
    return out


def b2_mps_export(ctx, mps):
    ns_tot, ne_tot, center = _i64(), _i64(), _i()
    _check(ctx.h, lib.b2_mps_size(mps, ctypes.byref(ns_tot), ctypes.byref(ne_tot), ctypes.byref(center)))
    n_bonds = None
    sec = np.zeros(3 * ns_tot.value, dtype=np.int32)
    data = np.zeros(ne_tot.value, dtype=np.float64)
    ns = np.zeros(64 + 1, dtype=np.int32)
    _check(ctx.h, lib.b2_mps_export(ctx.h, mps, ns.ctypes.data, sec.ctypes.data, data.ctypes.data))
    # number of bonds: sectors are consumed bond by bond until ns_tot is reached
    tot, n_bonds = 0, 0
    while tot < ns_tot.value:
        tot += int(ns[n_bonds])
        n_bonds += 1
    bonds, pos = [], 0
    for k in range(n_bonds):
        bonds.append([tuple(int(v) for v in sec[3 * (pos + j): 3 * (pos + j) + 3]) for j in range(ns[k])])
        pos += ns[k]
    sites, off = [], 0
    q = [(0, 0), (1, 1), (1, -1), (2, 0)]
    for k in range(n_bonds - 1):
        right = {(b[0], b[1]): j for j, b in enumerate(bonds[k + 1])}
        blocks = {}
        for jl, (N, tsz, ml) in enumerate(bonds[k]):
            for s in range(4):
                jr = right.get((N + q[s][0], tsz + q[s][1]))
                if jr is None:
                    continue
                mr = bonds[k + 1][jr][2]
                blocks[(jl, s, jr)] = data[off:off + ml * mr].reshape(ml, mr).copy()
                off += ml * mr
        sites.append(blocks)
    return bonds, sites, center.value


def b2_mps_random(ctx, mpo, bond_dim, occ=None, seed=0):
    out = _vp()
    occ_arr = None if occ is None else np.ascontiguousarray(occ, dtype=np.float64)
    _check(ctx.h, lib.b2_mps_random(ctx.h, mpo, bond_dim,
                                    None if occ_arr is None else occ_arr.ctypes.data,
                                    ctypes.c_uint64(seed), ctypes.byref(out)))
    return out


def b2_env_init(ctx, mpo, mps, center=0):
    out = _vp()
    _check(ctx.h, lib.b2_env_init(ctx.h, mpo, mps, center, ctypes.byref(out)))
    return out


def b2_env_update(ctx, env, site, direction):
    _check(ctx.h, lib.b2_env_update(ctx.h, env, site, direction))


def b2_psi_layout(ctx, env, site):
    n, nb = _i64(), _i64()
    _check(ctx.h, lib.b2_psi_layout(ctx.h, env, site, ctypes.byref(n), ctypes.byref(nb)))
    return n.value, nb.value


def b2_psi_blocks(ctx, env, site):
    _, nb = b2_psi_layout(ctx, env, site)
    t = np.zeros((nb, 6), dtype=np.int64)
    _check(ctx.h, lib.b2_psi_blocks(ctx.h, env, site, t.ctypes.data))
    return t


def b2_psi_from_mps(ctx, env, site, psi):
    _check(ctx.h, lib.b2_psi_from_mps(ctx.h, env, site, _ptr(psi)))


def b2_heff_apply(ctx, env, site, psi, out, prec=B2_FP64, e_shift=0.0):
    fl = _d()
    _check(ctx.h, lib.b2_heff_apply(ctx.h, env, site, _ptr(psi), _ptr(out), prec, e_shift,
                                    ctypes.byref(fl)))
    return fl.value


def b2_heff_diag(ctx, env, site, diag):
    _check(ctx.h, lib.b2_heff_diag(ctx.h, env, site, _ptr(diag)))


def b2_davidson(ctx, env, site, psi, max_iter=30, max_subspace=30, conv_tol=1e-10,
                prec=B2_FP64, refine_max=0):
    o = DavOpts(max_iter, max_subspace, conv_tol, prec, refine_max)
    e, nmv, r2 = _d(), _i(), _d()
    _check(ctx.h, lib.b2_davidson(ctx.h, env, site, _ptr(psi), ctypes.byref(o), ctypes.byref(e),
                                  ctypes.byref(nmv), ctypes.byref(r2)))
    return e.value, nmv.value, r2.value


def b2_sweep(ctx, mpo, mps, env, bond_dims, conv_tol=1e-10, dav_max_iter=30, max_subspace=30,
             prec=B2_FP64, trunc_cutoff=1e-14, dots=None, noise=None, n_roots=1):
    """dots: None (all two-site) or one entry of 1 / 2 per sweep; noise: None or one
    perturbative-noise weight per sweep; n_roots: state-averaged roots (result key
    "root_energy": their energies)."""
    bd = (_i * len(bond_dims))(*bond_dims)
    dt = None if dots is None else (_i * len(dots))(*dots)
    nz = None if noise is None else (_d * len(noise))(*noise)
    o = SweepOpts(len(bond_dims), bd, conv_tol, dav_max_iter, max_subspace, prec, trunc_cutoff,
                  dt, n_roots, nz)
    res = (SweepResult * len(bond_dims))()
    _check(ctx.h, lib.b2_sweep(ctx.h, mpo, mps, env, ctypes.byref(o), res))
    return [_result(r, n_roots) for r in res]


def b2_tdvp(ctx, mpo, mps, env, n_steps, tau, bond_dim, trunc_cutoff=1e-14, krylov_tol=1e-12,
            krylov_max=40):
    """Imaginary-time two-site TDVP steps; returns one dict per step."""
    o = TdvpOpts(n_steps, tau, bond_dim, trunc_cutoff, krylov_tol, krylov_max)
    res = (TdvpResult * max(1, n_steps))()
    _check(ctx.h, lib.b2_tdvp(ctx.h, mpo, mps, env, ctypes.byref(o), res))
    return [{f: getattr(r, f) for f, _ in TdvpResult._fields_} for r in res[:n_steps]]


def _result(r, n_roots=1):
    d = {f: getattr(r, f) for f, _ in SweepResult._fields_ if f != "root_energy"}
    d["root_energy"] = [r.root_energy[j] for j in range(max(1, n_roots))]
    return d


def b2_eigh_batched(ctx, dims, a, evals, evecs):
    d = np.ascontiguousarray(dims, dtype=np.int32)
    _check(ctx.h, lib.b2_eigh_batched(ctx.h, len(d), d.ctypes.data, _ptr(a), _ptr(evals), _ptr(evecs)))


def b2_eigh_batched_static(ctx, dims, a, evals, evecs):
    """b2_eigh_batched without any device allocation (scratch in a fixed device array);
    stream-ordered: synchronise before reading the results on the host."""
    d = np.ascontiguousarray(dims, dtype=np.int32)
    _check(ctx.h, lib.b2_eigh_batched_static(ctx.h, len(d), d.ctypes.data, _ptr(a), _ptr(evals),
                                             _ptr(evecs)))


def _handles(hs):
    return (_vp * len(hs))(*[h.value if isinstance(h, _vp) else h for h in hs])


def _dev_ptrs(ts):
    return (_vp * len(ts))(*[_ptr(t).value for t in ts])


def b2_heff_apply_batched(ctx, envs, sites, psis, outs, prec=B2_FP64):
    """One grouped launch of the H_eff products of several problems' windows."""
    n = len(envs)
    st = (_i * n)(*sites)
    fl = _d()
    _check(ctx.h, lib.b2_heff_apply_batched(ctx.h, n, _handles(envs), st, _dev_ptrs(psis),
                                            _dev_ptrs(outs), prec, ctypes.byref(fl)))
    return fl.value


def b2_davidson_batched(ctx, envs, sites, psis, max_iter=30, max_subspace=30, conv_tol=1e-10,
                        prec=B2_FP64, refine_max=0):
    n = len(envs)
    o = DavOpts(max_iter, max_subspace, conv_tol, prec, refine_max)
    e = np.zeros(n)
    nmv = np.zeros(n, dtype=np.int32)
    r2 = np.zeros(n)
    _check(ctx.h, lib.b2_davidson_batched(ctx.h, n, _handles(envs), (_i * n)(*sites),
                                          _dev_ptrs(psis), ctypes.byref(o), e.ctypes.data,
                                          nmv.ctypes.data, r2.ctypes.data))
    return e, nmv, r2


def b2_sweep_batched(ctx, envs, bond_dims, conv_tol=1e-10, dav_max_iter=30, max_subspace=30,
                     prec=B2_FP64, trunc_cutoff=1e-14):
    n = len(envs)
    bd = (_i * len(bond_dims))(*bond_dims)
    o = SweepOpts(len(bond_dims), bd, conv_tol, dav_max_iter, max_subspace, prec, trunc_cutoff)
    res = (SweepResult * (n * len(bond_dims)))()
    _check(ctx.h, lib.b2_sweep_batched(ctx.h, n, _handles(envs), ctypes.byref(o), res))
    k = len(bond_dims)
    return [[_result(r) for r in res[p * k:(p + 1) * k]]
            for p in range(n)]


def b2_sweep_batched_dims(ctx, envs, bond_dims, conv_tol=1e-10, dav_max_iter=30,
                          max_subspace=30, prec=B2_FP64, trunc_cutoff=1e-14):
    """bond_dims: one list of per-sweep bond dimensions per problem (equal lengths)."""
    n = len(envs)
    k = len(bond_dims[0])
    assert all(len(b) == k for b in bond_dims)
    flat = np.ascontiguousarray(np.array(bond_dims, dtype=np.int32).reshape(-1))
    o = SweepOpts(k, None, conv_tol, dav_max_iter, max_subspace, prec, trunc_cutoff)
    res = (SweepResult * (n * k))()
    _check(ctx.h, lib.b2_sweep_batched_dims(ctx.h, n, _handles(envs), ctypes.byref(o),
                                            flat.ctypes.data, res))
    return [[_result(r) for r in res[p * k:(p + 1) * k]]
            for p in range(n)]


def b2_rdm_grad(ctx, mpo, mps, n):
    """(gamma [n, n], Gamma / 2 [n, n, n, n]) as numpy FP64: dE/dh and dE/d(pq|rs)."""
    g1 = np.zeros((n, n), dtype=np.float64)
    g2 = np.zeros((n, n, n, n), dtype=np.float64)
    _check(ctx.h, lib.b2_rdm_grad(ctx.h, mpo, mps, g1.ctypes.data, g2.ctypes.data))
    return g1, g2


def b2_debug_limits(ctx, stuck_wait_polls=0, jacobi_max_sweeps=0):
    _check(ctx.h, lib.b2_debug_limits(ctx.h, stuck_wait_polls, jacobi_max_sweeps))


def b2_sync(ctx):
    _check(ctx.h, lib.b2_sync(ctx.h))


def b2_profile(ctx, enable=True):
    _check(ctx.h, lib.b2_profile(ctx.h, 1 if enable else 0))


def b2_profile_read(ctx):
    d = ProfileData()
    _check(ctx.h, lib.b2_profile_read(ctx.h, ctypes.byref(d)))
    return {f: getattr(d, f) for f, _ in ProfileData._fields_}


def b2_free_mpo(mpo):
    lib.b2_free_mpo(mpo)


def b2_free_mps(mps):
    lib.b2_free_mps(mps)


def b2_free_env(env):
    lib.b2_free_env(env)
