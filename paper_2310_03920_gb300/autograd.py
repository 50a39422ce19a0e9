"""torch.autograd.Function for the DMRG energy as a function of the integrals.

``DMRGEnergy.apply(h1, eri, e_core, solver)`` builds the MPO of the ab initio Hamiltonian
(Sec. 2.1.1) with ``b2_build_mpo``, starts from ``b2_mps_random`` and runs two-site sweeps
(``b2_sweep``, Sec. 2.1.2); the result is the energy of the final MPS.  The backward pass
calls ``b2_rdm_grad``: dE/dh_pq = gamma_pq, dE/d(pq|rs) = Gamma_pqrs / 2 (the spin-traced
density matrices of Sec. 2.5.1) and dE/de_core = 1.  These are the derivatives of
<psi|H|psi> at fixed psi, which equal those of the ground-state energy when the sweeps
have converged (Hellmann-Feynman); for a truncated MPS they are the fixed-state gradient.

Argument marshalling only: the MPO, the sweeps and the gradient run in libb2.
"""
import torch

from . import b2


class DMRGSolver:
    """Options of the forward solve, and the libb2 context it runs in."""

    def __init__(self, ctx, n_elec, two_sz, bond_dims, seed=0, init_bond_dim=None,
                 conv_tol=1e-12, dav_max_iter=200, max_subspace=40, prec=b2.B2_FP64,
                 trunc_cutoff=1e-14):
        self.ctx = ctx
        self.n_elec = n_elec
        self.two_sz = two_sz
        self.bond_dims = list(bond_dims)
        self.seed = seed
        self.init_bond_dim = init_bond_dim or self.bond_dims[0]
        self.conv_tol = conv_tol
        self.dav_max_iter = dav_max_iter
        self.max_subspace = max_subspace
        self.prec = prec
        self.trunc_cutoff = trunc_cutoff
        self.last_sweeps = None


class _State:
    """MPO and MPS handles of one forward solve, freed with this object."""

    def __init__(self, mpo, mps, n):
        self.mpo, self.mps, self.n = mpo, mps, n

    def __del__(self):
        try:
            if self.mps:
                b2.b2_free_mps(self.mps)
            if self.mpo:
                b2.b2_free_mpo(self.mpo)
        except Exception:
            pass
        self.mps = self.mpo = None


class DMRGEnergy(torch.autograd.Function):
    @staticmethod
    def forward(fctx, h1, eri, e_core, solver):
        n = h1.shape[0]
        h = h1.detach().to("cpu", torch.float64).contiguous().numpy()
        g = eri.detach().to("cpu", torch.float64).contiguous().numpy()
        ec = float(e_core)
        c = solver.ctx
        mpo = b2.b2_build_mpo(c, h, g, ec, solver.n_elec, solver.two_sz)
        mps = b2.b2_mps_random(c, mpo, solver.init_bond_dim, seed=solver.seed)
        state = _State(mpo, mps, n)
        env = b2.b2_env_init(c, mpo, mps, 0)
        try:
            res = b2.b2_sweep(c, mpo, mps, env, solver.bond_dims, conv_tol=solver.conv_tol,
                              dav_max_iter=solver.dav_max_iter, max_subspace=solver.max_subspace,
                              prec=solver.prec, trunc_cutoff=solver.trunc_cutoff)
        finally:
            b2.b2_free_env(env)
        solver.last_sweeps = res
        fctx.state = state
        fctx.ctx_ = c
        fctx.dev = (h1.device, eri.device)
        return torch.tensor(res[-1]["energy"], dtype=torch.float64)

    @staticmethod
    def backward(fctx, grad_e):
        st = fctx.state
        g1, g2 = b2.b2_rdm_grad(fctx.ctx_, st.mpo, st.mps, st.n)
        ge = grad_e.detach().to("cpu", torch.float64)
        d_h = (ge * torch.from_numpy(g1)).to(fctx.dev[0]) if fctx.needs_input_grad[0] else None
        d_eri = (ge * torch.from_numpy(g2)).to(fctx.dev[1]) if fctx.needs_input_grad[1] else None
        d_core = ge.clone() if fctx.needs_input_grad[2] else None
        return d_h, d_eri, d_core, None


def dmrg_energy(h1, eri, e_core, solver):
    """Differentiable DMRG energy E(h1, eri, e_core) (see ``DMRGEnergy``)."""
    if not torch.is_tensor(e_core):
        e_core = torch.tensor(float(e_core), dtype=torch.float64)
    return DMRGEnergy.apply(h1, eri, e_core, solver)
