// Davidson, truncation and sweep entry points (host orchestration).
#pragma once

#include "engine.hpp"

namespace b2 {

struct DavidsonResult {
  double energy = 0, resid2 = 0, flops = 0;
  int n_matvec = 0;
};

// Batched eigen-decomposition of the symmetric matrices a + offs[j] (dims[j]^2 doubles
// each, row-major): eigenvalues in descending order to evals + eoffs[j], eigenvectors as the
// columns of evecs + offs[j].  Plans a cluster size per matrix (b2k::plan_jacobi), allocates
// the work space and runs the size classes concurrently on the context's side streams.
// Stream-ordered on c->stream; flop_counter: optional device counter of applied rotations;
// unconverged: optional device counter of matrices that used up the sweep limit
// (c->jacobi_max_sweeps, 0 = the default).
void eigh_batched(Ctx* c, const std::vector<int>& dims, const std::vector<int64_t>& offs,
                  const std::vector<int64_t>& eoffs, const double* a, double* evals,
                  double* evecs, double* flop_counter = nullptr, int* unconverged = nullptr);
void contract_two_sites(Ctx* c, const Bond& ba, const Bond& bb, const SiteTensor& X,
                        const double* xd, const SiteTensor& Y, const double* yd,
                        const PsiLayout& lay, double* out, double* flops);
DavidsonResult davidson(b2_env_s* env, int site, double* psi, const b2_dav_opts& o);
// The n_roots lowest eigenpairs (FP64 block Davidson, see algo.cpp); returns the eigenvalues.
std::vector<double> davidson_roots(b2_env_s* env, int win, double* psis, int n_roots,
                                   const b2_dav_opts& o, int* n_matvec, double* max_resid2,
                                   double* flops);
// Splits of the window with id win (a site, or site | kOneSite), see algo.cpp.
// noise: weight of the perturbative noise added to the density matrix (0: none).
// nroot: psi holds that many states of the window layout one after the other; the density
// matrix is their average (weights 1/nroot) and each gets its own remainder and guess.
// keep_centre (two-site windows, one state): psi becomes the split remainder C itself, the
// one-site psi of the centre site (TDVP evolves it before moving on).
void split_left(b2_env_s* env, int win, DevBuf& psi, int M, double cutoff, double* discarded,
                double* flops, double noise = 0.0, int nroot = 1, bool keep_centre = false);
void split_right(b2_env_s* env, int win, DevBuf& psi, int M, double cutoff, double* discarded,
                 double* flops, bool make_guess, double noise = 0.0, int nroot = 1,
                 bool keep_centre = false);
// Imaginary-time two-site TDVP steps (see algo.cpp, b2_tdvp).
void tdvp(b2_env_s* env, const b2_tdvp_opts& o, b2_tdvp_result* res);
void sweep(b2_env_s* env, const b2_sweep_opts& o, b2_sweep_result* res);
// Many independent problems in lockstep, one grouped H_eff launch per Davidson iteration
// (batch.cpp); per problem identical to davidson / sweep.
std::vector<DavidsonResult> davidson_batched(Ctx* c, const std::vector<b2_env_s*>& envs,
                                             const std::vector<int>& sites,
                                             const std::vector<double*>& psis,
                                             const b2_dav_opts& o);
void sweep_batched(Ctx* c, const std::vector<b2_env_s*>& envs, const b2_sweep_opts& o,
                   b2_sweep_result* res, const int* dims_per_problem = nullptr);
// Integral gradient (spin-traced 1- and 2-particle density matrices) of the MPS energy;
// host outputs, see b2_rdm_grad.
void rdm_grad(Ctx* c, b2_mpo_s* mpo, b2_mps_s* mps, double* h1_grad, double* eri_grad);

}  // namespace b2
