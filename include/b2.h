/*
 * libb2 -- two-site DMRG hot path on one GB300 GPU (sm_103a).
 *
 * The method is ab initio two-site DMRG as described in the block2 paper (arXiv
 * 2310.03920): an MPO for the Hamiltonian built from the integrals h_pq and (pq|rs)
 * (Sec. 2.3), environments (the operators of the blocks left and right of a two-site
 * window, Sec. 2.1.2 and Sec. 2.3), the effective Hamiltonian H_eff acting on the
 * two-site wavefunction inside a Davidson eigensolver (Sec. 2.1.3 (iv); Listing 1 for the
 * thrds and dav_max_iter settings), truncation of each bond to M states, and the sweep
 * (Sec. 2.1.2).  Symmetry: particle number and projected spin, U(1) x U(1) (the SZ mode
 * of Sec. 2.1.1).
 *
 * Conventions shared by every call
 *   - Local site basis [|0>, |alpha>, |beta>, |alpha beta>] with (N, 2Sz) = (0,0), (1,1),
 *     (1,-1), (2,0) and |alpha beta> = a+_alpha a+_beta |0> (Listing 1, Part A).
 *   - Bond k lies between sites k-1 and k (k = 0..n).  Every bond sector is labelled by
 *     the (N, 2Sz) of the LEFT block (sites 0..k-1).  Bond 0 has the one sector (0, 0);
 *     bond n has the one sector (n_elec, two_sz); both of size 1.
 *   - Site tensor k: blocks (jl, s, jr) with q[jl] + q(s) = q[jr], each a dense
 *     row-major m_jl x m_jr FP64 array; blocks are stored in lexicographic (jl, s, jr)
 *     order, concatenated.
 *   - Two-site wavefunction of window (i, i+1) ("psi"): blocks (jl, s1, s2) with jl a
 *     sector of bond i and jr (the sector of bond i+2 with q[jr] = q[jl] + q(s1) + q(s2))
 *     existing; block (jl, s1, s2) is m_jl x m_jr row-major; blocks are ordered
 *     lexicographically by (jl, s1, s2) and concatenated.  b2_psi_layout gives the size
 *     and b2_psi_blocks the table.
 *
 * Memory and streams
 *   - All handles are owned by the library and released with b2_free_* / b2_destroy.
 *   - Host arrays passed in are copied during the call; the caller keeps ownership.
 *   - Device pointers passed in (psi, out, diag) are owned by the caller, must be
 *     8-byte aligned, live on the context's device, and are accessed on the context's
 *     stream.  Calls are stream-ordered; results are ready when the stream is.
 *   - Device memory the library needs is requested through the allocator callbacks given
 *     to b2_create (PyTorch's caching allocator from the Python binding); when they are
 *     NULL the library calls cudaMallocAsync / cudaFreeAsync on its stream.
 *
 * Errors: every int-returning call returns B2_OK or a negative code, checks its
 * arguments before launching any kernel, never aborts the process, and leaves a message
 * for b2_last_error.  Device-side waits are bounded; a wait that runs out reports
 * B2_ETIMEOUT.
 */
#ifndef B2_H
#define B2_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  B2_OK = 0,
  B2_EINVAL = -1,        /* invalid argument (shape, quantum numbers, aliasing, non-finite) */
  B2_ENOMEM = -2,        /* an allocation failed */
  B2_ECUDA = -3,         /* a CUDA runtime call failed */
  B2_ENOCONV = -4,       /* an iterative solver did not converge where convergence is required */
  B2_ETIMEOUT = -5,      /* a bounded device-side wait ran out */
  B2_EUNSUPPORTED = -6   /* valid request this build does not implement */
};

/* Arithmetic of the H_eff contraction.  B2_FP64: FP64 throughout.  B2_BF16X3: each FP64
 * operand split into bf16 hi + lo, products hi*hi + hi*lo + lo*hi on the tcgen05 tensor
 * cores with FP32 accumulation, block results added in FP64 (about 1e-4 relative error per
 * product).  B2_TF32X3: the same with tf32 hi + lo (22 significant bits, about 1e-6), at
 * half the tensor-core rate of bf16.  The split products are the mixed-precision path of
 * the Davidson solver, which refines their result with FP64 products (b2_davidson). */
typedef enum { B2_FP64 = 0, B2_BF16X3 = 1, B2_TF32X3 = 2 } b2_prec;

typedef struct b2_ctx_s* b2_ctx;
typedef struct b2_mpo_s* b2_mpo;
typedef struct b2_mps_s* b2_mps;
typedef struct b2_env_s* b2_env;

typedef void* (*b2_alloc_fn)(size_t bytes, void* user);
typedef void (*b2_free_fn)(void* ptr, void* user);

/* Context on CUDA device `device`, issuing all work on `stream` (a cudaStream_t owned by
 * the caller; NULL = the legacy default stream).  alloc/free may be NULL (see above).
 * *out is set only on success. */
int b2_create(b2_ctx* out, int device, void* stream, b2_alloc_fn alloc, b2_free_fn free_fn,
              void* user);
void b2_destroy(b2_ctx ctx);
/* Message of the last failed call on this context (owned by the library, valid until
 * the next call); "" if none.  ctx may be NULL (message of the last b2_create). */
const char* b2_last_error(b2_ctx ctx);

/* ----------------------------------------------------------------------------- MPO
 * Ab initio Hamiltonian (Sec. 2.1.1; formula H = E_core + sum_pq h_pq sum_s a+_ps a_qs
 * + 1/2 sum_pqrs (pq|rs) sum_st a+_ps a+_rt a_st a_qs) as an exact MPO built from the
 * operator strings (Sec. 2.3): operators with at most two elementary operators on the
 * left of a bond are normal operators, the rest are carried as complementary operators,
 * and the partition switches from normal/complementary to complementary/normal after
 * the middle site (the symbolic MPO construction of Sec. 2.3).
 *   h1   host, n_orb x n_orb row-major, h1[p*n+q] = h_pq (symmetric)
 *   eri  host, n_orb^4 row-major, eri[((p*n+q)*n+r)*n+s] = (pq|rs)
 *   integrals with |value| <= cutoff are dropped (0 keeps every nonzero)
 * Host work: ctx may be NULL.
 * Errors: B2_EINVAL for n_orb < 2, n_orb > 64, non-finite integrals, or (n_elec, two_sz)
 * impossible on n_orb orbitals. */
int b2_build_mpo(b2_ctx ctx, int n_orb, const double* h1, const double* eri, double e_core,
                 int n_elec, int two_sz, double cutoff, b2_mpo* out);
/* Number of channels on every bond (bond_dims has n_orb + 1 entries). */
int b2_mpo_info(b2_mpo mpo, int* n_orb, int* bond_dims);
/* Compresses the MPO's bonds (Sec. 2.3: the SVD construction, which reduces the bond
 * dimension at a controlled error; here applied to the built exact MPO).  Host work; ctx
 * may be NULL.  Across bond b, H = sum_w L_w (x) R_w.  The channels of the bond are grouped
 * by the quantum numbers and parity of their left part (the identity and whole-Hamiltonian
 * channels stay alone, so the split-precision products still take the block-Hamiltonian
 * terms in FP64).  Per group, the Gram matrices of the complete left and right operators
 * (trace inner products, built by recursions over the site tensors) give orthonormal bases
 * on both sides and the group's part of H as a coefficient matrix X.  Its singular values
 * above tol * largest are kept: the best approximation of that part in the Frobenius norm.
 * The new channels replace the group's: new columns of the site tensor left of the bond,
 * new rows of the one right of it.  Bonds 1..n_orb-1 are compressed in order.  tol = 0 keeps
 * every direction of nonzero weight (removes linear dependencies only: the contracted H is
 * unchanged to rounding).  discarded (may be NULL): the largest relative weight
 * sqrt(dropped / total squared singular values) over the groups.  The host cost grows
 * steeply with n (Gram recursions and Jacobi eigen-decompositions of each group: seconds at
 * n = 16, minutes at n = 24).  A compressed MPO has no coefficient Jacobian: b2_rdm_grad
 * returns B2_EUNSUPPORTED for it.  Errors: B2_EINVAL (tol outside [0, 1)). */
int b2_mpo_compress(b2_ctx ctx, b2_mpo mpo, double tol, double* discarded);
/* The MPO's tensors, host arrays: n_entries[k] (n_orb entries, always written) = entries of
 * site k; then, for all sites in order, entry_chan (2 ints per entry: channel on bond k,
 * channel on bond k+1) and entry_ops (16 doubles per entry: the local operator, row =
 * output state, before the parity factor of the right channel); chan_info (3 ints per
 * channel of bonds 0..n_orb: parity of the left part, its N and 2Sz change).  The fermion
 * convention: the dense Hamiltonian is the contraction over sites of
 * op_k * P^{parity of its right channel} (P = diag(+1, -1, -1, +1)), from the single channel
 * of bond 0 to the single channel of bond n_orb.  Pointers other than n_entries may be
 * NULL (sizes first). */
int b2_mpo_export(b2_mpo mpo, int64_t* n_entries, int* entry_chan, double* entry_ops,
                  int* chan_info);

/* ----------------------------------------------------------------------------- MPS
 * Import a block-sparse MPS (the layout above) from host arrays.
 *   n_sectors   host, n+1 ints: sectors per bond
 *   sectors     host, sum(n_sectors) x 3 ints (N, 2Sz, m), bond by bond, each bond's
 *               sectors sorted by (N, 2Sz)
 *   site_data   host, every site's blocks concatenated, site 0 first
 *   center      canonical centre c: sites < c left-orthonormal, sites > c
 *               right-orthonormal, site c carries the norm (not checked)
 * Errors: B2_EINVAL for inconsistent sectors. */
int b2_mps_import(b2_ctx ctx, int n, int n_elec, int two_sz, const int* n_sectors,
                  const int* sectors, const double* site_data, int center, b2_mps* out);
/* Sizes for b2_mps_export: total sectors (sum over bonds) and total FP64 elements. */
int b2_mps_size(b2_mps mps, int64_t* n_sector_total, int64_t* n_elem_total, int* center);
/* Copy the MPS back to host arrays sized by b2_mps_size (layout as for import). */
int b2_mps_export(b2_ctx ctx, b2_mps mps, int* n_sectors, int* sectors, double* site_data);
/* Random right-canonical MPS with sector sizes from per-spin occupation probabilities
 * (Sec. 2.1.6 (ii): independent site occupancies give the initial quantum-number
 * distribution; (i): random MPS).  occ: host, n_orb probabilities, or NULL for a Fermi
 * function centred at N/2 of width 2.  The tensors are Gaussian (counter-based
 * generator keyed by seed) made right-orthonormal on the GPU. */
int b2_mps_random(b2_ctx ctx, b2_mpo mpo, int bond_dim, const double* occ, uint64_t seed,
                  b2_mps* out);

/* --------------------------------------------------------------------- environments
 * Environments (renormalized operators, Sec. 2.3) of every MPO channel: all left
 * environments L_0..L_center built from the left-orthonormal sites and all right
 * environments R_{center+2}..R_n from the right-orthonormal sites.  The env keeps
 * references to mpo and mps, which must outlive it. */
int b2_env_init(b2_ctx ctx, b2_mpo mpo, b2_mps mps, int center, b2_env* out);
/* One environment step with the MPS's current tensor at `site`:
 *   dir = +1: L_{site+1} from L_site and site tensor `site` (left-orthonormal)
 *   dir = -1: R_site from R_{site+1} and site tensor `site` (right-orthonormal) */
int b2_env_update(b2_ctx ctx, b2_env env, int site, int dir);

/* ------------------------------------------------------------------- effective H
 * Windows.  The calls below that take `site` accept a window id: `site` itself names the
 * two-site window (site, site+1) with environments L_site and R_{site+2}; site | B2_ONE_SITE
 * names the one-site window of `site` (Sec. 2.1.2, one-site algorithm: the d = 4 space of
 * one site) with environments L_site and R_{site+1}.  A one-site psi has the blocks
 * (jl, s, 0, jr) on bonds (site, site+1), in the order and at the offsets of the MPS's site
 * tensor `site`; its H_eff is sum over MPO channel pairs of L_a (x) W_site (x) R_b.
 * Any other bit pattern, or a window past the chain's end, returns B2_EINVAL. */
#define B2_ONE_SITE (1 << 24)
/* Layout of the wavefunction of a window: number of FP64 elements and of blocks.  The
 * window's environments must exist. */
int b2_psi_layout(b2_ctx ctx, b2_env env, int site, int64_t* n_elem, int64_t* n_blocks);
/* Block table of that layout: n_blocks x 6 int64 (jl, s1, s2, jr, offset, m_l*m_r). */
int b2_psi_blocks(b2_ctx ctx, b2_env env, int site, int64_t* table);
/* Wavefunction of the MPS at a window: two sites, the contraction of site tensors site
 * and site+1; one site, a copy of site tensor `site`.  Written to psi (device, n_elem
 * FP64). */
int b2_psi_from_mps(b2_ctx ctx, b2_env env, int site, double* psi);
/* out = (H_eff - e_shift) psi for a window (Sec. 2.1.2; two sites: the operator is sum over
 * MPO channel pairs of L_a (x) W_site W_{site+1} (x) R_b).  psi, out: device,
 * n_elem FP64 each, must not overlap.  algo_flops (host, may be NULL) receives the
 * algorithmic floating-point operations of the contraction (2 per multiply-add of the
 * block GEMMs actually performed).  Errors: B2_EINVAL on overlap or bad site. */
int b2_heff_apply(b2_ctx ctx, b2_env env, int site, const double* psi, double* out,
                  b2_prec prec, double e_shift, double* algo_flops);
/* Diagonal of H_eff for a window into diag (device, n_elem FP64): the Davidson
 * preconditioner. */
int b2_heff_diag(b2_ctx ctx, b2_env env, int site, double* diag);

/* -------------------------------------------------------------------------- Davidson
 * Lowest eigenpair of H_eff of a window (either width) by the Davidson method (Sec. 2.1.3
 * (iv)): Rayleigh-Ritz in FP64 on the GPU, residual r = H v - theta v, converged when
 * |r|^2 <= conv_tol; correction (D - theta)^-1 r with D the diagonal, orthogonalised
 * twice; a full subspace restarts from the Ritz vector.  With prec != B2_FP64 the
 * products use the split-precision contraction and the run is refined: the Ritz vector
 * is re-checked with FP64 products until the FP64 residual meets conv_tol (or
 * refine_max rounds), and the returned energy is the FP64 Rayleigh quotient.
 *   psi   device, in: guess (need not be normalised), out: unit eigenvector
 * Returns B2_OK also when max_iter is reached unconverged (check *resid2). */
typedef struct {
  int max_iter;       /* products with H_eff per solve (Listing 1: 30) */
  int max_subspace;   /* subspace size before restart (30) */
  double conv_tol;    /* |r|^2 threshold (Listing 1 thrds: 1e-10) */
  b2_prec prec;
  int refine_max;     /* FP64 refinement rounds for split precision (0 = default 4) */
} b2_dav_opts;
int b2_davidson(b2_ctx ctx, b2_env env, int site, double* psi, const b2_dav_opts* opts,
                double* energy, int* n_matvec, double* resid2);

/* ----------------------------------------------------------------------------- sweep
 * DMRG sweeps (Sec. 2.1.2).  One two-site sweep = a forward half over windows 0..n-2
 * then a backward half over windows n-2..0.  After each window's Davidson the forward
 * half splits psi into a left-orthonormal site tensor by the density matrix of the left
 * part and moves right (except at window n-2); the backward half splits off a
 * right-orthonormal tensor and moves left (except at window 0).  Each split keeps the M
 * largest density-matrix eigenvalues over all sectors (eigenvalues <= trunc_cutoff *
 * largest dropped; ties within 1e-14 * largest broken by sector order, then by order in
 * the sector) using a batched FP64 Jacobi eigensolver on the GPU.  The next window's
 * guess is the split remainder contracted with the next site tensor.  The env must have
 * been made with center 0 for this mps, which must be in canonical form with centre 0;
 * on return the MPS is again centred at site 0 and the env consistent with it.
 * One-site sweeps (dots[k] = 1): forward over the one-site windows of sites 0..n-1,
 * backward over n-1..0, with the same splits on one site (rows (l, s) forward, columns
 * (s, r) backward); such a split keeps at most the rank of psi's matricisation, so bond
 * dimensions do not grow.  Mixed schedules switch width at the start of a sweep: two ->
 * one splits the window-0 psi backward with that sweep's M and cutoff; one -> two
 * contracts the site-0 psi with site tensor 1. */
#define B2_MAX_ROOTS 16
typedef struct {
  int n_sweeps;
  const int* bond_dims;       /* host, n_sweeps entries: M of each sweep */
  double conv_tol;            /* Davidson |r|^2 threshold */
  int dav_max_iter;
  int max_subspace;
  b2_prec prec;
  double trunc_cutoff;        /* relative eigenvalue cutoff, e.g. 1e-14 */
  const int* dots;            /* host, n_sweeps entries of 1 (one-site) or 2 (two-site), or
                                 NULL: all two-site.  Other values: B2_EINVAL.  The batched
                                 sweeps take two-site sweeps only (else B2_EUNSUPPORTED). */
  int n_roots;                /* state-averaged roots (Sec. 2.1.3 (i)); 0 or 1: ground state.
                                 k > 1 (at most B2_MAX_ROOTS): every window solves for the k
                                 lowest eigenpairs (block Davidson, FP64 products; other
                                 precisions or one-site sweeps: B2_EUNSUPPORTED) and splits
                                 with the averaged density matrix sum_j psi_j psi_j^T / k;
                                 each state is projected and carried to the next window.
                                 Roots beyond the first start from the unit vectors at the
                                 smallest H_eff diagonal elements; dav_max_iter (0: 30)
                                 bounds the products of one window's solve over all roots,
                                 max_subspace (0: 30, at least 2 n_roots) its subspace.  The MPS left at the end
                                 carries the first root at its centre.  Batched sweeps: one
                                 root only (else B2_EUNSUPPORTED). */
  const double* noise;        /* host, n_sweeps entries >= 0, or NULL: weight of the
                                 perturbative noise (Sec. 2.1.6; White 2005) in each sweep's
                                 splits.  The MPO factorises exactly across the bond being
                                 split, H = sum_w S_w (x) E_w; the kept part's density matrix
                                 becomes rho + noise * N / tr N with N = sum_w P_w P_w^T,
                                 P_w = S_w psi (forward) or E_w psi (backward), restricted to
                                 the sectors the new bond can hold.  It lets one-site sweeps
                                 grow the bond dimension.  Cost: one product per channel of
                                 the cut bond.  Batched sweeps: B2_EUNSUPPORTED unless 0. */
} b2_sweep_opts;
typedef struct {
  double energy;              /* energy at the last window of the sweep */
  double discarded_weight;    /* largest discarded weight of the sweep */
  double seconds;             /* wall time of the sweep */
  double matvec_flops;        /* algorithmic flops of all H_eff products of the sweep */
  double other_flops;         /* algorithmic flops of environment updates and splits */
  int n_matvec;
  int max_bond;               /* largest bond dimension after the sweep */
  double t_davidson;          /* wall time in the Davidson solves */
  double t_split;             /* wall time in truncation, environment update and guess */
  double root_energy[B2_MAX_ROOTS];   /* energies of the n_roots states at the last window */
} b2_sweep_result;
int b2_sweep(b2_ctx ctx, b2_mpo mpo, b2_mps mps, b2_env env, const b2_sweep_opts* opts,
             b2_sweep_result* per_sweep);

/* ---------------------------------------------------------------------------- TDVP
 * Imaginary-time evolution by the two-site time-dependent variational principle (Sec. 2.7.3:
 * TDVP sweeps, and imaginary time needs only real arithmetic for a real Hamiltonian).  One
 * step = the second-order projector-splitting integrator (Haegeman et al. 2016): a forward
 * half over windows 0..n-2 and a backward half n-2..0, each window's two-site psi evolved by
 * exp(-tau/2 H_eff), split (keeping at most bond_dim states, cutoff as in b2_sweep) and the
 * one-site remainder evolved backwards by exp(+tau/2 H_eff) on its one-site window before it
 * is contracted with the next site tensor.  Each exponential is a Krylov (Lanczos)
 * approximation built from H_eff products (FP64; converged when the next Krylov vector's
 * weight is <= krylov_tol of the result, at most krylov_max <= 64 vectors); every local
 * result is normalised, so the MPS follows exp(-tau H) psi / |exp(-tau H) psi|.  With bond
 * dimensions that keep every state the integrator is exact.  The env must have been made
 * with center 0 for this mps (centred at site 0); on return the MPS is again centred at site
 * 0.  Real-time evolution (complex arithmetic) is not offered.
 * Errors: B2_EINVAL (bad options, n < 3, env not at centre 0), B2_ENOCONV (non-finite). */
typedef struct {
  int n_steps;
  double tau;                 /* imaginary time per step, > 0 */
  int bond_dim;               /* M of every split */
  double trunc_cutoff;        /* relative eigenvalue cutoff (negative: 1e-14) */
  double krylov_tol;          /* <= 0: 1e-12 */
  int krylov_max;             /* <= 0: 40 */
} b2_tdvp_opts;
typedef struct {
  double energy;              /* <psi|H|psi> of the normalised state after the step */
  double discarded_weight;    /* largest of the step's splits */
  double seconds;
  double matvec_flops;        /* algorithmic flops of the step's H_eff products */
  int n_matvec;
  int max_bond;
} b2_tdvp_result;
int b2_tdvp(b2_ctx ctx, b2_mpo mpo, b2_mps mps, b2_env env, const b2_tdvp_opts* opts,
            b2_tdvp_result* per_step);

/* ------------------------------------------------------- many independent problems
 * Batched execution of independent problems on one context (one GPU, one stream): the
 * paper runs one large problem with MPI strategies (Sec. 2.2); for many small ones, which
 * alone leave most of a GB300 idle, these calls advance all problems in lockstep and issue
 * ONE grouped launch of the H_eff contraction over every problem's window per Davidson
 * iteration.  Per problem, the kernels, their arguments and their order are those of the
 * single-problem calls, so each result equals that of b2_heff_apply / b2_davidson /
 * b2_sweep on the same problem.  All envs must belong to ctx and be distinct (a window's
 * work space is per env); the psi / out buffers of different problems must not overlap.
 *
 * b2_heff_apply_batched: out_i = H_eff(envs[i], sites[i]) psi_i for i < n (device
 *   vectors in each window's layout; prec B2_FP64 or B2_BF16X3); *algo_flops (may be
 *   NULL) = sum of the problems' algorithmic flops.  No e_shift.
 * b2_davidson_batched: b2_davidson on every (envs[i], sites[i], psis[i]) with the same
 *   options; energies / n_matvec / resid2 (host, n entries each, may be NULL).
 * b2_sweep_batched: b2_sweep (same options) on every env's MPO and MPS; window step t of a
 *   sweep is window t of the forward half or window 2(n-1)-1-t of the backward half of
 *   each problem (problems with fewer sites finish earlier).  results: host,
 *   n * n_sweeps entries, problem-major; seconds, t_davidson and t_split are those of the
 *   whole batch. */
int b2_heff_apply_batched(b2_ctx ctx, int n, const b2_env* envs, const int* sites,
                          const double* const* psis, double* const* outs, b2_prec prec,
                          double* algo_flops);
int b2_davidson_batched(b2_ctx ctx, int n, const b2_env* envs, const int* sites,
                        double* const* psis, const b2_dav_opts* opts, double* energies,
                        int* n_matvec, double* resid2);
int b2_sweep_batched(b2_ctx ctx, int n, const b2_env* envs, const b2_sweep_opts* opts,
                     b2_sweep_result* results);
/* b2_sweep_batched with a bond dimension per problem and sweep: bond_dims (host,
 * n * opts->n_sweeps ints, problem-major) replaces opts->bond_dims (which may be NULL). */
int b2_sweep_batched_dims(b2_ctx ctx, int n, const b2_env* envs, const b2_sweep_opts* opts,
                          const int* bond_dims, b2_sweep_result* results);

/* ------------------------------------------------------------------ batched eigensolver
 * Eigen-decomposition of n_mat real symmetric matrices by cyclic Jacobi rotations in
 * FP64: the density-matrix step of the truncation.  Each matrix gets one thread block or a
 * cluster of 2 to 16 (8 where the device cannot run 16), sized on the host from the dims so
 * that the batch spreads over the SMs with the largest matrices on the largest clusters;
 * every size gives the same results (bitwise).  Rotations stop once
 * every off-diagonal element is below 1e-15 times the largest input element (or negligible
 * next to its diagonal entries): eigenvalues and eigenvectors are accurate to about that
 * fraction of the largest element, as from a backward-stable solver.
 *   dims     host, n_mat ints (1..1024)
 *   a        device, the matrices row-major and concatenated (sum dims^2 FP64); read only
 *   evals    device, sum dims FP64: eigenvalues of each matrix in descending order
 *   evecs    device, sum dims^2 FP64: row-major, column t is the eigenvector of evals[t] */
int b2_eigh_batched(b2_ctx ctx, int n_mat, const int* dims, const double* a, double* evals,
                    double* evecs);

/* Same eigensolver, for callers that cannot allocate device memory.  (The paper has no
 * counterpart; this is an interface for embedding.)  Some callers must not let a library
 * allocate: runtimes that own all device memory through their own pool and forbid other
 * allocators, and latency-critical loops where an allocation could synchronise with the
 * device or fail under memory pressure.  This variant calls no cudaMalloc, cudaFree or
 * allocating library routine: its scratch -- the per-matrix sizes and offsets and the
 * global-memory work space of matrices with dim > 112 -- lives in a fixed device array
 * inside the library, 4 MiB + 32 KiB, which every GPU that loads the library holds until
 * the process exits.  The caller still passes the inputs and outputs (same layout as
 * b2_eigh_batched); the sizes reach the device as a kernel argument.
 *   Limits: n_mat <= 1024; dims in [1, 1024]; the matrices with dim > 112 together need
 *   2 * dim^2 doubles of work space, at most 524288 doubles.  Larger requests return
 *   B2_EINVAL without touching the device.
 *   The first call on a device looks up the array's device address (cudaGetSymbolAddress
 *   with that device current) and keeps it for the life of the process; make that first
 *   call before any stream capture, and do not reset the device in between.
 *   All calls share the array and it keeps the last call's contents; calls whose work
 *   overlaps on the GPU (e.g. on two streams at once) race on it.  The call is
 *   stream-ordered and returns without waiting for the result. */
int b2_eigh_batched_static(b2_ctx ctx, int n_mat, const int* dims, const double* a,
                           double* evals, double* evecs);

/* ----------------------------------------------------------------- integral gradient
 * Gradient of the energy E = <psi|H|psi> / <psi|psi> of the MPS with respect to the
 * integrals of the Hamiltonian of Sec. 2.1.1, at fixed psi: the spin-traced one- and
 * two-particle density matrices of Sec. 2.5.1,
 *   dE/dh_pq      = gamma_pq      = sum_s    <a+_ps a_qs>
 *   dE/d(pq|rs)   = Gamma_pqrs / 2,  Gamma_pqrs = sum_st <a+_ps a+_rt a_st a_qs>,
 * every array element taken as an independent variable (E is linear in each; at a
 * converged ground state this is also the derivative of the ground-state energy).  The
 * mpo only names the system (n, electrons, 2Sz must match the mps): the gradient covers
 * every integral, also those that are zero in mpo.  The computation is the backward pass
 * of the one-site energy <psi| L (x) W_k (x) R |psi> with respect to each MPO entry at
 * each site k (the adjoint of the effective Hamiltonian), chained with the MPO builder's
 * coefficient Jacobian; it runs on a private copy of the MPS, whose centre must be at
 * site 0 (as b2_sweep leaves it).
 *   h1_grad   host, n*n FP64, row-major: gamma
 *   eri_grad  host, n^4 FP64, chemist order (pq|rs): Gamma / 2
 * Errors: B2_EINVAL (mismatched system, centre not 0, zero norm), B2_ECUDA. */
int b2_rdm_grad(b2_ctx ctx, b2_mpo mpo, b2_mps mps, double* h1_grad, double* eri_grad);

/* ------------------------------------------------------------------------ profiling
 * Measurement support for benchmarks (no counterpart in the paper).  While enabled, every
 * launch of the H_eff contraction kernel, of the truncation eigensolver (inside sweeps and
 * b2_eigh_batched) and of the Davidson Rayleigh-Ritz eigensolver is bracketed by CUDA events
 * on the context stream, and every kernel launch of the library is counted.
 * b2_profile(ctx, 1) also resets the counters. */
typedef struct {
  int64_t launches;        /* kernel launches of the library since the reset */
  int64_t heff_launches;   /* H_eff contraction kernel launches timed */
  double heff_ms;          /* their summed device time */
  double heff_flops;       /* their summed algorithmic flops */
  int64_t eig_launches;    /* truncation eigensolver calls timed (a kernel per cluster size) */
  double eig_ms;           /* their summed device time */
  double eig_flops;        /* 12 m_a + 6 m flops per applied Jacobi rotation of an m x m block
                              (m_a: rows active in that sweep) */
  int64_t rr_launches;     /* Davidson Rayleigh-Ritz eigensolves timed (k x k, one CTA) */
  double rr_ms;            /* their summed device time */
} b2_profile_data;
int b2_profile(b2_ctx ctx, int enable);
int b2_profile_read(b2_ctx ctx, b2_profile_data* out);

/* --------------------------------------------------------------------- test support
 * Failure injection for tests of the failure paths (no counterpart in the paper): tests
 * make a device-side limit run out on purpose and check the status that comes back,
 * without faulting or hanging anything.  stuck_wait_polls > 0: every CTA of the
 * tensor-core contraction first waits that many polls on a barrier nothing arrives on, so
 * the wait runs out, the CTA aborts cleanly (copies and MMAs in flight drained, tensor
 * memory freed) and the product reports B2_ETIMEOUT (through b2_sync, b2_davidson or
 * b2_sweep); the context stays usable.  jacobi_max_sweeps > 0: sweeps of the truncation
 * eigensolver before b2_sweep reports B2_ENOCONV for a sector still rotating (0 = the
 * built-in 60).  0 / 0 restores normal operation.  Per context. */
int b2_debug_limits(b2_ctx ctx, int stuck_wait_polls, int jacobi_max_sweeps);
/* Wait for the context's stream and report what its kernels flagged since the last check:
 * B2_ETIMEOUT if a bounded device-side wait ran out (the stream-ordered calls return before
 * their kernels run, so this is where such a failure of b2_heff_apply shows). */
int b2_sync(b2_ctx ctx);

void b2_free_mpo(b2_mpo mpo);
void b2_free_mps(b2_mps mps);
void b2_free_env(b2_env env);

#ifdef __cplusplus
}
#endif
#endif /* B2_H */
