// Environments, contraction programs and the algorithms built on them.
#pragma once

#include <map>

#include "common.hpp"
#include "kernels.cuh"

namespace b2 {

// Block GEMM task list (see kernels.cuh) with its device copy.
struct GemmProgram {
  std::vector<std::vector<b2k::GemmTerm>> by_out;
  std::vector<b2k::GemmOut> outs;
  std::vector<b2k::GemmTerm> terms;
  std::vector<b2k::GemmTask> tasks;              // FP64 work items (32x32 tiles, term ranges)
  std::vector<b2k::GemmReduce> reds;             // fixed-order sums of split tiles
  DevBuf d_terms, d_outs, d_tasks, d_reds, d_partial;
  double flops = 0;
  int add_out(uint8_t buf, int64_t off, int M, int N, int ld, bool accumulate);
  void add_term(int out, const b2k::GemmTerm& t);
  void finalize(Ctx* c);
  void launch(Ctx* c, const b2k::BufTable& bt) const;
  bool empty() const { return tasks.empty(); }
};

struct CombProgram {
  std::vector<b2k::CombOut> outs;
  std::vector<b2k::CombTerm> terms;
  std::vector<b2k::CombTile> tiles;
  DevBuf d_terms, d_outs, d_tiles;
  void finalize(Ctx* c);
  void launch(Ctx* c, const b2k::BufTable& bt) const;
};

// Operator environment on one bond: every channel w has a block (j' <- j) for each ket
// sector j whose bra sector j' (q[j'] = q[j] + dq(w)) exists; blocks are row-major.
struct EnvBond {
  bool valid = false;
  int version = 0;
  struct Blk {
    int jb, jk, mb, mk;
    int64_t off;
  };
  std::vector<Blk> blocks;
  std::vector<std::vector<int>> blk;   // [w][jk] -> block index or -1
  int64_t size = 0;
  DevBuf data;
  void layout(const Bond& b, const std::vector<QN>& dq);
  int find(int w, int jk) const { return blk[w][jk]; }
};

struct PsiBlock {
  int jl, s1, s2, jr, ml, mr;
  int64_t off;
};

// Window ids.  The two-site window (site, site+1) is `site`; the one-site window of `site`
// (Sec. 2.1.2, one-site algorithm) is site | kOneSite.  A one-site window is handled as a
// two-site window whose second site is trivial (its empty state only, identity operator):
// its psi blocks are (jl, s, 0, jr) on bonds (site, site+1), in the order and at the offsets
// of the site tensor's blocks (jl, s).
constexpr int kOneSite = 1 << 24;
inline int win_site(int win) { return win & (kOneSite - 1); }
inline int win_nsite(int win) { return (win & kOneSite) ? 1 : 2; }

// Wavefunction layout of a window on bonds i and i+nsite.  Two-site: blocks (jl, s1, s2, jr).
// One-site: blocks (jl, s, 0, jr), or with trivial_first (jl, 0, s, jr): the same blocks at
// the same offsets with the trivial site on the other side (the backward split reads psi
// that way).
struct PsiLayout {
  std::vector<PsiBlock> blocks;
  std::vector<int> lookup;   // [(jl * 4 + s1) * 4 + s2] -> block or -1
  int64_t size = 0;
  void build(const Bond& bl, const Bond& br, int nsite = 2, bool trivial_first = false);
  int find(int jl, int s1, int s2) const { return lookup[(size_t(jl) * 4 + s1) * 4 + s2]; }
};

// The H_eff contraction in the form of the split-precision tensor-core kernel (tc_heff.cu):
// outputs, terms and 128 x 128 tiles (most expensive first), the split tasks of the
// operand blocks the terms use (environments and precombined operators once per window,
// psi^T once per product) and the split planes ([hi | lo], elements * element size each).
struct TcProgram {
  bool built = false;
  GemmProgram block_h;   // FP64: the block-Hamiltonian terms (kBlockH), written first
  std::vector<b2k::TcOut> outs;
  std::vector<b2k::TcTerm> terms;
  std::vector<b2k::TcTile> tiles;
  std::vector<b2k::SplitTask> env_tasks, psi_tasks;
  int64_t env_elems = 0, psi_elems = 0;
  DevBuf d_outs, d_terms, d_tiles, d_env_tasks, d_psi_tasks;
  DevBuf env_planes, psi_planes;
  int env_prec = -1;   // precision of the split the env planes hold (-1: none)
};

struct WindowProgram {
  int win = -1;            // window id
  int site = -1, nsite = 2;
  int ver_l = -1, ver_r = -1;
  PsiLayout psi;
  GemmProgram heff;        // bufs: 0 psi, 1 out, 2 L env, 3 R env, 4 combination buffer
  CombProgram comb;
  DevBuf comb_buf;
  // Diagonal of H_eff: only channels that keep the sector (dq = 0, even parity) reach it,
  // diag[l][r] = sum_{(a,b)} c_ab dL_a[l] dR_b[r] = sum_a dL_a[l] S_a[r] with
  // S_a = sum_b c_ab dR_b per local pattern.  Work space (dg_buf): the diagonals of the
  // dq = 0 blocks of L (one row of all bond-i states per channel) and of R, and S per
  // pattern; dg_copy extracts the diagonals, dg_comb forms S, dg_gemm one product per psi
  // block (K = number of such left channels).
  std::vector<b2k::CopyTask> dg_copy;
  DevBuf d_dg_copy;
  CombProgram dg_comb;
  GemmProgram dg_gemm;
  int64_t dg_size = 0;
  DevBuf diag;              // the diagonal, computed on first use (environments are fixed)
  bool diag_done = false;
  bool comb_done = false;
  TcProgram tc;
};

// Eigenvectors of the density-matrix sectors of the last split at one window and
// direction, kept to warm-start the next sweep's eigensolver there: a sector whose
// composition is unchanged (same quantum numbers, same contributing (sector, site state)
// parts of the same dimensions) is first rotated into this basis, rho' = V^T rho V, which
// near convergence is almost diagonal, so Jacobi needs a few sweeps instead of ~20.  Any
// orthogonal V gives the same eigen-decomposition; the cache only changes the work.
struct RhoCache {
  std::map<std::vector<int64_t>, std::pair<int64_t, int>> by_sig;   // signature -> (offset, dim)
  DevBuf V;
};

}  // namespace b2

struct b2_env_s {
  b2::Ctx* ctx = nullptr;
  b2_mpo_s* mpo = nullptr;
  b2_mps_s* mps = nullptr;
  std::vector<b2::EnvBond> L, R;   // per bond
  std::map<int, std::unique_ptr<b2::WindowProgram>> windows;
  std::map<int, b2::RhoCache> rho_cache;   // key: 4 * site + 2 * (one-site) + (backward)
  int version_counter = 0;
};

namespace b2 {
WindowProgram& window_program(b2_env_s* env, int site);
void env_update_left(b2_env_s* env, int site);
void env_update_right(b2_env_s* env, int site);
void heff_apply(b2_env_s* env, int site, const double* psi, double* out, double e_shift,
                double* flops, b2_prec prec = B2_FP64);
void heff_diag(b2_env_s* env, int site, double* diag);
// H_eff products of the windows (envs[i], sites[i]) of independent problems on context c
// in one grouped launch (FP64: k_gemm_grouped + k_gemm_reduce_grouped; split precision:
// k_gemm_tc_grouped).  Each work item runs exactly the code of the single-problem launch.
// Split-precision form of window (env, site) for precision prec (host tables, device
// tables, environment split), built on first use and kept with the window program.
TcProgram& tc_program(b2_env_s* env, int site, b2_prec prec);
void heff_apply_batched(Ctx* c, int n, b2_env_s* const* envs, const int* sites,
                        const double* const* psis, double* const* outs, b2_prec prec,
                        double* flops);
}  // namespace b2
