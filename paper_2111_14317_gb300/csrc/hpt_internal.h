// Internal declarations of libhpt (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "hpt.h"

namespace hpt {

constexpr int kMaxN = 32;          // variables (equations = variables, or one fewer: projective form)
constexpr int kMixedMaxM = 128;    // monomials per equation in the mixed form
// Mixed form: monomials whose sum |a_j| exceeds this get their phase
// sum_j a_j arg(y_j) accumulated exactly modulo one revolution in 32-bit
// fixed point instead of by the FP32 exponent GEMM.
constexpr int kBigPhase = 64;
constexpr int kTile = 128;         // paths per tensor-core tile (MMA M)

// Per-equation constant image of the mixed form, laid out exactly as the
// kernel's shared-memory operands (bulk-copied per equation), in two parts:
// the exponent part [bexp | texp] and, from off_bhi (128-byte aligned), the
// coefficient part [bhi | blo].
//   bexp : MP x KX bf16, exponent operand, K index s*n + j holds a_j for the
//          three splits s of log y (K-major, 8x8 core matrices, no swizzle)
//   texp : MP floats, t-exponent numerators e (0 on padding)
//   bhi  : NJ x KC bf16, high part of the realified B_k^T
//   blo  : NJ x KC bf16, low part
struct MixedLayout {
  int MP = 0;   // monomials per equation, padded to 16
  int KX = 0;   // 3n padded to 16
  int NJ = 0;   // 2(n+2) padded to 16
  int KC = 0;   // 2 MP
  int off_bexp = 0, off_bhi = 0, off_blo = 0, off_texp = 0;
  // monomials with sum |a_j| > kBigPhase (their phase is accumulated in
  // fixed point): a bit mask per 32 columns and the exponent vectors as
  // int16, both in the exponent part; 0 when the system has none
  int off_bigm = 0, off_aint = 0;
  int chunk_bytes = 0;
  bool grouped = false;  // coefficient GEMM in the grouped form (j_grouped; affine systems only)
  int tmem_cols = 0;     // power of two >= 4 MP + NJ (3 NJ grouped)
  int smem_bytes = 0;    // dynamic shared memory of the eval kernel
};

// One system's operand shapes as the mixed evaluation kernel reads them
// (from its launch arguments for a single system, from a device table per
// tile for many systems).  n counts the variables (the K dimension of the
// exponent GEMM and the first columns of the extended Jacobian), ne the
// equations (one constant image each): ne = n, or n - 1 in the projective
// form.
struct MixedSys {
  int n, MP, KX, NJ, KC;
  int chunk_bytes, off_bexp, off_bhi, off_blo, off_texp;
  int off_bigm, off_aint;   // 0: no monomial with sum |a_j| > kBigPhase
  int jst;                  // coefficient GEMM in the grouped form (j_grouped)
  int tcols1, tcols2;       // tensor-memory columns with one / two W buffers and J
                            // (for the maxima of a batch: the largest over its systems)
  float inv_D;
  int ne;
  int64_t chunk_off;   // byte offset of the system's constant images
};

// One system's FP64 constants as the FP64 evaluation kernel reads them: n
// equations in nv variables (nv = n, or n + 1 in the projective form).
struct Fp64Sys {
  int n, nv;
  const int32_t* msz;
  const int32_t* off;
  const double* ahat;
  const double2* b;
};

// Whether a system's coefficient GEMM takes the grouped form, two MMAs per
// K-slice into three groups of NJ tensor-memory columns instead of three
// MMAs into one: when two W accumulators (Re and Im each) and the three J
// groups fit in the 512 columns of an SM and 2 NJ is a valid MMA width.
// Affine systems only (the pipelined evaluation and the batch serve those;
// a projective system keeps the narrower J, so that the bulk-synchronous
// kernel keeps two CTAs per SM).  It is fixed per system at creation, so
// every evaluation kernel of a system gives the same bits.
inline bool j_grouped(int MP, int NJ) { return 4 * MP + 3 * NJ <= 512 && 2 * NJ <= 256; }

// Byte offset of element (r, k) of an R x K bf16 operand in the canonical
// K-major no-swizzle layout used by the tensor-core descriptors: 8-row x
// 16-byte core matrices, K-adjacent cores 128 bytes apart (leading byte
// offset), 8-row groups K*16 bytes apart (stride byte offset).
inline int canon_offset(int r, int k, int K) {
  return (r >> 3) * (K * 16) + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2;
}

// Index of entry (path, k, u) of the extended Jacobian scratch, u < n+2:
// tiles of 128 paths, inside a tile entry (k, u) of all 128 paths is
// contiguous, so the 128 threads of a tile write (and the lane groups of the
// solve read) whole sectors.  The scratch holds ceil(p/128)*128 paths.
__host__ __device__ inline size_t ext_index(int64_t path, int k, int u, int n) {
  return ((size_t)(path >> 7) * (size_t)(n * (n + 2)) + (size_t)k * (n + 2) + (size_t)u) * 128 +
         (size_t)(path & 127);
}
inline size_t ext_entries(int64_t p, int n) { return (size_t)((p + 127) / 128) * 128 * n * (n + 2); }

// Paths per evaluate/solve round of hpt_step: the extended Jacobian of a
// chunk (n (n+2) complex per path) stays resident in L2 between the two
// kernels.  A multiple of the tensor-core tile.
constexpr int64_t kChunk = 65536;

// Positions of a launch and the paths behind them.  With every pointer null a
// launch covers one system: position q is path q, every path has n
// variables.  A many-systems launch walks a list of positions padded per
// system to whole 128-position tiles (entry -1 = padding), so every tile
// belongs to one system; tile_sys gives it, sys_n its size, vofs the offset of
// a path's first variable in the concatenated state.  The extended Jacobian
// scratch is indexed by position with the bucket's largest n (nmax).
struct PathMap {
  const int64_t* list = nullptr;
  const int32_t* tile_sys = nullptr;
  const int32_t* sys_n = nullptr;
  const int64_t* vofs = nullptr;
  const int32_t* npos = nullptr;   // device-side position count (null: the host count)
  int nmax = 0;
  const int32_t* pos_begin = nullptr;   // device-side first position (null: 0); a multiple of 128
  const struct MixedSys* sys_tab = nullptr;   // mixed evaluation: per-system operand shapes
};

struct KernelStat {
  std::string name;
  int64_t launches = 0;
  double ms = 0.0;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> pending;
};

void set_error(const char* fmt, ...);

// Start points of a pairs cell (Section 2; the paper leaves this step to the
// literature).  Every solution is log y = z0 + 2 pi i V^{-1} k, z0 = V^{-1}
// log b, for k in a set of coset representatives of Z^n / V Z^n: k_j in
// [0, h_j), h the diagonal of the Hermite normal form of V Z^n (product D =
// |det V|), enumerated in mixed radix (last coordinate fastest).  The phase
// V^{-1} k is reduced modulo 1 exactly: V^{-1} k = adjm k / D mod 1, adjm =
// sign(det V) adj(V) mod D; all below 2^62.
struct StartConsts {
  int32_t n = 0, pad_ = 0;
  uint64_t D = 1;
  int64_t h[kMaxN];
  double zr0[kMaxN], zi0[kMaxN];
  uint64_t adjm[kMaxN * kMaxN];
};

}  // namespace hpt

struct hpt_system_s {
  int n = 0, M = 0;
  // variables: nv = n (affine), or n + 1 homogeneous coordinates (projective
  // form, proj = 1: exponents (a, deg_k - 1^T a), Section 2.2); the device
  // constants below then describe the homogenized system, and `affine` holds
  // the FP64 constants of the affine one for the polish and the adjoint
  int nv = 0, proj = 0;
  std::vector<int64_t> deg;
  hpt_system_s* affine = nullptr;
  hpt_precision prec = HPT_FP64;
  int device = 0;
  std::vector<int32_t> msz, off, exps;
  std::vector<double> coef;          // 2M
  std::vector<int64_t> texp;         // M
  int64_t D = 1;
  std::vector<int64_t> alpha_num, beta_num;
  int max_m = 0;

  // device constants, FP64 form (also used by the mixed form's polish)
  int32_t* d_msz = nullptr;
  int32_t* d_off = nullptr;
  double* d_ahat = nullptr;          // M x (n+1): a_{k,i} and e/D
  double* d_b = nullptr;             // M x (n+2) complex: B_k columns
  // device constants, mixed form
  hpt::MixedLayout ml;
  uint8_t* d_chunks = nullptr;       // n x chunk_bytes

  // device error flag (bounded waits)
  int32_t* d_err = nullptr;

  // scratch (grown on demand)
  void* d_scratch = nullptr;
  size_t scratch_bytes = 0;
  void* d_track = nullptr;           // hpt_track state
  size_t track_bytes = 0;
  int32_t* h_count = nullptr;        // pinned host counter
  hpt_batch self_batch = nullptr;    // hpt_track of the mixed form: a one-system batch

  // profiling
  bool profiling = false;
  std::vector<hpt::KernelStat> stats;
  std::vector<cudaEvent_t> event_pool;
};

namespace hpt {

// Scratch helpers (hpt_host.cpp).
hpt_status ensure_scratch(hpt_system s, size_t bytes);
hpt_status ensure_track(hpt_system s, size_t bytes);

// Profiling helpers: returns an index to pass to prof_end, or -1.
int prof_begin(hpt_system s, const char* name, cudaStream_t st);
void prof_end(hpt_system s, int idx, cudaStream_t st);

// Kernel launchers (return cudaSuccess or the launch error).
// Output layout: either the extended Jacobian in z = log y coordinates (row
// k = [dH_k/dz_0 .. dH_k/dz_{n-1}, dH_k/dtau, H_k] with dH/dz_j =
// y_j dH/dy_j, stored at ext_index; the solves turn their solutions back into
// y coordinates) or the user layout of hpt_eval (H_y, H_t, H).
struct EvalOut {
  void* ext = nullptr;       // extended Jacobian (step scratch)
  void* H = nullptr;         // user layout
  void* Hy = nullptr;
  void* Ht = nullptr;
};

// FP64 SIMT evaluation.  Points are y[p][n] complex128 and either tau[p]
// (tau_is_t = 0) or t[p] (tau_is_t = 1).
cudaError_t launch_eval_fp64(hpt_system s, int64_t p, const void* y, const double* tau,
                             int tau_is_t, const EvalOut& out, cudaStream_t st);

Fp64Sys fp64_sys_of(const hpt_system s);
// The same over the position range [*pm.pos_begin, *pm.npos) of a map whose
// systems all have shape_of(n) == shape (tab: per-system constants), or with
// shape kEval24 all n <= 24; cap bounds the range's length.  Writes the
// extended Jacobian (FP64) only.
constexpr int kEval24 = 4;
cudaError_t launch_eval_fp64_map(int shape, const Fp64Sys* tab, int64_t cap, const void* y, const double* tau,
                                 const PathMap& pm, void* ext, cudaStream_t st);

// Mixed tensor-core evaluation, complex64 in and out.
cudaError_t launch_eval_mixed(hpt_system s, int64_t p, const void* y, const double* tau,
                              int tau_is_t, const EvalOut& out, cudaStream_t st);
// The same over a position map of many systems: pm.sys_tab describes each
// system, chunks holds every system's constant images, maxs the largest of
// each operand dimension (it sizes shared memory; maxs.n = pm.nmax) and
// tmem_cols the largest tensor-memory need.  p bounds the positions;
// ctas_per_sm 0 picks the most that fit.  Writes the extended Jacobian only.
cudaError_t launch_eval_mixed_map(hpt_system prof, const MixedSys& maxs, int tmem_cols, const uint8_t* chunks,
                                  int64_t p, const void* y, const double* tau, const PathMap& pm, void* ext,
                                  int32_t* err, int ctas_per_sm, cudaStream_t st);
// A one-CTA kernel whose bounded mbarrier wait runs out (nothing arrives):
// sets *err after ~2 s.
cudaError_t launch_bounded_wait_probe(int32_t* err, cudaStream_t st);
// Whether the mixed evaluation kernel can run these operand shapes at all
// (its leanest configuration within max_smem bytes of shared memory and the
// 512 tensor-memory columns of an SM).
bool eval_mixed_fits(int n, int MP, int KX, int NJ, int KC, int chunk_bytes, bool big, bool grouped, int max_smem);
// Resident eval CTAs per SM the tensor memory allows for tmem_cols (1 or 2).
int eval_mixed_max_ctas(int tmem_cols);
MixedSys mixed_sys_of(const hpt_system s);
// The pipelined evaluation of one system for the step (scratch output only):
// the dynamic shared memory it needs for shapes s (0: shapes it does not
// serve), and its launch (one persistent CTA per SM).
int eval_pipe_smem(const MixedSys& s);
cudaError_t launch_eval_pipe(hpt_system prof, const MixedSys& s, int64_t p, const uint8_t* chunks, const void* y,
                             const double* tau, void* ext, int32_t* err, int num_sms, cudaStream_t st);

struct StepArgs {
  int n;
  int64_t p;                       // positions (an upper bound when map.npos is set)
  PathMap map;
  const void* ext;           // extended Jacobian of every path
  hpt_paths st;
  hpt_params prm;
  int32_t* err;
  int32_t* redo_count = nullptr;   // mixed form: FP64 re-solve list (scratch)
  int64_t* redo_list = nullptr;
};

// Consolidated solve + update + step control.  T = double for HPT_FP64,
// float for HPT_MIXED.
cudaError_t launch_solve_update(hpt_system s, const StepArgs& a, cudaStream_t st);
// The state arrays of paths q0.. of S (nv complex entries per path of cs bytes).
hpt_paths offset_paths(const hpt_paths& S, int64_t q0, int nv, size_t cs);
// Many-systems pieces of the mixed step: the FP32 solve of one lane-group
// shape (shape_of(n)) over the map's position range, appending FP64
// re-solves to a.redo_list (the caller zeroes a.redo_count once per step),
// and the FP64 re-solve of the whole list with a shape that covers a.map.nmax
// (shapes: 0, 1, 2 as solve_shape_of, kShape8x3 for the FP32 solve).
int solve_shape_of(int n);
constexpr int kShape8x3 = 3;   // FP32 solve only: 8 lanes x 3 rows per path, n <= 24
// FP64 Newton polish update over the position range [*pm.pos_begin,
// *pm.npos) of a map (shape as above; cap bounds the range's length); x is
// complex128 at pm.vofs, done and last (the previous relative correction)
// per path.
cudaError_t launch_newton_map(int shape, int64_t cap, const void* ext, void* x, int32_t* done, float* last,
                              double tol, const PathMap& pm, cudaStream_t st);
cudaError_t launch_solve_fp32_shape(int shape, const StepArgs& a, cudaStream_t st);
cudaError_t launch_redo_fp64_shape(int shape, const StepArgs& a, cudaStream_t st);

// Newton update at t = 1 for the polish: x += dN where the path is not done;
// done[q] set once the error left is below tol (last[q]: the previous
// relative correction, 0 before the first).
cudaError_t launch_newton_update(hpt_system s, int64_t p, const void* ext, void* x,
                                 int32_t* done, float* last, double tol, cudaStream_t st);

// Adjoint: per-solution lambda and the per-block partial sums of the
// coefficient gradient (two kernels).
cudaError_t launch_adjoint(hpt_system s, int64_t p, const void* ext, const void* x,
                           const void* gx, void* partial, void* part, void* gc,
                           cudaStream_t st);
// Bytes of the adjoint's partial column sums (part) for M coefficients.
size_t adjoint_part_bytes(int M);

// FP64 Newton polish at t = 1 of p solutions x (complex128) whose done flag
// is 0, polish_iters rounds over chunks of `chunk` paths; ext holds the
// extended Jacobian of a chunk (FP64), last p floats of scratch.
hpt_status polish_paths(hpt_system s, int64_t p, void* x, int32_t* done, float* last, const hpt_params& prm,
                        void* ext, int64_t chunk, cudaStream_t st);
hpt_status check_params(const hpt_params* prm);
typedef __int128 i128;
// det V exactly for an n x n integer matrix (row-major): HPT_ERANGE when
// Hadamard's bound is beyond the exact range (about 2^120).
hpt_status exact_det(int n, const std::vector<int64_t>& V, i128& det);
// Host setup of the start points (exact diagonal form, z0, phase constants);
// validates first + count <= |det V| (written to *total when not NULL).
hpt_status binomial_setup(int32_t n, const int32_t* msz, const int32_t* exps, const double* coeffs,
                          const int32_t* pairs, int64_t first, int64_t count, bool need_out, StartConsts& S,
                          int64_t* total);
// Every array of the state present (and the *_prev arrays for the Hermite
// predictor).
hpt_status check_state(const hpt_paths* S, const hpt_params* prm);
hpt_status cuda_fail(cudaError_t e, const char* what);

// State init / conversion helpers.
cudaError_t launch_paths_init(hpt_system s, int64_t p, const void* y0, double tau0,
                              const hpt_params& prm, const hpt_paths& st, cudaStream_t stm);
cudaError_t launch_count_active(int64_t p, const int32_t* status, int32_t* count,
                                cudaStream_t st);
cudaError_t launch_finish_track(hpt_system s, int64_t p, const hpt_paths& st, void* x_out,
                                int32_t* status_out, int32_t* steps_out, int32_t* done,
                                cudaStream_t stm);
cudaError_t launch_init_done(int64_t p, const int32_t* status, int32_t* done, cudaStream_t st);

// Algorithm 3 (QR null-space form) for the points of one system: from the
// extended Jacobian in log coordinates (ext, rows k < n, columns u < nv + 2)
// and, in the projective form, the y^* row built from y.  mode 0 writes the
// Euler and Newton directions (dE, dN: p x nv complex of the state precision)
// and ok (p int32) for positions [0, p); mode 1 is one projective step of
// the path state (step control of the projective form).  Shapes: N = rows of
// J (n + proj) <= 8, 16, 24 (FP32), 32.
cudaError_t launch_qr_directions(hpt_system s, int64_t p, const void* ext, const void* y, void* dE, void* dN,
                                 int32_t* ok, cudaStream_t st);
cudaError_t launch_qr_step(hpt_system s, int64_t p, const void* ext, const hpt_paths& S, const hpt_params& prm,
                           cudaStream_t st);
// Projective form: start points x0 (p x n complex128) become
// (x0, 1)/|(x0, 1)| in the state (p x nv); the end points y_acc are
// dehomogenized into x_out (p x n complex128).
cudaError_t launch_paths_init_proj(hpt_system s, int64_t p, const void* x0, double tau0, const hpt_params& prm,
                                   const hpt_paths& st, cudaStream_t stm);
cudaError_t launch_finish_track_proj(hpt_system s, int64_t p, const hpt_paths& st, void* x_out,
                                     int32_t* status_out, int32_t* steps_out, int32_t* done, cudaStream_t stm);

}  // namespace hpt
