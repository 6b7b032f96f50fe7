// Internal declarations of the kqr library (not part of the ABI).
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/kqr.h"

namespace kqr {

// Tile geometry of the Gram-product kernels: a CTA owns 128 rows of K and
// sweeps 128-column tiles; 256 threads each hold an 8 x 8 block of entries.
constexpr int kTile = 128;
constexpr int kThreads = 256;
constexpr int kMaxP = 64;          // features supported by the tile kernels
constexpr int kMaxRhs = 8;         // right-hand sides of one Gram product
constexpr int kExpTableBits = 10;  // 2^-f table of the double-float exp2
constexpr int kRbfEmuMaxP = 40;    // features of the fixed-point FP64-class RBF product

// Status values a kernel writes to the device error word.
constexpr int kErrWaitTimeout = 1;

struct Allocator {
  void* (*alloc)(size_t, void*) = nullptr;
  void (*free_fn)(void*, void*) = nullptr;
  void* ctx = nullptr;
};

struct Handle;
struct BatchData;
struct GridRdv;

// ---- device memory ---------------------------------------------------------
void* dev_alloc(Handle* h, size_t bytes);
void dev_free(Handle* h, void* p);

// ---- Gram products (gram_f32.cu, gram_high.cu) ------------------------------
// Epilogue applied when the per-split partial sums are combined:
//   out[i, c] = sum_s part[s][i][c]                       (plain product), or
//   out[i]    = sum_s part[s][i] + gam * sum_p + L[i] p[i] (CG operator, m = 1),
// with dot_out (device, nullable) accumulating sum_i p[i] out[i].
struct GramEpilogue {
  double gam = 0.0;
  const double* gam_dev = nullptr; // device scalar read instead of gam when set (graph-captured CG)
  const double* sum_p = nullptr;   // device scalar 1^T p
  const double* L = nullptr;       // device diagonal
  const double* pvec = nullptr;    // device vector p (FP64)
  double* dot_out = nullptr;       // device scalar, accumulates p^T out
  double* raw_out = nullptr;       // device, receives K p alone (nullable)
};

cudaError_t gram_f32(Handle* h, const double* V, double* U, int m, const GramEpilogue* ep, cudaStream_t st);
// RBF product with the cross term on tcgen05 (gram_rbf_tc.cu): FP32 accuracy
// (three TF32 terms) or TF32 (one term); ep as for gram_f32.
cudaError_t gram_rbf_tc(Handle* h, const double* V, double* U, int m, bool three_terms, const GramEpilogue* ep,
                        cudaStream_t st);
// RBF product with the cross term as one bf16 tensor-core product (KQR_PREC_BF16).
cudaError_t gram_rbf_tc_bf16(Handle* h, const double* V, double* U, int m, cudaStream_t st);
// m = 1 product with each off-diagonal tile formed once (gram_f32_sym.cu).
cudaError_t gram_f32_sym(Handle* h, const double* V, double* U, const GramEpilogue* ep, cudaStream_t st);
cudaError_t gram_high(Handle* h, const double* V, double* U, int m, cudaStream_t st);
// Laplacian m = 1 FP64-class product with each off-diagonal tile formed once (gram_high_sym.cu).
cudaError_t gram_high_sym(Handle* h, const double* V, double* U, cudaStream_t st);
// Stored-K product (gram_stored.cu): kstore_setup fills the packed upper-triangle tiles
// when options.gram_store asks for it and they fit; gram_stored streams them (m = 1).
size_t kstore_bytes(int64_t ldn);
kqr_status kstore_setup(Handle* h);
void kstore_free(Handle* h);
cudaError_t gram_stored(Handle* h, const double* V, double* U, const GramEpilogue* ep, cudaStream_t st);
// Column s of K in FP64 (RPCholesky).

struct Handle {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  Allocator alloc;

  int64_t n = 0, p = 0, ldn = 0;      // ldn = n rounded up to a multiple of kTile
  kqr_kernel kind = KQR_RBF;
  double gamma = 0.0;
  kqr_options opt{};

  // FP32 tile layout: feature-major [p][ldn], centred and scaled so that
  // K_ij = exp2(-||xs_i - xs_j||_1) (Laplacian) or exp2(-||xs_i - xs_j||_2^2) (RBF).
  float* xs32 = nullptr;
  float* nrm32 = nullptr;             // RBF: ||xs_i||^2 (FP32 of the FP64 value)
  CUtensorMap tm_xs32{};

  // FP64-class layout.  Laplacian: xs = hq * 2^-grid_G + hl, hq int32, hl float.
  int32_t* hq = nullptr;
  float* hl = nullptr;
  int grid_G = 0;
  CUtensorMap tm_hq{}, tm_hl{};
  float2* exp_table = nullptr;        // 2^-(k / 2^kExpTableBits) as (hi, lo) floats
  // Centred FP64 copy, feature-major [p][ldn] (RBF high-precision product and K columns).
  double* xc64 = nullptr;
  double* y = nullptr;

  // RPCholesky factor, column-major [r][n] (column c at F32 + c * n).
  int r0 = 0, r = 0;
  float* F32 = nullptr;
  double* dres = nullptr;             // residual diagonal diag(K - F F^T), FP32 factor
  std::vector<int64_t> pivots;

  // Woodbury core (r + 1)^2, its Cholesky factor and work vectors.
  double* core = nullptr;
  double* tvec = nullptr;             // r + 1
  double* Linv = nullptr;             // n
  bool core_valid = false;
  double core_gam = 0.0;              // gam the current core was built for
  kqr_precond core_kind = KQR_PRECOND_NYSTROM_DIAG;
  int64_t core_builds = 0, core_reuses = 0;

  // RBF tensor-core path: row-major TF32 parts [ldn][tc_Kp] and their swizzled tensor maps.
  float* tc_hi = nullptr;
  float* tc_lo = nullptr;
  int tc_Kp = 0;
  int tc_fold_rows = 0;   // apply exp2(-|xs_i|^2) to finished row sums (all norms < 60)
  CUtensorMap tm_tc_hi{}, tm_tc_lo{};
  __nv_bfloat16* tc_bf = nullptr;     // row-major bf16 copy [ldn][64] (KQR_PREC_BF16)
  CUtensorMap tm_tc_bf{};
  // fp16 copies for the symmetric FP32-class tiles: per row A' = [hi | hi | lo] and
  // B' = [hi | lo | hi] over the p features, zero padded to 64 tc16_katoms halves, with
  // their swizzled tensor maps (the rows viewed as FP32 pairs).
  float* tc_a16 = nullptr;
  float* tc_b16 = nullptr;
  int tc16_katoms = 0;
  CUtensorMap tm_tc_a16{}, tm_tc_b16{};

  // Symmetric Gram product: work-unit table (row tile, first and end column tile).
  int4* sym_units = nullptr;
  int sym_nunits = 0, sym_T = 0;
  int4* tc_sym_units = nullptr;       // the same for the symmetric tensor-core tiles (fewer, longer units)
  int tc_sym_nunits = 0, tc_sym_T = 0;

  // Gram-product scratch.
  float* part = nullptr;  size_t part_cap = 0;      // per-split partial sums (bytes)
  float* v32 = nullptr;   size_t v32_cap = 0;       // FP32 / hi-lo copy of V (bytes)

  // Solver vectors (FP64, length ldn each) and scalars.
  double* vec_pool = nullptr;
  double* scal = nullptr;              // device scalars
  double* scal_host = nullptr;         // pinned mirror
  unsigned int* red_counter = nullptr; // last-block counters of the reductions
  double* red_part = nullptr;          // per-block reduction partials
  int* err_flag = nullptr;             // device error word written by kernels

  // Last solve state (device): alpha, v, z and beta.
  double* st_alpha = nullptr;
  double* st_v = nullptr;
  double* st_z = nullptr;
  double st_beta = 0.0;
  double st_tau = 0.0, st_lam = 0.0;   // (tau, lambda) of the last solve
  bool has_state = false;

  int64_t launches = 0;
  std::string err;
  // Event timing of the Gram tile kernels (kqr_profile): pairs per kernel id.
  bool profile = false;
  std::vector<cudaEvent_t> prof_ev[3];
  size_t prof_used[3] = {0, 0, 0};
  int num_sms = 0;
  int64_t cg_truncations = 0;         // CG runs stopped at a non-positive curvature
  bool cg_met = false;                // the last CG run met its residual tolerance
  bool cg_truncated = false;          // the last CG run stopped at a non-positive (rounding-level) curvature
  double dres_mean = 1.0;             // RPCholesky's mean residual diagonal (before the floor)
  bool cg_high_on = false;            // this solve's CG products are FP64-class
  BatchData* batch = nullptr;         // set for batched-product handles (batch.cu)

  // CUDA graphs of a block of CG iterations (solver.cu), one per solution vector
  // (Phase I alpha, Phase II direction d); rebuilt when a pointer they captured changes.
  struct CgGraph {
    cudaGraphExec_t exec = nullptr;
    std::vector<const void*> key;
    int64_t launches = 0;              // kernel launches one graph launch stands for
  } cg_graph[2];
  bool cg_graphs_off = false;         // capture failed once: enqueue directly from then on

  // Grid solves (grid.cu): set on the per-column clones, whose products meet in the rendezvous.
  GridRdv* rdv = nullptr;
  cudaEvent_t rdv_ev = nullptr;
  int64_t grid_rounds = 0, grid_columns = 0;   // products run for grids, and columns they carried

  // Stored upper-triangle tiles of K (gram_stored.cu; options.gram_store), or null.
  float* kstore = nullptr;
  size_t kstore_bytes = 0;
  int4* kstore_sched = nullptr;       // per-CTA (first tile, end tile, I, J) of the product
  int kstore_grid = 0;
};

kqr_status fail(Handle* h, kqr_status s, const std::string& msg);
kqr_status cuda_fail(Handle* h, cudaError_t e, const char* what);
cudaStream_t pick_stream(Handle* h, void* stream);
// Records the start (begin = true) or end event of a profiled launch of kernel id k.
void prof_mark(Handle* h, int k, bool begin, cudaStream_t st);

// ---- vector kernels (vec_ops.cu) ------------------------------------------------
// Reductions: compute NS sums of per-element terms into out[0..NS) (device).
enum RedKind {
  RED_DOT = 0,         // x . y
  RED_SUM = 1,         // 1^T x
  RED_KKT = 2,         // 10 sums of the Sec. 4 residuals
  RED_LS_PRE = 3,      // line-search inner products
  RED_MOREAU_DIFF = 4, // sum dist^2(w + c d) - dist^2(w)
  RED_NORM2 = 5,       // ||x||^2
};
struct RedArgs {
  const double* a = nullptr; const double* b = nullptr; const double* c = nullptr;
  const double* d = nullptr; const double* e = nullptr;
  double s0 = 0, s1 = 0, s2 = 0, s3 = 0;
};
cudaError_t reduce(Handle* h, RedKind kind, const RedArgs& a, int64_t n, double* out, cudaStream_t st);

cudaError_t vec_fill(Handle* h, double* x, double val, int64_t n, cudaStream_t st);
cudaError_t vec_copy(Handle* h, double* dst, const double* src, int64_t n, cudaStream_t st);
// y = a * x + y (device scalar a read from *a_dev, scaled by sgn)
cudaError_t cg_update(Handle* h, double* x, double* Kx, double* r, const double* p, const double* Kp,
                      const double* Ap, const double* a_dev, int64_t n, double* rr_out, cudaStream_t st);
// p = z + beta p (beta read from beta_dev); a non-zero *stop_dev (nullable) skips it;
// ||p||^2 into *pp_out (device).
cudaError_t cg_direction(Handle* h, double* p, const double* z, const double* beta_dev, const double* stop_dev,
                         int64_t n, double* pp_out, cudaStream_t st);
cudaError_t op_residual(Handle* h, double* r, const double* b, const double* x, const double* Kx, double gam,
                        const double* sum_x, const double* L, int64_t n, cudaStream_t st);
cudaError_t admm_rhs(Handle* h, double* b, const double* y, double beta, const double* z, const double* v,
                     double sigma, double lam, int64_t n, cudaStream_t st);
cudaError_t admm_update(Handle* h, const double* alpha, double* v, double* z, double sigma, double tau,
                        double step, int64_t n, cudaStream_t st);
cudaError_t alm_update(Handle* h, const double* alpha, double* v, double* z, double sigma, double tau,
                       int64_t n, cudaStream_t st);
cudaError_t box_grad(Handle* h, const double* alpha, const double* z, const double* Kalpha, const double* y,
                     double beta, double sigma, double tau, double lam, double eps, const double* dres,
                     double* v, double* S, double* grad, double* Ldiag, double* Lpre, int64_t n, cudaStream_t st);
cudaError_t scale_vec(Handle* h, double* out, const double* x, double s, int64_t n, cudaStream_t st);
cudaError_t axpy_vec(Handle* h, double* y, const double* x, double a, int64_t n, cudaStream_t st);
cudaError_t fill_L(Handle* h, double* L, double base, const double* dres, int64_t n, cudaStream_t st);
// Bounded wait on an mbarrier nothing arrives on (the wait-timeout path; kqr_test_bounded_wait).
cudaError_t launch_wait_probe(Handle* h, uint32_t max_polls, cudaStream_t st);

// ---- preconditioner (woodbury.cu, rpchol.cu) -------------------------------------
kqr_status precond_build(Handle* h, const double* Ldiag, double gam, cudaStream_t st);
// As precond_build, but keeps the current core when it was built for the same gam
// and max_i |Lpre_i - Lcore_i| / Lcore_i <= rtol (the preconditioner stays SPD; only
// its distance to the exact P changes).  Lcore_i = 1 / Linv_i.
kqr_status precond_update(Handle* h, const double* Lpre, double gam, double rtol, cudaStream_t st);
cudaError_t precond_apply(Handle* h, const double* Ldiag, const double* r, double* out, double* rz_out,
                          cudaStream_t st);
kqr_status rpcholesky_setup(Handle* h, const double* uniforms);

// ---- solver (solver.cu) --------------------------------------------------------
kqr_status solve(Handle* h, double tau, double lam, double tol, kqr_info* info);
kqr_status pcg(Handle* h, const double* Ldiag, const double* Lpre, double gam, const double* b, double* x,
               double* Kx, bool warm, double tol, int maxit, int* iters, cudaStream_t st, bool lowprec = false);
// PCG whose products use the one-term TF32 tensor-core RBF product, iteratively
// refined against FP32 residuals until ||b - A x|| <= tol (FP32 operator);
// Kx receives the FP32 K x.  Counts FP32 and TF32 products.
kqr_status pcg_refined(Handle* h, const double* Ldiag, const double* Lpre, double gam, const double* b, double* x,
                       double* Kx, bool warm, double tol, int maxit, int* iters, int* fp32_products,
                       int* low_products, cudaStream_t st);
kqr_status kkt(Handle* h, const double* alpha, const double* v, double beta, const double* z,
               const double* Kalpha, double tau, double lam, double* out7, cudaStream_t st);

// One CG iteration after the Gram product K p has landed in vec(h, V_KP): the operator's
// other terms, the device-resident step lengths and stopping test, the preconditioner and
// the direction update (solver.cu).  Used by the grid's shared CG engine (grid.cu), which
// runs the products of several columns together and this chain on each column's stream.
struct CgArgs {
  const double* L = nullptr;
  const double* Lpre = nullptr;
  double gam = 0.0;
  double* x = nullptr;
  double* Kx = nullptr;
  double noise_coef = 0.0;
};
cudaError_t cg_after_product(Handle* h, const CgArgs& a, cudaStream_t st);
// Runs a grid column's CG (set up by pcg on the column's stream) in the grid's shared
// engine until its device status leaves "running" (grid.cu).
cudaError_t grid_cg(Handle* h, const CgArgs& a);

// Solver work vector slots in vec_pool.
enum Vec {
  V_ALPHA = 0, V_V, V_Z, V_KALPHA, V_B, V_D, V_KD, V_R, V_ZZ, V_P, V_AP, V_KP, V_L, V_LPRE, V_GRAD,
  V_S, V_TMP, V_TMP2, V_DX, V_RT, V_COUNT
};
inline double* vec(Handle* h, Vec v) { return h->vec_pool + (size_t)v * h->ldn; }

// Scalar slots in scal / scal_host.
enum Scal {
  S_RED0 = 0, S_SUMP = 16, S_PAP = 17, S_A = 18, S_BETA = 19, S_RR = 20, S_RZ = 21,
  // device-resident CG control (solver.cu): new rz, status, iterations, tol^2, pending status, maxit
  S_RZN = 22, S_CGST = 23, S_CGITS = 24, S_TOL2 = 25, S_PEND = 26, S_MAXIT = 27, S_GAM = 28, S_PP = 29,
  S_COUNT = 32
};

// Launch configuration for element-wise kernels.
// ---- batched multi-RHS products (batch.cu) ---------------------------------------
struct BatchData {
  int64_t B = 0, p = 0, R = 0;          // problems, features, padded rows (each problem to 128)
  std::vector<int64_t> off, roff;       // row offsets: caller's (dense) and padded
  int n_items = 0;
  double entries = 0.0;                 // sum_b n_b^2
  float* xt = nullptr;                  // [R][32] TF32 coordinates
  float* nrm = nullptr;                 // [R] squared norms
  float* vt = nullptr;                  // [64][R] TF32 right-hand sides
  int* items = nullptr;                 // [n_items][4]
  int* out0 = nullptr;                  // [n_items]
  int64_t* d_off = nullptr;
  int64_t* d_roff = nullptr;
  CUtensorMap tm_xi, tm_xj, tm_v;
  bool p_in_smem = false;               // stage the Gram tile through shared memory, not TMEM
};
kqr_status batch_create(Handle* h, const double* X, const int64_t* offsets, int64_t B, int64_t p,
                        const double* gammas, int32_t flags);
cudaError_t batch_kmatmul(Handle* h, const double* V, double* U, int m, cudaStream_t st);
void batch_free(Handle* h);
#define KQR_SINGLE(h)                                                                          \
  do {                                                                                         \
    if ((h)->batch) return fail((h), KQR_INVALID_ARG, "this call takes a single-problem handle"); \
  } while (0)

inline int grid_for(int64_t n, int threads = 256, int max_blocks = 1216) {
  int64_t b = (n + threads - 1) / threads;
  return (int)(b < 1 ? 1 : (b > max_blocks ? max_blocks : b));
}

}  // namespace kqr

// Opaque C handle wraps the internal one.
struct kqr_handle {
  kqr::Handle h;
};
