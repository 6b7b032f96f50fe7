// Two-phase PALM-KQR driver: Phase I inexact ADMM (Alg. 1) and Phase II
// semismooth Newton ALM (Alg. 2 with Alg. 3), with preconditioned CG for the
// linear systems (2.1) and (3.1).  Vectors live on the device; the host keeps
// the handful of scalars each step needs (step lengths, norms, sigma).
//
// Arithmetic: CG uses FP32 Gram products (entries ~1e-7 relative); the
// gradient of phi_k (eq. (2.3)), the line search and the KKT residuals of
// Sec. 4 use the FP64-class product, because they divide K alpha by lambda.
// Phase I's stopping test uses the K alpha that CG tracks (the FP32 operator):
// Phase I only supplies the warm start.
#include <chrono>
#include <cmath>
#include <cstdio>

#include "kqr_internal.h"

namespace kqr {

cudaError_t reduce_ls_pre(Handle* h, const double* Ka, const double* d, const double* Kd, const double* y,
                          const double* g, const double* alpha, int64_t n, double* out, cudaStream_t st);

#define CK(call)                                              \
  do {                                                        \
    cudaError_t _e = (call);                                  \
    if (_e != cudaSuccess) return cuda_fail(h, _e, #call);    \
  } while (0)
#define KS(call)                         \
  do {                                   \
    kqr_status _s = (call);              \
    if (_s != KQR_OK) return _s;         \
  } while (0)

static cudaError_t fetch(Handle* h, int slot, int count, cudaStream_t st) {
  cudaError_t e = cudaMemcpyAsync(h->scal_host + slot, h->scal + slot, sizeof(double) * count,
                                  cudaMemcpyDeviceToHost, st);
  if (e != cudaSuccess) return e;
  return cudaStreamSynchronize(st);
}

static cudaError_t put(Handle* h, int slot, double v, cudaStream_t st) {
  h->scal_host[slot] = v;
  return cudaMemcpyAsync(h->scal + slot, h->scal_host + slot, sizeof(double), cudaMemcpyHostToDevice, st);
}

static kqr_status check_device_flag(Handle* h, cudaStream_t st) {
  int flag = 0;
  cudaError_t e = cudaMemcpyAsync(&flag, h->err_flag, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(h, e, "error flag");
  if (flag) return fail(h, KQR_DEVICE_WAIT_TIMEOUT, "a Gram kernel gave up waiting for a tile copy");
  return KQR_OK;
}

// K p with the FP64-class (high) or FP32 product; a grid column (kqr_solve_grid) posts it
// to the columns' shared multi-right-hand-side product instead.
cudaError_t grid_product(Handle* h, const double* p, double* out, bool high, cudaStream_t st);
static cudaError_t raw_product(Handle* h, const double* p, double* out, bool high, cudaStream_t st) {
  if (h->rdv) return grid_product(h, p, out, high, st);
  return high ? gram_high(h, p, out, 1, st) : gram_f32(h, p, out, 1, nullptr, st);
}

// Ap = K p + gam (1^T p) 1 + L o p; Kp = K p; pAp into *dot.
__global__ void high_op_kernel(double* __restrict__ Ap, const double* __restrict__ Kp, const double* __restrict__ p,
                               const double* __restrict__ L, const double* __restrict__ sump, double gam, int64_t n) {
  const double sg = gam * (*sump);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    Ap[i] = Kp[i] + sg + L[i] * p[i];
}

static cudaError_t op_product(Handle* h, const double* p, double* Ap, double* Kp, const double* L, double gam,
                              double* sump, double* dot, bool high, cudaStream_t st) {
  RedArgs rs;
  rs.a = p;
  cudaError_t e = reduce(h, RED_SUM, rs, h->n, sump, st);
  if (e != cudaSuccess) return e;
  if ((e = raw_product(h, p, Kp, high, st)) != cudaSuccess) return e;
  high_op_kernel<<<grid_for(h->n), 256, 0, st>>>(Ap, Kp, p, L, sump, gam, h->n);
  h->launches++;
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  RedArgs rd;
  rd.a = p;
  rd.b = Ap;
  return reduce(h, RED_DOT, rd, h->n, dot, st);
}

// ---- device-resident CG control ---------------------------------------------------
// CG's scalars live in device slots; the update and direction kernels compute the step
// lengths and the stopping test themselves (in the CTA that finishes their reduction
// last), so the host reads one status word per block of iterations instead of three
// blocking copies per iteration.  Status (S_CGST):
// 0 running, 1 met tol, 2 stopped at a non-positive curvature, 3 non-finite, 4 maxit.
enum CgState { CG_RUN = 0, CG_MET = 1, CG_TRUNC = 2, CG_NONFINITE = 3, CG_MAXIT = 4 };

// Block sum of v over the CTA's 256 threads into part[blockIdx.x]; returns true in the
// CTA that finishes last, whose thread 0 then holds the sum over all CTAs (added in
// CTA order) in *total.  Resets the counter for the next reduction.
__device__ __forceinline__ bool cg_block_sum(double v, double* __restrict__ part, unsigned int* __restrict__ counter,
                                             double* total) {
  __shared__ double ws[8];
  __shared__ bool last;
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double b = 0.0;
    for (int w = 0; w < 8; ++w) b += ws[w];
    part[blockIdx.x] = b;
    __threadfence();
    last = (atomicAdd(counter, 1u) == gridDim.x - 1);
  }
  __syncthreads();
  if (!last) return false;
  if (threadIdx.x == 0) {
    __threadfence();
    double t = 0.0;
    for (int b = 0; b < (int)gridDim.x; ++b) t += __ldcg(part + b);
    *total = t;
    *counter = 0u;
  }
  return true;
}

// One CG step after p^T A p is known: the step length a = rz / pAp (rz in S_RZN), or the
// truncation step when the curvature is at or below the product's rounding level
// (noise_coef: that level per unit ||p||^2, 2^-22 sqrt(n) for FP32 entries and sums);
// x += a p, Kx += a Kp, r -= a Ap; then, in the CTA that finishes last, ||r||^2, the
// iteration count, rz copied to S_RZ for the next direction, and the status
// (0 running, 1 met tol, 2 rounding-level curvature, 3 non-finite, 4 maxit).  A stopped CG
// (status != 0, set by an earlier launch, so the same in every CTA) makes this a no-op.
__global__ void __launch_bounds__(256) cg_step_kernel(double* __restrict__ s, double noise_coef, double* __restrict__ x,
                                                      double* __restrict__ Kx, double* __restrict__ r,
                                                      const double* __restrict__ p, const double* __restrict__ Kp,
                                                      const double* __restrict__ Ap, int64_t n,
                                                      double* __restrict__ part, unsigned int* __restrict__ counter) {
  if ((int)s[S_CGST] != CG_RUN) return;
  const double pAp = s[S_PAP];
  double a;
  int pend;
  if (!isfinite(pAp)) {
    a = 0.0;
    pend = CG_NONFINITE;
  } else if (!(pAp > 4.0 * noise_coef * s[S_PP])) {
    // The operator is positive definite; a curvature at or below the product's
    // rounding level is rounding in directions whose eigenvalues lie below its
    // accuracy (a numerically low-rank K), and dividing by it would blow the step
    // up.  Truncate: keep x, or at the first step take the preconditioned residual
    // itself (a Newton step with the preconditioner as the Hessian model).
    a = s[S_CGITS] == 0.0 ? 1.0 : 0.0;
    pend = CG_TRUNC;
  } else {
    a = s[S_RZN] / pAp;
    pend = CG_RUN;
  }
  double acc = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    x[i] += a * p[i];
    if (Kx) Kx[i] += a * Kp[i];
    const double ri = r[i] - a * Ap[i];
    r[i] = ri;
    acc += ri * ri;
  }
  double rr;
  if (!cg_block_sum(acc, part, counter, &rr) || threadIdx.x != 0) return;
  s[S_RR] = rr;
  s[S_A] = a;
  s[S_RZ] = s[S_RZN];
  if (a != 0.0) s[S_CGITS] += 1.0;
  int st = pend;
  if (st == CG_RUN) {
    if (!isfinite(rr)) st = CG_NONFINITE;
    else if (rr <= s[S_TOL2]) st = CG_MET;
    else if (s[S_CGITS] >= s[S_MAXIT]) st = CG_MAXIT;
  }
  s[S_CGST] = st;
}

// p = z + beta p with beta = rz_new / rz (S_RZN, S_RZ), and ||p||^2 into S_PP, while CG runs.
__global__ void __launch_bounds__(256) cg_dir_kernel(double* __restrict__ s, double* __restrict__ p,
                                                     const double* __restrict__ z, int64_t n,
                                                     double* __restrict__ part, unsigned int* __restrict__ counter) {
  if ((int)s[S_CGST] != CG_RUN) return;
  const double b = s[S_RZN] / s[S_RZ];
  double acc = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double pi = z[i] + b * p[i];
    p[i] = pi;
    acc += pi * pi;
  }
  double pp;
  if (!cg_block_sum(acc, part, counter, &pp) || threadIdx.x != 0) return;
  s[S_PP] = pp;
  s[S_BETA] = b;
}

static cudaError_t cg_step(Handle* h, double noise_coef, double* x, double* Kx, double* r, const double* p,
                           const double* Kp, const double* Ap, cudaStream_t st) {
  cg_step_kernel<<<grid_for(h->n, 256, 304), 256, 0, st>>>(h->scal, noise_coef, x, Kx, r, p, Kp, Ap, h->n, h->red_part,
                                                           h->red_counter);
  h->launches++;
  return cudaGetLastError();
}

static cudaError_t cg_dir(Handle* h, double* p, const double* z, cudaStream_t st) {
  cg_dir_kernel<<<grid_for(h->n, 256, 304), 256, 0, st>>>(h->scal, p, z, h->n, h->red_part, h->red_counter);
  h->launches++;
  return cudaGetLastError();
}

__global__ void cg_init_kernel(double* __restrict__ s, double tol2, double maxit, double gam) {
  s[S_CGST] = CG_RUN;
  s[S_CGITS] = 0.0;
  s[S_TOL2] = tol2;
  s[S_MAXIT] = maxit;
  s[S_GAM] = gam;
}

// CG iterations per host status read: one per product when a product costs far more
// than a host round trip, more when the products are cheap (small n).
static int cg_block(Handle* h) {
  if (h->rdv) return 1;                 // grid columns meet at every product on the host
  if (h->n <= 8192) return 16;
  if (h->n <= 32768) return 4;
  return 1;
}

cudaError_t cg_after_product(Handle* h, const CgArgs& a, cudaStream_t st) {
  const int64_t n = h->n;
  double* s = h->scal;
  double* r = vec(h, V_R);
  double* zz = vec(h, V_ZZ);
  double* p = vec(h, V_P);
  double* Ap = vec(h, V_AP);
  double* Kp = vec(h, V_KP);
  RedArgs rs;
  rs.a = p;
  cudaError_t e = reduce(h, RED_SUM, rs, n, s + S_SUMP, st);
  if (e != cudaSuccess) return e;
  high_op_kernel<<<grid_for(n), 256, 0, st>>>(Ap, Kp, p, a.L, s + S_SUMP, a.gam, n);
  h->launches++;
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  RedArgs rd;
  rd.a = p;
  rd.b = Ap;
  if ((e = reduce(h, RED_DOT, rd, n, s + S_PAP, st)) != cudaSuccess) return e;
  if ((e = cg_step(h, a.noise_coef, a.x, a.Kx, r, p, Kp, Ap, st)) != cudaSuccess) return e;
  if ((e = precond_apply(h, a.Lpre, r, zz, s + S_RZN, st)) != cudaSuccess) return e;
  return cg_dir(h, p, zz, st);
}

kqr_status pcg(Handle* h, const double* L, const double* Lpre, double gam, const double* b, double* x, double* Kx,
               bool warm, double tol, int maxit, int* iters, cudaStream_t st, bool lowprec) {
  const int64_t n = h->n;
  double* r = vec(h, V_R);
  double* zz = vec(h, V_ZZ);
  double* p = vec(h, V_P);
  double* Ap = vec(h, V_AP);
  double* Kp = vec(h, V_KP);
  double* s = h->scal;
  h->cg_met = false;
  h->cg_truncated = false;
  if (!warm) {
    CK(vec_fill(h, x, 0.0, n, st));
    if (Kx) CK(vec_fill(h, Kx, 0.0, n, st));
    CK(vec_copy(h, r, b, n, st));
  } else {
    RedArgs ra;
    ra.a = x;
    CK(reduce(h, RED_SUM, ra, n, s + S_SUMP, st));
    CK(op_residual(h, r, b, x, Kx, gam, s + S_SUMP, L, n, st));
  }
  RedArgs rn;
  rn.a = r;
  CK(reduce(h, RED_NORM2, rn, n, s + S_RR, st));
  CK(precond_apply(h, Lpre, r, zz, s + S_RZN, st));
  CK(vec_copy(h, p, zz, n, st));
  RedArgs rp;
  rp.a = p;
  CK(reduce(h, RED_NORM2, rp, n, s + S_PP, st));
  cg_init_kernel<<<1, 1, 0, st>>>(s, tol * tol, (double)maxit, gam);
  h->launches++;
  CK(cudaGetLastError());
  CK(fetch(h, S_RR, 1, st));
  const double rr0 = h->scal_host[S_RR];
  if (!std::isfinite(rr0)) return fail(h, KQR_BREAKDOWN, "CG: non-finite residual");
  if (std::sqrt(rr0) <= tol) {
    if (iters) *iters = 0;
    h->cg_met = true;
    return KQR_OK;
  }
  const int block = cg_block(h);
  const bool high_products = (h->rdv || !lowprec) && h->cg_high_on;
  // TF32 CG (lowprec) is refined against FP32 residuals, which absorb its inaccuracy:
  // there the guard only keeps the step from overflowing on a near-zero curvature.
  const double noise_coef = std::sqrt((double)n) * (high_products ? std::ldexp(1.0, -44)
                                                                   : (lowprec ? std::ldexp(1.0, -40) : std::ldexp(1.0, -22)));
  // One block of CG iterations, every scalar on the device.
  auto enqueue_block = [&]() -> cudaError_t {
    cudaError_t e = cudaSuccess;
    for (int j = 0; j < block && e == cudaSuccess; ++j) {
      GramEpilogue ep;
      ep.gam = gam;
      ep.gam_dev = s + S_GAM;
      ep.sum_p = s + S_SUMP;
      ep.L = L;
      ep.pvec = p;
      ep.dot_out = s + S_PAP;
      ep.raw_out = Kp;
      if (h->rdv) e = op_product(h, p, Ap, Kp, L, gam, s + S_SUMP, s + S_PAP, h->cg_high_on, st);
      else if (h->cg_high_on && !lowprec) e = op_product(h, p, Ap, Kp, L, gam, s + S_SUMP, s + S_PAP, true, st);
      else if (lowprec) e = gram_rbf_tc(h, p, Ap, 1, false, &ep, st);
      else e = gram_f32(h, p, Ap, 1, &ep, st);
      if (e != cudaSuccess) break;
      if ((e = cg_step(h, noise_coef, x, Kx, r, p, Kp, Ap, st)) != cudaSuccess) break;
      if ((e = precond_apply(h, Lpre, r, zz, s + S_RZN, st)) != cudaSuccess) break;
      e = cg_dir(h, p, zz, st);
    }
    return e;
  };
  // With several iterations per status read, the block is captured once as a CUDA
  // graph and relaunched (kernel arguments are pointers and device scalars only;
  // gam is read from S_GAM).  A graph is captured only after a block has run
  // directly with the same buffers, so that every buffer the products use exists
  // before capture; later calls with the same buffers launch it from the start.
  const bool graphs = block > 1 && !h->profile && !h->cg_graphs_off && !h->rdv && !(h->cg_high_on && !lowprec);
  Handle::CgGraph* g = nullptr;
  std::vector<const void*> key;
  if (graphs) {
    g = &h->cg_graph[x == vec(h, V_ALPHA) ? 0 : 1];
    key = {x, Kx, b, L, Lpre, h->v32, h->part, h->F32, h->core, h->Linv, h->tvec, h->kstore, h->sym_units,
           h->tc_hi, reinterpret_cast<const void*>((intptr_t)(h->r * 8 + (lowprec ? 1 : 0) + 2 * h->opt.precond)),
           reinterpret_cast<const void*>((intptr_t)block), reinterpret_cast<const void*>(st)};
  }
  int state = CG_RUN, it = 0;
  bool first = true;
  if (h->rdv) {
    // a grid column: its iterations run in the grid's shared CG engine
    CgArgs ca;
    ca.L = L;
    ca.Lpre = Lpre;
    ca.gam = gam;
    ca.x = x;
    ca.Kx = Kx;
    ca.noise_coef = noise_coef;
    CK(grid_cg(h, ca));
    CK(fetch(h, S_RR, S_CGITS - S_RR + 1, st));
    state = (int)h->scal_host[S_CGST];
    it = (int)h->scal_host[S_CGITS];
  }
  while (state == CG_RUN) {
    if (graphs && !first && (!g->exec || g->key != key)) {
      // capture the block (relaxed mode: the launch helpers set kernel attributes)
      cudaGraph_t graph = nullptr;
      const int64_t l0 = h->launches;
      cudaError_t e = cudaStreamBeginCapture(st, cudaStreamCaptureModeRelaxed);
      cudaError_t e2 = e == cudaSuccess ? enqueue_block() : e;
      if (e == cudaSuccess) e = cudaStreamEndCapture(st, &graph);
      const int64_t nodes = h->launches - l0;
      h->launches = l0;
      if (e == cudaSuccess) e = e2;
      if (e == cudaSuccess && g->exec) {
        cudaGraphExecUpdateResultInfo info;
        if (cudaGraphExecUpdate(g->exec, graph, &info) != cudaSuccess) {
          cudaGetLastError();
          cudaGraphExecDestroy(g->exec);
          g->exec = nullptr;
        }
      }
      if (e == cudaSuccess && !g->exec) e = cudaGraphInstantiate(&g->exec, graph, 0);
      if (graph) cudaGraphDestroy(graph);
      if (e != cudaSuccess) {
        // leave graphs off for this handle and carry on with direct launches
        cudaGetLastError();
        if (g->exec) cudaGraphExecDestroy(g->exec);
        g->exec = nullptr;
        h->cg_graphs_off = true;
      } else {
        g->key = key;
        g->launches = nodes;
      }
    }
    if (graphs && g->exec && g->key == key && !h->cg_graphs_off) {
      CK(cudaGraphLaunch(g->exec, st));
      h->launches += g->launches;
    } else {
      CK(enqueue_block());
    }
    first = false;
    CK(fetch(h, S_RR, S_CGITS - S_RR + 1, st));
    state = (int)h->scal_host[S_CGST];
    it = (int)h->scal_host[S_CGITS];
  }
  if (iters) *iters = it;
  if (state == CG_NONFINITE) {
    KS(check_device_flag(h, st));
    return fail(h, KQR_BREAKDOWN, "CG: non-finite curvature or residual");
  }
  if (state == CG_TRUNC) {
    h->cg_truncations++;
    h->cg_truncated = true;
  }
  h->cg_met = state == CG_MET;
  KS(check_device_flag(h, st));
  return KQR_OK;
}

__global__ void residual_kernel(double* __restrict__ r, const double* __restrict__ b, const double* __restrict__ Ax,
                                int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    r[i] = b[i] - Ax[i];
}

kqr_status pcg_refined(Handle* h, const double* L, const double* Lpre, double gam, const double* b, double* x,
                       double* Kx, bool warm, double tol, int maxit, int* iters, int* fp32_products,
                       int* low_products, cudaStream_t st) {
  const int64_t n = h->n;
  double* rt = vec(h, V_RT);
  double* dx = vec(h, V_DX);
  int total = 0, nf = 0, nl = 0;
  if (!warm) {
    CK(vec_fill(h, x, 0.0, n, st));
    if (Kx) CK(vec_fill(h, Kx, 0.0, n, st));
  }
  const int max_rounds = 6;
  for (int round = 0;; ++round) {
    // FP32 residual of the current x (x = 0 needs no product).
    if (round == 0 && !warm) {
      CK(vec_copy(h, rt, b, n, st));
    } else {
      GramEpilogue ep;
      ep.gam = gam;
      ep.sum_p = h->scal + S_SUMP;
      ep.L = L;
      ep.pvec = x;
      ep.raw_out = Kx;
      CK(gram_f32(h, x, rt, 1, &ep, st));
      ++nf;
      residual_kernel<<<grid_for(n), 256, 0, st>>>(rt, b, rt, n);
      h->launches++;
      CK(cudaGetLastError());
    }
    RedArgs rn;
    rn.a = rt;
    CK(reduce(h, RED_NORM2, rn, n, h->scal + S_RR, st));
    CK(fetch(h, S_RR, 1, st));
    const double rr = std::sqrt(h->scal_host[S_RR]);
    if (!std::isfinite(rr)) return fail(h, KQR_BREAKDOWN, "refined CG: non-finite residual");
    if (rr <= tol || round == max_rounds) break;
    // Correction from the TF32 operator: its ~1e-3 relative error limits one
    // round to a ~1e-2 reduction, so do not ask for more.
    int its = 0;
    KS(pcg(h, L, Lpre, gam, rt, dx, nullptr, false, std::fmax(tol, 1e-2 * rr), maxit, &its, st, true));
    total += its;
    nl += its;
    CK(axpy_vec(h, x, dx, 1.0, n, st));
  }
  if (iters) *iters = total;
  if (fp32_products) *fp32_products += nf;
  if (low_products) *low_products += nl;
  return KQR_OK;
}

kqr_status kkt(Handle* h, const double* alpha, const double* v, double beta, const double* z, const double* Kalpha,
               double tau, double lam, double* out7, cudaStream_t st) {
  RedArgs ra;
  ra.a = alpha; ra.b = v; ra.c = z; ra.d = h->y; ra.e = Kalpha;
  ra.s0 = beta; ra.s1 = tau; ra.s2 = lam;
  CK(reduce(h, RED_KKT, ra, h->n, h->scal + S_RED0, st));
  CK(fetch(h, S_RED0, 10, st));
  const double* s = h->scal_host + S_RED0;
  const double eta_p = std::sqrt(s[0]) / (1.0 + std::sqrt(s[6]));
  const double eta_d = std::sqrt(s[1] * s[1] + s[2]) / (1.0 + std::sqrt(s[3]));
  const double eta_c = std::sqrt(s[4]) / (1.0 + std::sqrt(s[5]));
  const double quad = s[7] / (2.0 * lam);
  const double objp = s[9] + quad;
  const double objd = -quad + s[8];
  out7[0] = eta_p;
  out7[1] = eta_d;
  out7[2] = eta_c;
  out7[3] = std::fmax(eta_p, std::fmax(eta_d, eta_c));
  out7[4] = std::fabs(objp - objd) / (1.0 + std::fabs(objp) + std::fabs(objd));
  out7[5] = objp;
  out7[6] = objd;
  return KQR_OK;
}

__global__ void make_L_kernel(double* L, double* Lpre, const double* S, double a, double b, const double* dres,
                              int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double li = a * (1.0 - S[i]) + b;
    L[i] = li;
    Lpre[i] = li + (dres ? dres[i] : 0.0);
  }
}

static double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

// options.cg_high = 2: a CG run that stopped at a rounding-level curvature shows
// that the FP32 products cannot resolve this operator (a numerically low-rank K);
// the rest of the solve runs its CG products FP64-class.
static void adapt_cg_products(Handle* h) {
  if (h->opt.cg_high == 2 && !h->cg_high_on && h->cg_truncated && !(h->opt.cg_tf32 && h->kind == KQR_RBF))
    h->cg_high_on = true;
}

kqr_status solve(Handle* h, double tau, double lam, double tol, kqr_info* info) {
  const kqr_options& o = h->opt;
  const int64_t n = h->n;
  cudaStream_t st = h->stream;
  const double t_start = now_s();
  double* alpha = vec(h, V_ALPHA);
  double* v = vec(h, V_V);
  double* z = vec(h, V_Z);
  double* Ka = vec(h, V_KALPHA);
  double* b = vec(h, V_B);
  double* d = vec(h, V_D);
  double* Kd = vec(h, V_KD);
  double* L = vec(h, V_L);
  double* Lpre = vec(h, V_LPRE);
  double* g = vec(h, V_GRAD);
  double* S = vec(h, V_S);
  const double* dres = (o.precond == KQR_PRECOND_NYSTROM_DIAG) ? h->dres : nullptr;
  const bool mixed = o.cg_tf32 && h->kind == KQR_RBF;
  h->cg_high_on = !mixed && (o.cg_high == 1 || (o.cg_high == 2 && h->dres_mean < std::ldexp((double)n, -24)));
  kqr_info inf{};
  inf.rank = h->r;
  inf.gram_stored = h->kstore ? 1 : 0;
  const int64_t builds0 = h->core_builds;
  const int64_t trunc0 = h->cg_truncations;
  double res[7] = {0, 0, 0, 0, 0, 0, 0};
  CK(vec_fill(h, alpha, 0.0, n, st));
  CK(vec_fill(h, v, 0.0, n, st));
  CK(vec_fill(h, z, 0.0, n, st));
  CK(vec_fill(h, Ka, 0.0, n, st));
  CK(cudaMemsetAsync(h->err_flag, 0, sizeof(int), st));
  double beta = 0.0;
  double sigma = o.sigma0;
  RedArgs ry;
  ry.a = h->y;
  CK(reduce(h, RED_NORM2, ry, n, h->scal + S_RED0 + 14, st));
  CK(fetch(h, S_RED0 + 14, 1, st));
  const double ynorm = std::sqrt(h->scal_host[S_RED0 + 14]);
  auto timed_out = [&]() { return o.time_limit_s > 0 && now_s() - t_start > o.time_limit_s; };
  kqr_status status = KQR_OK;

  // ---------------- Phase I: inexact ADMM (Alg. 1) ----------------
  CK(fill_L(h, L, lam * sigma, nullptr, n, st));
  CK(fill_L(h, Lpre, lam * sigma, dres, n, st));
  KS(precond_build(h, Lpre, lam * sigma, st));
  int k = 0;
  for (k = 0; k < o.admm_maxit; ++k) {
    CK(admm_rhs(h, b, h->y, beta, z, v, sigma, lam, n, st));
    RedArgs rb;
    rb.a = b;
    CK(reduce(h, RED_NORM2, rb, n, h->scal + S_RED0 + 15, st));
    CK(fetch(h, S_RED0 + 15, 1, st));
    // inexactness eps_k = admm_cg_rtol ||b_k|| / (k + 1)^1.5: summable while ||b_k|| stays bounded
    const double eps_k = o.admm_cg_rtol * std::sqrt(h->scal_host[S_RED0 + 15]) / std::pow(k + 1.0, 1.5);
    int its = 0;
    if (mixed) {
      KS(pcg_refined(h, L, Lpre, lam * sigma, b, alpha, Ka, k > 0, eps_k, o.pcg_maxit, &its, &inf.matvecs_fp32,
                     &inf.matvecs_low, st));
    } else {
      const bool high_before = h->cg_high_on;
      KS(pcg(h, L, Lpre, lam * sigma, b, alpha, Ka, k > 0, eps_k, o.pcg_maxit, &its, st));
      (high_before ? inf.matvecs_high : inf.matvecs_fp32) += its;
      adapt_cg_products(h);
    }
    inf.pcg_iters += its;
    RedArgs rs;
    rs.a = alpha;
    CK(reduce(h, RED_SUM, rs, n, h->scal + S_RED0 + 11, st));
    CK(fetch(h, S_RED0 + 11, 1, st));
    beta += o.gamma_admm * sigma * h->scal_host[S_RED0 + 11];
    CK(admm_update(h, alpha, v, z, sigma, tau, o.gamma_admm * sigma, n, st));
    KS(kkt(h, alpha, v, beta, z, Ka, tau, lam, res, st));
    if (o.verbose)
      fprintf(stderr, "[kqr] admm %3d sigma %.3g cg %4d eta_p %.2e eta_d %.2e eta_c %.2e gap %.2e\n", k, sigma, its,
              res[0], res[1], res[2], res[4]);
    if (std::fmax(res[3], res[4]) <= o.admm_tol) {
      ++k;
      break;
    }
    if (timed_out()) {
      status = fail(h, KQR_TIMEOUT, "time limit in Phase I");
      ++k;
      break;
    }
    if (o.balance_every > 0 && (k + 1) % o.balance_every == 0) {
      double ns = sigma;
      if (res[1] > o.balance_ratio * res[0]) ns = sigma * o.balance_factor;
      else if (res[0] > o.balance_ratio * res[1]) ns = sigma / o.balance_factor;
      if (ns != sigma) {
        sigma = ns;
        CK(fill_L(h, L, lam * sigma, nullptr, n, st));
        CK(fill_L(h, Lpre, lam * sigma, dres, n, st));
        KS(precond_build(h, Lpre, lam * sigma, st));
      }
    }
  }
  inf.phase1_iters = k;

  // FP64-class K alpha from here on.
  CK(raw_product(h, alpha, Ka, true, st));
  inf.matvecs_high++;
  KS(kkt(h, alpha, v, beta, z, Ka, tau, lam, res, st));
  bool converged = std::fmax(res[3], res[4]) <= tol;

  // ---------------- Phase II: SSN-ALM (Alg. 2, Alg. 3) ----------------
  if (!o.phase1_only && !converged && status == KQR_OK) {
    double g0 = -1.0, prev_eta_d = -1.0;
    sigma = std::fmax(sigma, o.sigma_alm_scale / lam);
    int kk = 0;
    for (kk = 0; kk < o.alm_maxit; ++kk) {
      // Alg. 3: Newton steps on phi_k with (beta, z, sigma) fixed.
      double tol_grad = 0.0;
      for (int t = 0; t < o.ssn_maxit; ++t) {
        CK(box_grad(h, alpha, z, Ka, h->y, beta, sigma, tau, lam, 0.0, nullptr, nullptr, S, g, nullptr, nullptr, n,
                    st));
        CK(fetch(h, S_RED0 + 13, 1, st));
        const double ng = std::sqrt(h->scal_host[S_RED0 + 13]);
        if (g0 < 0) g0 = ng;
        if (t == 0) tol_grad = std::fmax(0.1 * tol * (1.0 + ynorm), g0 * std::pow(0.2, kk + 1));
        if (!std::isfinite(ng)) return fail(h, KQR_BREAKDOWN, "non-finite gradient");
        if (ng <= tol_grad) break;
        const double eps = o.tau1 * std::fmin(o.tau2, ng);
        make_L_kernel<<<grid_for(n), 256, 0, st>>>(L, Lpre, S, lam * sigma, lam * eps, dres, n);
        h->launches++;
        CK(cudaGetLastError());
        KS(precond_update(h, Lpre, lam * sigma, o.core_reuse_rtol, st));
        CK(scale_vec(h, b, g, -lam, n, st));
        const double ptol = lam * std::fmin(o.eta_bar, std::pow(ng, 1.0 + o.iota));
        int its = 0;
        if (mixed) {
          KS(pcg_refined(h, L, Lpre, lam * sigma, b, d, Kd, false, ptol, o.pcg_maxit, &its, &inf.matvecs_fp32,
                         &inf.matvecs_low, st));
        } else {
          const bool high_before = h->cg_high_on;
          KS(pcg(h, L, Lpre, lam * sigma, b, d, Kd, false, ptol, o.pcg_maxit, &its, st));
          (high_before ? inf.matvecs_high : inf.matvecs_fp32) += its;
          adapt_cg_products(h);
        }
        inf.pcg_iters += its;
        // Armijo backtracking on phi_k(alpha + c d) - phi_k(alpha), term by term.
        CK(reduce_ls_pre(h, Ka, d, Kd, h->y, g, alpha, n, h->scal + S_RED0, st));
        CK(fetch(h, S_RED0, 6, st));
        const double Kad = h->scal_host[S_RED0 + 0], dKd = h->scal_host[S_RED0 + 1];
        const double yd = h->scal_host[S_RED0 + 2], sd = h->scal_host[S_RED0 + 3];
        const double gd = h->scal_host[S_RED0 + 4], sa = h->scal_host[S_RED0 + 5];
        const double s0 = sa + beta / sigma;
        double c = 1.0;
        for (int ls = 0; ls < o.ls_maxit; ++ls) {
          RedArgs rm;
          rm.a = alpha; rm.b = z; rm.c = d;
          rm.s0 = sigma; rm.s1 = tau; rm.s2 = c;
          CK(reduce(h, RED_MOREAU_DIFF, rm, n, h->scal + S_RED0 + 8, st));
          CK(fetch(h, S_RED0 + 8, 1, st));
          const double md = h->scal_host[S_RED0 + 8];
          const double dphi = (c * Kad + 0.5 * c * c * dKd) / lam - c * yd +
                              0.5 * sigma * ((s0 + c * sd) * (s0 + c * sd) - s0 * s0) + 0.5 * sigma * md;
          if (dphi <= o.mu * c * gd) break;
          c *= o.r_ls;
        }
        CK(axpy_vec(h, alpha, d, c, n, st));
        CK(raw_product(h, alpha, Ka, true, st));
        inf.matvecs_high++;
        inf.newton_steps++;
        if (o.verbose)
          fprintf(stderr, "[kqr]   ssn %d |grad| %.3e eps %.1e cg %4d step %.3g\n", t, ng, eps, its, c);
        if (timed_out()) break;
      }
      // Alg. 2 multiplier updates.
      RedArgs rs;
      rs.a = alpha;
      CK(reduce(h, RED_SUM, rs, n, h->scal + S_RED0 + 11, st));
      CK(fetch(h, S_RED0 + 11, 1, st));
      beta += sigma * h->scal_host[S_RED0 + 11];
      CK(alm_update(h, alpha, v, z, sigma, tau, n, st));
      KS(kkt(h, alpha, v, beta, z, Ka, tau, lam, res, st));
      if (o.verbose)
        fprintf(stderr, "[kqr] alm %3d sigma %.3g eta_p %.2e eta_d %.2e eta_c %.2e gap %.2e\n", kk, sigma, res[0],
                res[1], res[2], res[4]);
      if (std::fmax(res[3], res[4]) <= tol) {
        converged = true;
        ++kk;
        break;
      }
      if (timed_out()) {
        status = fail(h, KQR_TIMEOUT, "time limit in Phase II");
        ++kk;
        break;
      }
      if (prev_eta_d >= 0 && res[1] > 0.5 * prev_eta_d) sigma = std::fmin(o.sigma_max, sigma * o.sigma_factor);
      prev_eta_d = res[1];
    }
    inf.phase2_iters = kk;
  }
  KS(check_device_flag(h, st));
  CK(vec_copy(h, h->st_alpha, alpha, n, st));
  CK(vec_copy(h, h->st_v, v, n, st));
  CK(vec_copy(h, h->st_z, z, n, st));
  CK(cudaStreamSynchronize(st));
  h->st_beta = beta;
  h->st_tau = tau;
  h->st_lam = lam;
  h->has_state = true;
  inf.eta_p = res[0];
  inf.eta_d = res[1];
  inf.eta_c = res[2];
  inf.eta_kkt = res[3];
  inf.eta_gap = res[4];
  inf.obj_p = res[5];
  inf.obj_d = res[6];
  inf.sigma_final = sigma;
  inf.core_builds = (int32_t)(h->core_builds - builds0);
  inf.cg_truncations = (int32_t)(h->cg_truncations - trunc0);
  inf.seconds = now_s() - t_start;
  inf.cg_high_used = h->cg_high_on ? 1 : 0;
  if (info) *info = inf;
  if (status != KQR_OK) return status;
  if (o.phase1_only) return KQR_OK;
  if (!converged) return fail(h, KQR_NOT_CONVERGED, "iteration cap reached");
  return KQR_OK;
}

}  // namespace kqr
