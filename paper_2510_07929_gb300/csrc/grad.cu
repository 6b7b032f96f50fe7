// Held-out check loss of a solved problem and its gradient with respect to
// log gamma, log lambda and the training inputs X, by implicit
// differentiation through the KKT conditions at the solution.  This extends
// the method (the paper has no counterpart); it builds on the dual (1.3), the
// representer form f(x) = beta + (1/lambda) sum_j alpha_j k(x_j, x) (Sec. 1)
// and the KKT conditions of Sec. 4.  RBF kernel, k = exp(-gamma ||x - x'||^2).
//
// With E = {i : tau - 1 < alpha_i < tau} held fixed, (alpha_E, beta) solve
//   F_E = (K alpha)_E / lambda + beta - y_E = 0,  1^T alpha = 0.
// For the held-out loss l = sum_h rho_tau(y_h - f_h) with g_h = d rho / d f_h,
// let a = [(K_{E,h} g) / lambda ; sum_h g_h] and solve
//   [K_EE / lambda, 1; 1^T, 0] [u; w] = a
// (two CG solves with K_EE, FP64-class products, on the training problem's
// preconditioner); then
//   dl/dtheta = g^T (d f_h / d theta)|_{alpha,beta} - u^T (d F_E / d theta)|_{alpha,beta}.
// Every Gram-weighted sum the partial derivatives need is a product of the
// tiled Gram kernels with one of the vectors
//   b1 = [alpha; 0], b2 = [0; g], b3 = [u; 0]  (over the points [X; Xh]),
// multiplied element-wise by 1, the centred squared norm, or one coordinate:
//   ((D o K) b)_i = |x_i|^2 (K b)_i + (K (|x|^2 o b))_i - 2 sum_c x_ic (K (x_c o b))_i,
//   sum_j K_kj b_j (x_kc - x_jc) = x_kc (K b)_k - (K (x_c o b))_k,
// so the Gram tiles are recomputed, never stored.  Every product is FP64-class: the
// 1/lambda factors and the cancellation in x_k (K b)_k - (K x b)_k amplify FP32 errors.
#include <cmath>
#include <vector>

#include "kqr_internal.h"

namespace kqr {

#define GRID_LOOP(i, n) \
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (n); i += (int64_t)gridDim.x * blockDim.x)

// Block sum of v added atomically to *out.  The leading barrier keeps a second call in the
// same kernel from overwriting ws while thread 0 still reads the first call's values.
__device__ __forceinline__ void block_add(double v, double* out) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __shared__ double ws[32];
  __syncthreads();
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += ws[w];
    atomicAdd(out, t);
  }
}

// Held-out residuals: f_h = beta + Kb1[n + h] / lambda; loss, sum g; b2 = [0; g].
__global__ void heldout_kernel(const double* __restrict__ Kb1, const double* __restrict__ yh, int64_t n, int64_t nh,
                               double beta, double tau, double lam, double* __restrict__ b2, double* __restrict__ sums) {
  double loss = 0.0, gs = 0.0;
  GRID_LOOP(h, nh) {
    const double r = yh[h] - (beta + Kb1[n + h] / lam);
    loss += r > 0.0 ? tau * r : -(1.0 - tau) * r;
    const double g = r > 0.0 ? -tau : 1.0 - tau;
    b2[n + h] = g;
    gs += g;
  }
  block_add(loss, sums + 0);
  block_add(gs, sums + 1);
}

// Elbow set from the consensus variable v; right-hand sides and diagonal of the K_EE solves.
__global__ void elbow_kernel(const double* __restrict__ v, const double* __restrict__ Kb2, int64_t n, double tau,
                             double lam, double edge, double big, double small, double* __restrict__ rhs1,
                             double* __restrict__ rhs2, double* __restrict__ L, double* __restrict__ mask,
                             double* __restrict__ sums) {
  double cnt = 0.0;
  GRID_LOOP(i, n) {
    const bool e = v[i] > tau - 1.0 + edge && v[i] < tau - edge;
    mask[i] = e ? 1.0 : 0.0;
    rhs1[i] = e ? Kb2[i] : 0.0;          // lambda * a_E, a_E = (K_{X,h} g)_E / lambda
    rhs2[i] = e ? 1.0 : 0.0;
    L[i] = e ? small : big;
    cnt += e ? 1.0 : 0.0;
  }
  block_add(cnt, sums + 2);
}

// sum_i mask_i x_i and sum_i mask_i y_i
__global__ void masked_sums_kernel(const double* __restrict__ x, const double* __restrict__ y,
                                   const double* __restrict__ mask, int64_t n, double* __restrict__ out) {
  double a = 0.0, b = 0.0;
  GRID_LOOP(i, n) {
    a += mask[i] * x[i];
    b += mask[i] * y[i];
  }
  block_add(a, out + 0);
  block_add(b, out + 1);
}

// u = mask (s1 - c s2), written into b3 = [u; 0] (length N).
__global__ void adjoint_kernel(const double* __restrict__ s1, const double* __restrict__ s2,
                               const double* __restrict__ mask, int64_t n, int64_t N, double c,
                               double* __restrict__ b3) {
  GRID_LOOP(i, N) b3[i] = i < n ? mask[i] * (s1[i] - c * s2[i]) : 0.0;
}

// Columns of a multi-RHS block: V[i * 8 + j] = base[i] * mult(col0 + j, i), where
// multiplier index 0 is 1, index 1 is |x_i|^2, index 1 + c is x_ic (centred).
// Columns of a multi-RHS block (row-major, ncols columns): V[i * ncols + j] =
// base[i] * mult(col0 + j, i), where multiplier index 0 is 1 (or |x_i|^2 when
// first_norm), and index 1 + c is x_ic (centred).
__global__ void cols_kernel(const double* __restrict__ base, const double* __restrict__ xc, int64_t ldn,
                            const double* __restrict__ nrm, int64_t N, int col0, int ncols, int first_norm,
                            double* __restrict__ V) {
  GRID_LOOP(e, N * ncols) {
    const int64_t i = e / ncols;
    const int c = col0 + (int)(e % ncols);
    double m = 1.0;
    if (c == 0) m = first_norm ? nrm[i] : 1.0;
    else m = xc[(size_t)(c - 1) * ldn + i];
    V[e] = base[i] * m;
  }
}

__global__ void scatter_cols_kernel(const double* __restrict__ U, int64_t N, int col0, int ncols, int64_t ldr,
                                    double* __restrict__ R) {
  GRID_LOOP(e, N * ncols) {
    const int64_t i = e / ncols;
    const int j = (int)(e % ncols);
    R[(size_t)(col0 + j) * ldr + i] = U[e];
  }
}

__global__ void sqnorm_kernel(const double* __restrict__ xc, int64_t ldn, int p, int64_t N, double* __restrict__ nrm) {
  GRID_LOOP(i, N) {
    double s = 0.0;
    for (int c = 0; c < p; ++c) {
      const double x = xc[(size_t)c * ldn + i];
      s += x * x;
    }
    nrm[i] = s;
  }
}

// Scalar gradient pieces.  R1 columns: K b1 (col 0 computed in FP64-class separately
// and passed as Kb1), K(|x|^2 b1), K(x_c b1).
//   (D o K) b1 at row i = nrm_i Kb1_i + R1n_i - 2 sum_c x_ic R1c_i.
__global__ void scalar_grad_kernel(const double* __restrict__ Kb1, const double* __restrict__ R1, int64_t ldr,
                                   const double* __restrict__ xc, int64_t ldn, const double* __restrict__ nrm, int p,
                                   const double* __restrict__ b2, const double* __restrict__ b3, int64_t n, int64_t N,
                                   double* __restrict__ sums) {
  double dlam = 0.0, dgam = 0.0;
  GRID_LOOP(i, N) {
    double dk = nrm[i] * Kb1[i] + R1[(size_t)0 * ldr + i];
    for (int c = 0; c < p; ++c) dk -= 2.0 * xc[(size_t)c * ldn + i] * R1[(size_t)(1 + c) * ldr + i];
    if (i >= n) {                 // held-out rows: g^T d f_h
      const double g = b2[i];
      dlam += -g * Kb1[i];
      dgam += -g * dk;
    } else {                      // training rows in E: - u^T d F_E
      const double u = b3[i];
      dlam += u * Kb1[i];
      dgam += u * dk;
    }
  }
  block_add(dlam, sums + 0);
  block_add(dgam, sums + 1);
}

// dX_kc = -(2 gamma / lambda) alpha_k [x_kc (K b2)_k - (K x_c b2)_k]
//         + (2 gamma / lambda) [u_k (x_kc (K b1)_k - (K x_c b1)_k) + alpha_k (x_kc (K b3)_k - (K x_c b3)_k)]
// written row-major n x p.
__global__ void dx_kernel(const double* __restrict__ alpha, const double* __restrict__ u,
                          const double* __restrict__ Kb1, const double* __restrict__ R1, const double* __restrict__ R2,
                          const double* __restrict__ R3, int64_t ldr, const double* __restrict__ xc, int64_t ldn,
                          int p, int64_t n, double coef, double* __restrict__ dX) {
  GRID_LOOP(e, n * p) {
    const int64_t k = e / p;
    const int c = (int)(e % p);
    const double x = xc[(size_t)c * ldn + k];
    const double t2 = x * R2[k] - R2[(size_t)(1 + c) * ldr + k];
    const double t1 = x * Kb1[k] - R1[(size_t)(1 + c) * ldr + k];
    const double t3 = x * R3[k] - R3[(size_t)(1 + c) * ldr + k];
    dX[e] = coef * (-alpha[k] * t2 + u[k] * t1 + alpha[k] * t3);
  }
}

// Ap = K p + gam (1^T p) 1 + L o p, with K p from the FP64-class product.
__global__ void adj_op_kernel(double* __restrict__ Ap, const double* __restrict__ Kp, const double* __restrict__ p,
                              const double* __restrict__ L, const double* __restrict__ sump, double gam, int64_t n) {
  const double sg = gam * (*sump);
  GRID_LOOP(i, n) Ap[i] = Kp[i] + sg + L[i] * p[i];
}

__global__ void adj_step_kernel(double* __restrict__ x, double* __restrict__ r, const double* __restrict__ p,
                                const double* __restrict__ Ap, double a, int64_t n) {
  GRID_LOOP(i, n) {
    x[i] += a * p[i];
    r[i] -= a * Ap[i];
  }
}

__global__ void adj_dir_kernel(double* __restrict__ p, const double* __restrict__ z, double b, int64_t n) {
  GRID_LOOP(i, n) p[i] = z[i] + b * p[i];
}

// PCG on (K + gam 1 1^T + diag(L)) x = b with FP64-class Gram products and the problem's
// Woodbury preconditioner (built for Lpre).  The adjoint system is as ill-conditioned as
// K on the elbow set, where FP32 products would cap the gradient's accuracy.  dsc: 4
// device doubles of scratch.
static kqr_status adjoint_cg(Handle* h, const double* L, const double* Lpre, double gam, const double* b, double* x,
                             double tol, int maxit, double* dsc, cudaStream_t st) {
  const int64_t n = h->n;
  double* r = vec(h, V_R);
  double* z = vec(h, V_ZZ);
  double* p = vec(h, V_P);
  double* Kp = vec(h, V_KP);
  double* Ap = vec(h, V_AP);
  double hs[4];
  auto get = [&](int k) -> cudaError_t {
    cudaError_t e = cudaMemcpyAsync(hs + k, dsc + k, sizeof(double), cudaMemcpyDeviceToHost, st);
    return e == cudaSuccess ? cudaStreamSynchronize(st) : e;
  };
#define AK(call)                                              \
  do {                                                        \
    cudaError_t _e = (call);                                  \
    if (_e != cudaSuccess) return cuda_fail(h, _e, #call);    \
  } while (0)
  AK(vec_fill(h, x, 0.0, n, st));
  AK(vec_copy(h, r, b, n, st));
  RedArgs rn;
  rn.a = r;
  AK(reduce(h, RED_NORM2, rn, n, dsc + 0, st));
  AK(get(0));
  if (std::sqrt(hs[0]) <= tol) return KQR_OK;
  AK(precond_apply(h, Lpre, r, z, dsc + 1, st));
  AK(get(1));
  double rz = hs[1];
  AK(vec_copy(h, p, z, n, st));
  for (int it = 0; it < maxit; ++it) {
    RedArgs rs;
    rs.a = p;
    AK(reduce(h, RED_SUM, rs, n, dsc + 2, st));
    AK(gram_high(h, p, Kp, 1, st));
    adj_op_kernel<<<grid_for(n), 256, 0, st>>>(Ap, Kp, p, L, dsc + 2, gam, n);
    AK(cudaGetLastError());
    RedArgs rd;
    rd.a = p;
    rd.b = Ap;
    AK(reduce(h, RED_DOT, rd, n, dsc + 3, st));
    AK(get(3));
    const double pAp = hs[3];
    if (!std::isfinite(pAp)) return fail(h, KQR_BREAKDOWN, "adjoint CG: non-finite curvature");
    if (!(pAp > 0.0)) break;
    adj_step_kernel<<<grid_for(n), 256, 0, st>>>(x, r, p, Ap, rz / pAp, n);
    AK(cudaGetLastError());
    AK(reduce(h, RED_NORM2, rn, n, dsc + 0, st));
    AK(get(0));
    if (std::sqrt(hs[0]) <= tol) break;
    AK(precond_apply(h, Lpre, r, z, dsc + 1, st));
    AK(get(1));
    adj_dir_kernel<<<grid_for(n), 256, 0, st>>>(p, z, hs[1] / rz, n);
    AK(cudaGetLastError());
    rz = hs[1];
  }
#undef AK
  return KQR_OK;
}

}  // namespace kqr

using namespace kqr;

extern "C" kqr_status kqr_heldout_grad(kqr_handle* kh, const double* X, const double* Xh, const double* yh, int64_t nh,
                                       double* loss, double* d_loggamma, double* d_loglambda, double* dX) {
  if (!kh) return KQR_INVALID_ARG;
  Handle* h = &kh->h;
  KQR_SINGLE(h);
  if (!X || !Xh || !yh || nh < 1) return fail(h, KQR_INVALID_ARG, "X, Xh, yh must be non-null and nh >= 1");
  if (h->kind != KQR_RBF) return fail(h, KQR_INVALID_ARG, "held-out gradients are implemented for the RBF kernel");
  if (!h->has_state) return fail(h, KQR_INVALID_ARG, "solve the problem first");
  const int64_t n = h->n, p = h->p, N = n + nh;
  const double tau = h->st_tau, lam = h->st_lam, beta = h->st_beta, gamma = h->gamma;
  cudaStream_t st = h->stream;
  // Union point set [X; Xh] as a second problem (its own preconditioner is not used).
  std::vector<double> Xu((size_t)N * p), yu((size_t)N, 0.0);
  std::copy(X, X + n * p, Xu.begin());
  std::copy(Xh, Xh + nh * p, Xu.begin() + n * p);
  kqr_options uo;
  kqr_default_options(&uo);
  uo.rank0 = 2;
  uo.adaptive_rank = 0;
  uo.precond = KQR_PRECOND_NONE;
  uo.rbf_tensor_cores = h->opt.rbf_tensor_cores;
  kqr_handle* ukh = nullptr;
  kqr_status s = kqr_create(Xu.data(), yu.data(), N, p, KQR_RBF, gamma, &uo, &ukh);
  if (s != KQR_OK) {
    const std::string msg = ukh ? kqr_last_error(ukh) : "union problem";
    kqr_destroy(ukh);
    return fail(h, s, "held-out union problem: " + msg);
  }
  Handle* U = &ukh->h;
  kqr_set_stream(ukh, st);
  const int64_t ldr = U->ldn;
  const int ncol = (int)p + 1;
  // Work buffers on the training handle's allocator.
  const size_t nvec = 8;
  double* buf = (double*)dev_alloc(h, sizeof(double) * ((size_t)N * (nvec + 2 * 8) + 3 * (size_t)ncol * ldr + 16));
  if (!buf) {
    kqr_destroy(ukh);
    return fail(h, KQR_OOM, "gradient buffers");
  }
  double* b1 = buf;
  double* b2 = b1 + N;
  double* b3 = b2 + N;
  double* Kb1 = b3 + N;
  double* Kb2 = Kb1 + N;
  double* nrm = Kb2 + N;
  double* yhd = nrm + N;
  double* V = buf + (size_t)N * nvec;
  double* UU = V + (size_t)N * 8;
  double* R1 = UU + (size_t)N * 8;
  double* R2 = R1 + (size_t)ncol * ldr;
  double* R3 = R2 + (size_t)ncol * ldr;
  double* sums = R3 + (size_t)ncol * ldr;
  auto done = [&](kqr_status r) {
    cudaStreamSynchronize(st);
    dev_free(h, buf);
    kqr_destroy(ukh);
    return r;
  };
#define GK(call)                                           \
  do {                                                     \
    cudaError_t _e = (call);                               \
    if (_e != cudaSuccess) return done(cuda_fail(h, _e, #call)); \
  } while (0)
  GK(cudaMemsetAsync(b1, 0, sizeof(double) * N * 3, st));
  GK(cudaMemsetAsync(sums, 0, sizeof(double) * 16, st));
  GK(cudaMemcpyAsync(b1, h->st_alpha, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
  GK(cudaMemcpyAsync(yhd, yh, sizeof(double) * nh, cudaMemcpyHostToDevice, st));
  // f_h and (K alpha) on the training rows, FP64-class.
  GK(gram_high(U, b1, Kb1, 1, st));
  heldout_kernel<<<grid_for(nh), 256, 0, st>>>(Kb1, yhd, n, nh, beta, tau, lam, b2, sums);
  GK(cudaGetLastError());
  GK(gram_high(U, b2, Kb2, 1, st));
  // K_EE solves on the training problem: (K + gam 1 1^T + diag(L)) s = rhs with L tiny on E, huge off E.
  double* rhs1 = vec(h, V_B);
  double* rhs2 = vec(h, V_TMP);
  double* Ld = vec(h, V_L);
  double* mask = vec(h, V_S);
  double* s1 = vec(h, V_D);
  double* s2 = vec(h, V_DX);
  double* Lp = vec(h, V_LPRE);
  elbow_kernel<<<grid_for(n), 256, 0, st>>>(h->st_v, Kb2, n, tau, lam, 1e-7, 1e12, 0.0, rhs1, rhs2, Ld, mask, sums);
  GK(cudaGetLastError());
  GK(vec_copy(h, Lp, Ld, n, st));
  if (h->opt.precond == KQR_PRECOND_NYSTROM_DIAG) GK(axpy_vec(h, Lp, h->dres, 1.0, n, st));
  const double gam = 1e-12;
  h->core_valid = false;   // the adjoint solves replace the Woodbury core
  s = precond_build(h, Lp, gam, st);
  if (s != KQR_OK) return done(s);
  std::vector<double> hs(16);
  GK(cudaMemcpyAsync(hs.data(), sums, sizeof(double) * 16, cudaMemcpyDeviceToHost, st));
  GK(cudaStreamSynchronize(st));
  const double loss_v = hs[0], gsum = hs[1], nE = hs[2];
  if (nE > 0) {
    RedArgs rn;
    rn.a = rhs1;
    GK(reduce(h, RED_NORM2, rn, n, h->scal + S_RED0 + 15, st));
    GK(cudaMemcpyAsync(h->scal_host + S_RED0 + 15, h->scal + S_RED0 + 15, sizeof(double), cudaMemcpyDeviceToHost, st));
    GK(cudaStreamSynchronize(st));
    const double nb1 = std::sqrt(h->scal_host[S_RED0 + 15]);
    s = adjoint_cg(h, Ld, Lp, gam, rhs1, s1, std::fmax(1e-300, 1e-11 * nb1), 3000, sums + 12, st);
    if (s != KQR_OK) return done(s);
    s = adjoint_cg(h, Ld, Lp, gam, rhs2, s2, 1e-11 * std::sqrt(nE), 3000, sums + 12, st);
    if (s != KQR_OK) return done(s);
    masked_sums_kernel<<<grid_for(n), 256, 0, st>>>(s1, s2, mask, n, sums + 4);
    GK(cudaGetLastError());
    GK(cudaMemcpyAsync(hs.data(), sums, sizeof(double) * 16, cudaMemcpyDeviceToHost, st));
    GK(cudaStreamSynchronize(st));
    // u = s1 - c s2 with 1^T u = sum_h g_h
    const double c = (hs[4] - gsum) / hs[5];
    adjoint_kernel<<<grid_for(N), 256, 0, st>>>(s1, s2, mask, n, N, c, b3);
    GK(cudaGetLastError());
  }
  // Multi-RHS Gram products over [X; Xh]: R1 = K[|x|^2 b1, x_c b1], R2 = K[b2, x_c b2], R3 = K[b3, x_c b3].
  sqnorm_kernel<<<grid_for(N), 256, 0, st>>>(U->xc64, U->ldn, (int)p, N, nrm);
  GK(cudaGetLastError());
  const double* bases[3] = {b1, b2, b3};
  double* outs[3] = {R1, R2, R3};
  for (int set = 0; set < 3; ++set) {
    for (int col0 = 0; col0 < ncol; col0 += 8) {
      const int nc = ncol - col0 < 8 ? ncol - col0 : 8;
      cols_kernel<<<grid_for(N * nc), 256, 0, st>>>(bases[set], U->xc64, U->ldn, nrm, N, col0, nc, set == 0, V);
      GK(cudaGetLastError());
      GK(gram_high(U, V, UU, nc, st));
      scatter_cols_kernel<<<grid_for(N * nc), 256, 0, st>>>(UU, N, col0, nc, ldr, outs[set]);
      GK(cudaGetLastError());
    }
  }
  scalar_grad_kernel<<<grid_for(N), 256, 0, st>>>(Kb1, R1, ldr, U->xc64, U->ldn, nrm, (int)p, b2, b3, n, N, sums + 8);
  GK(cudaGetLastError());
  if (dX) {
    double* dXbuf = (double*)dev_alloc(h, sizeof(double) * (size_t)n * p);
    if (!dXbuf) return done(fail(h, KQR_OOM, "dX buffer"));
    dx_kernel<<<grid_for(n * p), 256, 0, st>>>(h->st_alpha, b3, Kb1, R1, R2, R3, ldr, U->xc64, U->ldn, (int)p, n,
                                               2.0 * gamma / lam, dXbuf);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(dX, dXbuf, sizeof(double) * n * p, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    dev_free(h, dXbuf);
    if (e != cudaSuccess) return done(cuda_fail(h, e, "dX"));
  }
  GK(cudaMemcpyAsync(hs.data(), sums, sizeof(double) * 16, cudaMemcpyDeviceToHost, st));
  GK(cudaStreamSynchronize(st));
  if (loss) *loss = loss_v;
  if (d_loglambda) *d_loglambda = hs[8] / lam;
  if (d_loggamma) *d_loggamma = hs[9] * gamma / lam;
  return done(KQR_OK);
#undef GK
}
