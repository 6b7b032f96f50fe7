// O(n) kernels of the solver: the projection onto B = [tau - 1, tau]^n with
// its 0/1 Clarke-Jacobian element and the gradient of phi_k (Sec. 2.2,
// eq. (2.3)), the diagonal L of eq. (3.1), ADMM / ALM multiplier updates
// (Alg. 1, Alg. 2), CG vector updates, and the reductions of the Sec. 4 KKT
// residuals and of the line search of Alg. 3.  All FP64.
//
// Reductions are deterministic: each block writes its partial sums, and the
// last block to finish adds the partials in block order.
#include "kqr_internal.h"
#include "ptx.cuh"

namespace kqr {

constexpr int kRedBlocks = 304;  // partial-sum slots per reduction

__device__ __forceinline__ double clampd(double x, double lo, double hi) { return fmin(fmax(x, lo), hi); }

template <int NS, typename F>
__global__ void __launch_bounds__(256) reduce_kernel(F f, int64_t n, double* __restrict__ part,
                                                     unsigned int* __restrict__ counter, double* __restrict__ out) {
  double acc[NS];
#pragma unroll
  for (int s = 0; s < NS; ++s) acc[s] = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    f(i, acc);
  __shared__ double ws[8][NS];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    double v = acc[s];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) ws[warp][s] = v;
  }
  __syncthreads();
  if (threadIdx.x < NS) {
    double v = 0.0;
    for (int w = 0; w < 8; ++w) v += ws[w][threadIdx.x];
    part[blockIdx.x * NS + threadIdx.x] = v;
  }
  __threadfence();
  __shared__ bool last;
  if (threadIdx.x == 0) last = (atomicAdd(counter, 1u) == gridDim.x - 1);
  __syncthreads();
  if (last) {
    __threadfence();
    if (threadIdx.x < NS) {
      double v = 0.0;
      for (int b = 0; b < (int)gridDim.x; ++b) v += part[b * NS + threadIdx.x];
      out[threadIdx.x] = v;
    }
    if (threadIdx.x == 0) *counter = 0u;
  }
}

template <int NS, typename F>
static cudaError_t run_reduce(Handle* h, F f, int64_t n, double* out, cudaStream_t st) {
  int blocks = grid_for(n, 256, kRedBlocks);
  reduce_kernel<NS, F><<<blocks, 256, 0, st>>>(f, n, h->red_part, h->red_counter, out);
  h->launches++;
  return cudaGetLastError();
}

struct FDot { const double *a, *b; __device__ void operator()(int64_t i, double* acc) const { acc[0] += a[i] * b[i]; } };
struct FSum { const double* a; __device__ void operator()(int64_t i, double* acc) const { acc[0] += a[i]; } };
struct FNorm2 { const double* a; __device__ void operator()(int64_t i, double* acc) const { acc[0] += a[i] * a[i]; } };

// Sec. 4: eta_p, eta_d, eta_c, objectives.
struct FKkt {
  const double *alpha, *v, *z, *y, *Ka;
  double beta, tau, lam;
  __device__ void operator()(int64_t i, double* acc) const {
    const double a = alpha[i], vi = v[i], zi = z[i], yi = y[i], ka = Ka[i];
    const double t = zi - yi + beta + ka / lam;
    acc[0] += t * t;
    acc[1] += a;
    acc[2] += (a - vi) * (a - vi);
    acc[3] += a * a;
    const double pc = vi - clampd(zi + vi, tau - 1.0, tau);
    acc[4] += pc * pc;
    acc[5] += vi * vi;
    acc[6] += yi * yi;
    acc[7] += a * ka;
    acc[8] += yi * a;
    acc[9] += zi > 0.0 ? tau * zi : -(1.0 - tau) * zi;
  }
};

// Inner products used by the line search of Alg. 3.
struct FLsPre {
  const double *Ka, *d, *Kd, *y, *g, *alpha;
  __device__ void operator()(int64_t i, double* acc) const {
    const double di = d[i];
    acc[0] += Ka[i] * di;
    acc[1] += di * Kd[i];
    acc[2] += y[i] * di;
    acc[3] += di;
    acc[4] += g[i] * di;
    acc[5] += alpha[i];
  }
};

// sum_i dist^2(w_i + c d_i) - dist^2(w_i), dist(u) = u - Pi_[tau-1,tau](u), w = alpha + z / sigma.
struct FMoreauDiff {
  const double *alpha, *z, *d;
  double sigma, tau, c;
  __device__ void operator()(int64_t i, double* acc) const {
    const double w = alpha[i] + z[i] / sigma;
    const double w1 = w + c * d[i];
    const double e0 = w - clampd(w, tau - 1.0, tau);
    const double e1 = w1 - clampd(w1, tau - 1.0, tau);
    acc[0] += e1 * e1 - e0 * e0;
  }
};

cudaError_t reduce(Handle* h, RedKind kind, const RedArgs& a, int64_t n, double* out, cudaStream_t st) {
  switch (kind) {
    case RED_DOT: return run_reduce<1>(h, FDot{a.a, a.b}, n, out, st);
    case RED_SUM: return run_reduce<1>(h, FSum{a.a}, n, out, st);
    case RED_NORM2: return run_reduce<1>(h, FNorm2{a.a}, n, out, st);
    case RED_KKT: return run_reduce<10>(h, FKkt{a.a, a.b, a.c, a.d, a.e, a.s0, a.s1, a.s2}, n, out, st);
    case RED_MOREAU_DIFF: return run_reduce<1>(h, FMoreauDiff{a.a, a.b, a.c, a.s0, a.s1, a.s2}, n, out, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t reduce_ls_pre(Handle* h, const double* Ka, const double* d, const double* Kd, const double* y,
                          const double* g, const double* alpha, int64_t n, double* out, cudaStream_t st) {
  return run_reduce<6>(h, FLsPre{Ka, d, Kd, y, g, alpha}, n, out, st);
}

// ---- element-wise kernels -----------------------------------------------------
#define GRID_LOOP(i, n) \
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (n); i += (int64_t)gridDim.x * blockDim.x)

__global__ void fill_kernel(double* x, double v, int64_t n) { GRID_LOOP(i, n) x[i] = v; }
__global__ void copy_kernel(double* d, const double* s, int64_t n) { GRID_LOOP(i, n) d[i] = s[i]; }
__global__ void scale_kernel(double* o, const double* x, double s, int64_t n) { GRID_LOOP(i, n) o[i] = s * x[i]; }
__global__ void axpy_kernel(double* y, const double* x, double a, int64_t n) { GRID_LOOP(i, n) y[i] += a * x[i]; }
__global__ void fill_L_kernel(double* L, double base, const double* dres, int64_t n) {
  GRID_LOOP(i, n) L[i] = base + (dres ? dres[i] : 0.0);
}

// CG step: x += a p, Kx += a Kp, r -= a Ap, and ||r||^2.
struct FCgUpdate {
  double *x, *Kx, *r;
  const double *p, *Kp, *Ap, *a_dev;
  __device__ void operator()(int64_t i, double* acc) const {
    const double a = *a_dev;
    x[i] += a * p[i];
    if (Kx) Kx[i] += a * Kp[i];
    const double ri = r[i] - a * Ap[i];
    r[i] = ri;
    acc[0] += ri * ri;
  }
};

// p = z + beta p, unless the device-resident CG status (stop_dev, nullable) says it
// stopped; and ||p||^2 of the resulting p.
struct FCgDir {
  double* p;
  const double *z, *beta_dev, *stop_dev;
  __device__ void operator()(int64_t i, double* acc) const {
    double pi = p[i];
    if (!(stop_dev && *stop_dev != 0.0)) {
      pi = z[i] + (*beta_dev) * pi;
      p[i] = pi;
    }
    acc[0] += pi * pi;
  }
};

__global__ void op_residual_kernel(double* r, const double* b, const double* x, const double* Kx, double gam,
                                   const double* sum_x, const double* L, int64_t n) {
  const double sx = *sum_x;
  GRID_LOOP(i, n) r[i] = b[i] - (Kx[i] + gam * sx + L[i] * x[i]);
}

// Alg. 1: b_k = lambda (y - beta 1 - z + sigma v).
__global__ void admm_rhs_kernel(double* b, const double* y, double beta, const double* z, const double* v,
                                double sigma, double lam, int64_t n) {
  GRID_LOOP(i, n) b[i] = lam * (y[i] - beta - z[i] + sigma * v[i]);
}

// v = Pi_B(alpha + z / sigma); z += step (alpha - v)  (Alg. 1 with step gamma sigma, Alg. 2 with step sigma).
__global__ void mult_update_kernel(const double* alpha, double* v, double* z, double sigma, double tau, double step,
                                   int64_t n) {
  GRID_LOOP(i, n) {
    const double a = alpha[i];
    const double vi = clampd(a + z[i] / sigma, tau - 1.0, tau);
    v[i] = vi;
    z[i] += step * (a - vi);
  }
}

// Eq. (2.3) and eq. (3.1): w, v = Pi_B(w), S, grad, L (and L + residual diagonal), ||grad||^2.
struct FBoxGrad {
  const double *alpha, *z, *Ka, *y, *dres;
  double beta, sigma, tau, lam, eps, sum_alpha;
  double *v, *S, *grad, *L, *Lpre;
  __device__ void operator()(int64_t i, double* acc) const {
    const double w = alpha[i] + z[i] / sigma;
    const double vi = clampd(w, tau - 1.0, tau);
    const double si = (w > tau - 1.0 && w < tau) ? 1.0 : 0.0;
    const double g = Ka[i] / lam - y[i] + beta + sigma * sum_alpha + sigma * (w - vi);
    if (v) v[i] = vi;
    if (S) S[i] = si;
    if (grad) grad[i] = g;
    const double li = lam * sigma * (1.0 - si) + lam * eps;
    if (L) L[i] = li;
    if (Lpre) Lpre[i] = li + (dres ? dres[i] : 0.0);
    acc[0] += g * g;
  }
};

static cudaError_t post(Handle* h) {
  h->launches++;
  return cudaGetLastError();
}

cudaError_t vec_fill(Handle* h, double* x, double val, int64_t n, cudaStream_t st) {
  fill_kernel<<<grid_for(n), 256, 0, st>>>(x, val, n);
  return post(h);
}
cudaError_t vec_copy(Handle* h, double* dst, const double* src, int64_t n, cudaStream_t st) {
  copy_kernel<<<grid_for(n), 256, 0, st>>>(dst, src, n);
  return post(h);
}
cudaError_t scale_vec(Handle* h, double* out, const double* x, double s, int64_t n, cudaStream_t st) {
  scale_kernel<<<grid_for(n), 256, 0, st>>>(out, x, s, n);
  return post(h);
}
cudaError_t axpy_vec(Handle* h, double* y, const double* x, double a, int64_t n, cudaStream_t st) {
  axpy_kernel<<<grid_for(n), 256, 0, st>>>(y, x, a, n);
  return post(h);
}
cudaError_t fill_L(Handle* h, double* L, double base, const double* dres, int64_t n, cudaStream_t st) {
  fill_L_kernel<<<grid_for(n), 256, 0, st>>>(L, base, dres, n);
  return post(h);
}
cudaError_t cg_update(Handle* h, double* x, double* Kx, double* r, const double* p, const double* Kp,
                      const double* Ap, const double* a_dev, int64_t n, double* rr_out, cudaStream_t st) {
  return run_reduce<1>(h, FCgUpdate{x, Kx, r, p, Kp, Ap, a_dev}, n, rr_out, st);
}
cudaError_t cg_direction(Handle* h, double* p, const double* z, const double* beta_dev, const double* stop_dev,
                         int64_t n, double* pp_out, cudaStream_t st) {
  return run_reduce<1>(h, FCgDir{p, z, beta_dev, stop_dev}, n, pp_out, st);
}
cudaError_t op_residual(Handle* h, double* r, const double* b, const double* x, const double* Kx, double gam,
                        const double* sum_x, const double* L, int64_t n, cudaStream_t st) {
  op_residual_kernel<<<grid_for(n), 256, 0, st>>>(r, b, x, Kx, gam, sum_x, L, n);
  return post(h);
}
cudaError_t admm_rhs(Handle* h, double* b, const double* y, double beta, const double* z, const double* v,
                     double sigma, double lam, int64_t n, cudaStream_t st) {
  admm_rhs_kernel<<<grid_for(n), 256, 0, st>>>(b, y, beta, z, v, sigma, lam, n);
  return post(h);
}
cudaError_t admm_update(Handle* h, const double* alpha, double* v, double* z, double sigma, double tau, double step,
                        int64_t n, cudaStream_t st) {
  mult_update_kernel<<<grid_for(n), 256, 0, st>>>(alpha, v, z, sigma, tau, step, n);
  return post(h);
}
cudaError_t alm_update(Handle* h, const double* alpha, double* v, double* z, double sigma, double tau, int64_t n,
                       cudaStream_t st) {
  mult_update_kernel<<<grid_for(n), 256, 0, st>>>(alpha, v, z, sigma, tau, sigma, n);
  return post(h);
}
cudaError_t box_grad(Handle* h, const double* alpha, const double* z, const double* Kalpha, const double* y,
                     double beta, double sigma, double tau, double lam, double eps, const double* dres, double* v,
                     double* S, double* grad, double* Ldiag, double* Lpre, int64_t n, cudaStream_t st) {
  // sum_i alpha_i first (deterministic), then the fused element-wise pass.
  cudaError_t e = run_reduce<1>(h, FSum{alpha}, n, h->scal + S_RED0 + 12, st);
  if (e != cudaSuccess) return e;
  e = cudaMemcpyAsync(h->scal_host + S_RED0 + 12, h->scal + S_RED0 + 12, sizeof(double), cudaMemcpyDeviceToHost, st);
  if (e != cudaSuccess) return e;
  if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return e;
  const double sa = h->scal_host[S_RED0 + 12];
  return run_reduce<1>(h, FBoxGrad{alpha, z, Kalpha, y, dres, beta, sigma, tau, lam, eps, sa, v, S, grad, Ldiag, Lpre},
                       n, h->scal + S_RED0 + 13, st);
}

// One CTA waits, bounded by max_polls, on an mbarrier that nothing arrives on:
// the timeout path of mbar_wait_bounded, which records kErrWaitTimeout in the
// error word.  No copy or MMA is in flight, so the early exit leaves nothing
// behind.
__global__ void wait_probe_kernel(int* err, uint32_t max_polls) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    fence_mbar_init();
    (void)mbar_wait_bounded(&bar, 0u, err, max_polls);
  }
}

cudaError_t launch_wait_probe(Handle* h, uint32_t max_polls, cudaStream_t st) {
  wait_probe_kernel<<<1, 32, 0, st>>>(h->err_flag, max_polls);
  return post(h);
}

}  // namespace kqr
