// Low-rank preconditioner of Sec. 3.
//
// Set-up (once per (X, kernel, gamma)): F = RPCholesky(K, r0), K ~= F F^T,
// pivots drawn with probability proportional to the residual diagonal; then
// the rank heuristic of Sec. 3 (smallest r with xi lambda_1 >= lambda_r over
// the eigenvalues of F0^T F0) and truncation to r columns (re-running
// RPCholesky with the same pivot stream reproduces exactly the first r
// columns).  lambda_1 comes from power iteration and the count of eigenvalues
// above xi lambda_1 from the inertia of an LDL^T factorisation of
// F0^T F0 - xi lambda_1 I (Sylvester's law), so no full eigensolver is needed.
//
// Per linear system: Lemma 1,
//   P^{-1} = L^{-1} - L^{-1} U (C + U^T L^{-1} U)^{-1} U^T L^{-1},
//   U = [F 1], C = diag(I_r, 1/gam),
// with the (r+1)^2 core built in FP64, Cholesky-factorised and inverted on the
// device; each apply is two skinny FP64 products with the FP32 factor.
#include <cmath>
#include <cstring>
#include <vector>

#include "kqr_internal.h"

namespace kqr {

#define GRID_LOOP(i, n) \
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (n); i += (int64_t)gridDim.x * blockDim.x)

// ---- weighted Gram of the columns of U = [F, 1] (optional ones column) -----------
// G[a][b] += sum_{i in chunk} U_ai U_bi w_i for a 32 x 32 tile pair (ta <= tb).
constexpr int kCT = 32;    // core tile
constexpr int kCR = 32;    // rows per shared-memory step
constexpr int kChunk = 4096;

template <typename T>
__global__ void __launch_bounds__(256) core_gram_kernel(const T* __restrict__ F, int rr, int ncols, int64_t n,
                                                        const double* __restrict__ w, double* __restrict__ G,
                                                        int ntile) {
  // blockIdx.x enumerates tile pairs (ta <= tb), blockIdx.y row chunks.
  int pair = blockIdx.x, ta = 0;
  while (pair >= ntile - ta) { pair -= ntile - ta; ++ta; }
  const int tb = ta + pair;
  __shared__ double Ua[kCR][kCT + 1];
  __shared__ double Ub[kCR][kCT + 1];
  const int tid = threadIdx.x;
  const int la = tid / 8;          // 0..31: row of the 32x32 output tile
  const int lb0 = (tid % 8) * 4;   // 4 consecutive columns
  double acc[4] = {0, 0, 0, 0};
  const int64_t i0 = (int64_t)blockIdx.y * kChunk;
  const int64_t i1 = min(n, i0 + kChunk);
  for (int64_t ib = i0; ib < i1; ib += kCR) {
    __syncthreads();
    for (int e = tid; e < kCR * kCT; e += 256) {
      const int rrow = e / kCT, c = e % kCT;
      const int64_t i = ib + rrow;
      const int ca = ta * kCT + c, cb = tb * kCT + c;
      double ua = 0.0, ub = 0.0;
      if (i < i1) {
        const double wi = w ? w[i] : 1.0;
        ua = ca < rr ? (double)F[(size_t)ca * n + i] : (ca < ncols ? 1.0 : 0.0);
        ub = cb < rr ? (double)F[(size_t)cb * n + i] : (cb < ncols ? 1.0 : 0.0);
        ua *= wi;
      }
      Ua[rrow][c] = ua;
      Ub[rrow][c] = ub;
    }
    __syncthreads();
#pragma unroll 8
    for (int k = 0; k < kCR; ++k) {
      const double a = Ua[k][la];
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[q] = fma(a, Ub[k][lb0 + q], acc[q]);
    }
  }
  const int a = ta * kCT + la;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int b = tb * kCT + lb0 + q;
    if (a < ncols && b < ncols) {
      atomicAdd(&G[(size_t)a * ncols + b], acc[q]);
      if (ta != tb) atomicAdd(&G[(size_t)b * ncols + a], acc[q]);
    }
  }
}

template <typename T>
static cudaError_t core_gram(Handle* h, const T* F, int rr, bool ones, const double* w, double* G, cudaStream_t st) {
  const int ncols = rr + (ones ? 1 : 0);
  cudaError_t e = cudaMemsetAsync(G, 0, sizeof(double) * ncols * ncols, st);
  if (e != cudaSuccess) return e;
  const int ntile = (ncols + kCT - 1) / kCT;
  const int pairs = ntile * (ntile + 1) / 2;
  const int chunks = (int)((h->n + kChunk - 1) / kChunk);
  core_gram_kernel<T><<<dim3(pairs, chunks), 256, 0, st>>>(F, rr, ncols, h->n, w, G, ntile);
  h->launches++;
  return cudaGetLastError();
}

__global__ void add_diag_kernel(double* G, int N, double v, double last) {
  GRID_LOOP(i, N) G[i * N + i] += (i == N - 1) ? last : v;
}

// In-place lower Cholesky of the N x N row-major matrix (single CTA).
// info[0] = 0 on success, j + 1 if pivot j was not positive.
__global__ void __launch_bounds__(1024) cholesky_kernel(double* G, int N, int* info) {
  __shared__ double piv;
  __shared__ int bad;
  if (threadIdx.x == 0) bad = 0;
  __syncthreads();
  for (int j = 0; j < N; ++j) {
    if (threadIdx.x == 0) {
      const double d = G[(size_t)j * N + j];
      if (!(d > 0.0)) {
        bad = j + 1;
        piv = 1.0;
      } else {
        piv = sqrt(d);
      }
      G[(size_t)j * N + j] = piv;
    }
    __syncthreads();
    if (bad) break;
    const double inv = 1.0 / piv;
    for (int i = j + 1 + threadIdx.x; i < N; i += blockDim.x) G[(size_t)i * N + j] *= inv;
    __syncthreads();
    // trailing update of the lower triangle, one warp per row
    const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int i = j + 1 + (int)(threadIdx.x >> 5); i < N; i += nw) {
      const double gij = G[(size_t)i * N + j];
      for (int k = j + 1 + lane; k <= i; k += 32) G[(size_t)i * N + k] -= gij * G[(size_t)k * N + j];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) *info = bad;
}

// W = L^{-1} (lower) from the Cholesky factor stored in the lower triangle of G;
// one thread per column of W (single CTA).  W is written to Winv.
__global__ void __launch_bounds__(1024) tri_inverse_kernel(const double* G, int N, double* W) {
  for (int c = threadIdx.x; c < N; c += blockDim.x) {
    for (int i = 0; i < c; ++i) W[(size_t)i * N + c] = 0.0;
    for (int i = c; i < N; ++i) {
      double s = (i == c) ? 1.0 : 0.0;
      for (int k = c; k < i; ++k) s -= G[(size_t)i * N + k] * W[(size_t)k * N + c];
      W[(size_t)i * N + c] = s / G[(size_t)i * N + i];
    }
  }
}

// Ginv = W^T W (symmetric), one output entry per thread.
__global__ void wtw_kernel(const double* W, int N, double* Ginv) {
  GRID_LOOP(e, (int64_t)N * N) {
    const int a = (int)(e / N), b = (int)(e % N);
    const int i0 = a > b ? a : b;
    double s = 0.0;
    for (int i = i0; i < N; ++i) s += W[(size_t)i * N + a] * W[(size_t)i * N + b];
    Ginv[e] = s;
  }
}

__global__ void recip_kernel(double* out, const double* L, int64_t n) { GRID_LOOP(i, n) out[i] = 1.0 / L[i]; }

// t[a] += sum_i U_ai (Linv_i r_i) over a chunk of 2048 rows and 8 columns of U = [F 1].
__global__ void __launch_bounds__(256) ut_kernel(const float* __restrict__ F, int r, int64_t n,
                                                 const double* __restrict__ Linv, const double* __restrict__ rv,
                                                 double* __restrict__ t) {
  const int c0 = blockIdx.y * 8;
  double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  const int64_t base = (int64_t)blockIdx.x * 2048;
  for (int q = 0; q < 8; ++q) {
    const int64_t i = base + q * 256 + threadIdx.x;
    if (i >= n) break;
    const double wi = Linv[i] * rv[i];
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      const int col = c0 + c;
      if (col < r) acc[c] = fma((double)F[(size_t)col * n + i], wi, acc[c]);
      else if (col == r) acc[c] += wi;
    }
  }
  __shared__ double ws[8][8];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    double v = acc[c];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) ws[warp][c] = v;
  }
  __syncthreads();
  if (threadIdx.x < 8 && c0 + (int)threadIdx.x <= r) {
    double v = 0.0;
    for (int w = 0; w < 8; ++w) v += ws[w][threadIdx.x];
    atomicAdd(&t[c0 + threadIdx.x], v);
  }
}

// t2 = Ginv t (N x N times N), one block per output row.
__global__ void gemv_core_kernel(const double* __restrict__ Ginv, const double* __restrict__ t, int N,
                                 double* __restrict__ t2) {
  const int a = blockIdx.x;
  double s = 0.0;
  for (int b = threadIdx.x; b < N; b += blockDim.x) s += Ginv[(size_t)a * N + b] * t[b];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  __shared__ double ws[8];
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double v = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += ws[w];
    t2[a] = v;
  }
}

// out_i = Linv_i (r_i - (F t2_F)_i - t2_r); rz += r_i out_i.
__global__ void __launch_bounds__(256) woodbury_out_kernel(const float* __restrict__ F, int r, int64_t n,
                                                           const double* __restrict__ Linv,
                                                           const double* __restrict__ rv,
                                                           const double* __restrict__ t2, double* __restrict__ out,
                                                           double* __restrict__ rz) {
  extern __shared__ double ts[];
  for (int c = threadIdx.x; c <= r; c += blockDim.x) ts[c] = t2[c];
  __syncthreads();
  double dot = 0.0;
  GRID_LOOP(i, n) {
    double s = ts[r];
    for (int c = 0; c < r; ++c) s = fma((double)F[(size_t)c * n + i], ts[c], s);
    const double o = Linv[i] * (rv[i] - s);
    out[i] = o;
    dot += rv[i] * o;
  }
  if (rz) {
    for (int o = 16; o > 0; o >>= 1) dot += __shfl_xor_sync(0xffffffffu, dot, o);
    __shared__ double ws[8];
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = dot;
    __syncthreads();
    if (threadIdx.x == 0) {
      double v = 0.0;
      for (int w = 0; w < 8; ++w) v += ws[w];
      atomicAdd(rz, v);
    }
  }
}

__global__ void ident_dot_kernel(const double* __restrict__ rv, double* __restrict__ out, int64_t n,
                                 double* __restrict__ rz) {
  double dot = 0.0;
  GRID_LOOP(i, n) {
    out[i] = rv[i];
    dot += rv[i] * rv[i];
  }
  if (rz) {
    for (int o = 16; o > 0; o >>= 1) dot += __shfl_xor_sync(0xffffffffu, dot, o);
    __shared__ double ws[8];
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = dot;
    __syncthreads();
    if (threadIdx.x == 0) {
      double v = 0.0;
      for (int w = 0; w < 8; ++w) v += ws[w];
      atomicAdd(rz, v);
    }
  }
}

// max_i |Lpre_i Linv_i - 1| (relative change of the diagonal since the last build)
__global__ void rel_change_kernel(const double* __restrict__ Lpre, const double* __restrict__ Linv, int64_t n,
                                  unsigned long long* __restrict__ out) {
  double m = 0.0;
  GRID_LOOP(i, n) m = fmax(m, fabs(Lpre[i] * Linv[i] - 1.0));
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, (unsigned long long)__double_as_longlong(m));  // m >= 0: bit order = value order
}

kqr_status precond_update(Handle* h, const double* Lpre, double gam, double rtol, cudaStream_t st) {
  if (h->core_valid && h->core_gam == gam && h->core_kind == h->opt.precond && h->opt.precond != KQR_PRECOND_NONE) {
    unsigned long long* slot = reinterpret_cast<unsigned long long*>(h->scal + S_COUNT - 2);
    cudaError_t e = cudaMemsetAsync(slot, 0, sizeof(unsigned long long), st);
    if (e != cudaSuccess) return cuda_fail(h, e, "core reuse check");
    rel_change_kernel<<<grid_for(h->n), 256, 0, st>>>(Lpre, h->Linv, h->n, slot);
    h->launches++;
    unsigned long long bits = 0;
    if ((e = cudaMemcpyAsync(&bits, slot, sizeof(bits), cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
        (e = cudaStreamSynchronize(st)) != cudaSuccess)
      return cuda_fail(h, e, "core reuse check");
    double change;
    std::memcpy(&change, &bits, sizeof(change));
    if (change <= rtol) {
      h->core_reuses++;
      return KQR_OK;
    }
  }
  return precond_build(h, Lpre, gam, st);
}

kqr_status precond_build(Handle* h, const double* Lpre, double gam, cudaStream_t st) {
  h->core_valid = false;
  h->core_gam = gam;
  h->core_kind = h->opt.precond;
  h->core_builds++;
  if (h->opt.precond == KQR_PRECOND_NONE) {
    h->core_valid = true;
    return KQR_OK;
  }
  const int N = h->r + 1;
  double* G = h->core;                       // N x N, factor / scratch
  double* W = h->core + (size_t)N * N;       // N x N, L^{-1}
  double* Ginv = W + (size_t)N * N;          // N x N
  cudaError_t e;
  recip_kernel<<<grid_for(h->n), 256, 0, st>>>(h->Linv, Lpre, h->n);
  h->launches++;
  if ((e = core_gram<float>(h, h->F32, h->r, true, h->Linv, G, st)) != cudaSuccess) return cuda_fail(h, e, "core");
  add_diag_kernel<<<grid_for(N), 256, 0, st>>>(G, N, 1.0, 1.0 / gam);
  h->launches++;
  int* info = reinterpret_cast<int*>(h->scal + S_COUNT - 1);
  cholesky_kernel<<<1, 1024, 0, st>>>(G, N, info);
  h->launches++;
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(h, e, "cholesky");
  int hinfo = 0;
  if ((e = cudaMemcpyAsync(&hinfo, info, sizeof(int), cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
      (e = cudaStreamSynchronize(st)) != cudaSuccess)
    return cuda_fail(h, e, "cholesky info");
  if (hinfo != 0) return fail(h, KQR_BREAKDOWN, "Woodbury core not positive definite at pivot " + std::to_string(hinfo - 1));
  tri_inverse_kernel<<<1, 1024, 0, st>>>(G, N, W);
  h->launches++;
  wtw_kernel<<<grid_for((int64_t)N * N), 256, 0, st>>>(W, N, Ginv);
  h->launches++;
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(h, e, "core inverse");
  h->core_valid = true;
  return KQR_OK;
}

// out = P^{-1} r with the core built by precond_build for the same Lpre; rz_out
// (device, nullable, zeroed here) receives r^T out.
cudaError_t precond_apply(Handle* h, const double* Lpre, const double* rv, double* out, double* rz_out,
                          cudaStream_t st) {
  (void)Lpre;
  cudaError_t e;
  if (rz_out && (e = cudaMemsetAsync(rz_out, 0, sizeof(double), st)) != cudaSuccess) return e;
  if (h->opt.precond == KQR_PRECOND_NONE) {
    ident_dot_kernel<<<grid_for(h->n), 256, 0, st>>>(rv, out, h->n, rz_out);
    h->launches++;
    return cudaGetLastError();
  }
  const int N = h->r + 1;
  const double* Ginv = h->core + 2 * (size_t)N * N;
  double* t = h->tvec;
  double* t2 = h->tvec + N;
  if ((e = cudaMemsetAsync(t, 0, sizeof(double) * N, st)) != cudaSuccess) return e;
  ut_kernel<<<dim3((unsigned)((h->n + 2047) / 2048), (N + 7) / 8), 256, 0, st>>>(h->F32, h->r, h->n, h->Linv, rv, t);
  h->launches++;
  gemv_core_kernel<<<N, 256, 0, st>>>(Ginv, t, N, t2);
  h->launches++;
  woodbury_out_kernel<<<grid_for(h->n), 256, (size_t)N * sizeof(double), st>>>(h->F32, h->r, h->n, h->Linv, rv, t2,
                                                                                out, rz_out);
  h->launches++;
  return cudaGetLastError();
}

// ---- RPCholesky set-up --------------------------------------------------------------
constexpr int kPivChunks = 256;

__global__ void chunk_sum_kernel(const double* __restrict__ d, int64_t n, int64_t chunk, double* __restrict__ out) {
  const int64_t i0 = (int64_t)blockIdx.x * chunk;
  const int64_t i1 = min(n, i0 + chunk);
  double s = 0.0;
  for (int64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) s += d[i];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  __shared__ double ws[8];
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double v = 0.0;
    for (int w = 0; w < 8; ++w) v += ws[w];
    out[blockIdx.x] = v;
  }
}

// ---- fused RPCholesky steps ---------------------------------------------------------
// One launch per pivot.  CTA b owns rows [b * kRpcChunk, (b + 1) * kRpcChunk); step t
// forms column t of F for the pivot s = piv[t] chosen by the previous launch, updates the
// residual diagonal and writes its chunk's sum of the new diagonal; the last CTA to finish
// (a ticket counter, no waiting) draws the next pivot from the chunk sums.  state[0] is
// the stop flag, state[1] the number of columns produced, state[2] the ticket counter.
constexpr int kRpcChunk = 512;
constexpr int kRpcThreads = 256;

// Residual column entry g_i = k(x_i, x_s) - sum_{c<t} F[c][i] F[c][s]; every CTA calls it
// for row s too, so the pivot's g_s is bit-identical to the one its own row computes.
__device__ __forceinline__ double rpc_entry(const double* __restrict__ xc, int64_t ldn, int p, double gamma, int lap,
                                            const double* __restrict__ F, int64_t n, int t, int64_t i,
                                            const double* xs, const double* fs) {
  double dist = 0.0;
  for (int k = 0; k < p; ++k) {
    const double v = xc[(size_t)k * ldn + i] - xs[k];
    dist = lap ? dist + fabs(v) : fma(v, v, dist);
  }
  double acc = exp(-gamma * dist);
  for (int c = 0; c < t; ++c) acc -= F[(size_t)c * n + i] * fs[c];
  return acc;
}

// Pivot draw by the last CTA: the smallest s with running sum of d > u * sum(d), the
// sums taken chunk by chunk in a fixed order.  Thread 0 only.
__device__ void rpc_pick(const double* d, const double* csum, int64_t n, int nchunks, double u, long long* piv_out,
                         int* state) {
  double total = 0.0;
  for (int c = 0; c < nchunks; ++c) total += __ldcg(csum + c);
  if (!(total > 0.0)) {
    *piv_out = -1;
    state[0] = 1;
    return;
  }
  const double target = u * total;
  double run = 0.0;
  int c = 0;
  for (; c < nchunks - 1; ++c) {
    const double cs = __ldcg(csum + c);
    if (run + cs > target) break;
    run += cs;
  }
  int64_t s = (int64_t)c * kRpcChunk;
  const int64_t end = min(n, s + kRpcChunk);
  int64_t found = -1;
  for (; s < end; ++s) {
    run += __ldcg(d + s);
    if (run > target) {
      found = s;
      break;
    }
  }
  if (found < 0) {  // rounding left the target past the last positive entry: take the last positive one
    for (int64_t q = n - 1; q >= 0; --q)
      if (__ldcg(d + q) > 0.0) {
        found = q;
        break;
      }
  }
  *piv_out = found;
}

__device__ __forceinline__ void rpc_chunk_sum_and_ticket(double local, double* csum, const double* d, int64_t n,
                                                         int nchunks, const double* u, int t, int r0,
                                                         long long* piv, int* state) {
  __shared__ double ws[kRpcThreads / 32];
  __shared__ int last;
  for (int o = 16; o > 0; o >>= 1) local += __shfl_xor_sync(0xffffffffu, local, o);
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = local;
  __syncthreads();
  if (threadIdx.x == 0) {
    double v = 0.0;
    for (int w = 0; w < kRpcThreads / 32; ++w) v += ws[w];
    csum[blockIdx.x] = v;
    __threadfence();
    last = atomicAdd(state + 2, 1) == nchunks - 1;
  }
  __syncthreads();
  if (last && threadIdx.x == 0) {
    __threadfence();
    state[2] = 0;
    state[1] = t + 1;
    if (t + 1 < r0) rpc_pick(d, csum, n, nchunks, u[t + 1], piv + t + 1, state);
  }
}

// d = diag(K) = 1 and the draw of the first pivot.
__global__ void rpc_init_kernel(double* __restrict__ d, int64_t n, int nchunks, double* __restrict__ csum,
                                const double* __restrict__ u, int r0, long long* __restrict__ piv,
                                int* __restrict__ state) {
  const int64_t i0 = (int64_t)blockIdx.x * kRpcChunk;
  const int64_t i1 = min(n, i0 + kRpcChunk);
  double local = 0.0;
  for (int64_t i = i0 + threadIdx.x; i < i1; i += kRpcThreads) {
    d[i] = 1.0;   // k(x, x) = 1 for the RBF and Laplacian kernels
    local += 1.0;
  }
  rpc_chunk_sum_and_ticket(local, csum, d, n, nchunks, u, -1, r0, piv, state);
}

__global__ void __launch_bounds__(kRpcThreads) rpc_step_kernel(const double* __restrict__ xc, int64_t ldn, int p,
                                                              double gamma, int lap, double* __restrict__ F,
                                                              double* __restrict__ d, int64_t n, int t, int r0,
                                                              int nchunks, double* __restrict__ csum,
                                                              const double* __restrict__ u,
                                                              long long* __restrict__ piv, int* __restrict__ state) {
  if (*(volatile int*)state) return;   // an earlier step stopped the factorization
  const long long s = piv[t];
  extern __shared__ double sm[];
  double* fs = sm;            // F[c][s], c < t
  double* xs = sm + t;        // x_s
  __shared__ double gs_sh;
  for (int c = threadIdx.x; c < t; c += kRpcThreads) fs[c] = F[(size_t)c * n + s];
  for (int k = threadIdx.x; k < p; k += kRpcThreads) xs[k] = xc[(size_t)k * ldn + s];
  __syncthreads();
  if (threadIdx.x == 0) gs_sh = rpc_entry(xc, ldn, p, gamma, lap, F, n, t, s, xs, fs);
  __syncthreads();
  const double gs = gs_sh;
  if (!(gs > 0.0)) {     // the residual at the pivot vanished: stop with t columns
    if (blockIdx.x == 0 && threadIdx.x == 0) state[0] = 1;
    return;
  }
  const double inv = 1.0 / sqrt(gs);
  const int64_t i0 = (int64_t)blockIdx.x * kRpcChunk;
  const int64_t i1 = min(n, i0 + kRpcChunk);
  double local = 0.0;
  double* Ft = F + (size_t)t * n;
  for (int64_t i = i0 + threadIdx.x; i < i1; i += kRpcThreads) {
    const double f = rpc_entry(xc, ldn, p, gamma, lap, F, n, t, i, xs, fs) * inv;
    Ft[i] = f;
    const double di = fmax(d[i] - f * f, 0.0);
    d[i] = di;
    local += di;
  }
  rpc_chunk_sum_and_ticket(local, csum, d, n, nchunks, u, t, r0, piv, state);
}

__global__ void to_float_kernel(const double* __restrict__ src, float* __restrict__ dst, int64_t cnt) {
  GRID_LOOP(i, cnt) dst[i] = (float)src[i];
}

__global__ void dres_kernel(const float* __restrict__ F, int r, int64_t n, double* __restrict__ dres) {
  GRID_LOOP(i, n) {
    double s = 0.0;
    for (int c = 0; c < r; ++c) {
      const double f = (double)F[(size_t)c * n + i];
      s += f * f;
    }
    dres[i] = fmax(1.0 - s, 0.0);   // k(x, x) = 1 for the RBF and Laplacian kernels
  }
}

__global__ void floor_kernel(double* __restrict__ d, int64_t n, double nu) { GRID_LOOP(i, n) d[i] = fmax(d[i], nu); }

// lambda_1 of the SPD matrix A (N x N) by power iteration (single CTA).
__global__ void __launch_bounds__(512) power_iter_kernel(const double* __restrict__ A, int N, double* __restrict__ x,
                                                         double* __restrict__ y, int iters, double* __restrict__ lam) {
  __shared__ double red[16];
  __shared__ double cur;
  for (int i = threadIdx.x; i < N; i += blockDim.x) x[i] = 1.0 / sqrt((double)N) * (1.0 + 1e-3 * (i % 7));
  __syncthreads();
  double prev = 0.0;
  for (int it = 0; it < iters; ++it) {
    double loc = 0.0;
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
      double s = 0.0;
      for (int k = 0; k < N; ++k) s += A[(size_t)i * N + k] * x[k];
      y[i] = s;
      loc += s * s;
    }
    for (int o = 16; o > 0; o >>= 1) loc += __shfl_xor_sync(0xffffffffu, loc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = loc;
    __syncthreads();
    if (threadIdx.x == 0) {
      double v = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += red[w];
      cur = sqrt(v);
    }
    __syncthreads();
    const double nv = cur;
    for (int i = threadIdx.x; i < N; i += blockDim.x) x[i] = y[i] / nv;
    __syncthreads();
    if (fabs(nv - prev) <= 1e-15 * nv) break;
    prev = nv;
  }
  if (threadIdx.x == 0) *lam = cur;
}

// Number of negative pivots of the LDL^T factorisation (no pivoting) of A - c I,
// i.e. the number of eigenvalues of A below c (single CTA, A overwritten).
__global__ void __launch_bounds__(1024) inertia_kernel(double* A, int N, double c, int* neg) {
  __shared__ double dj;
  __shared__ int cnt;
  if (threadIdx.x == 0) cnt = 0;
  for (int i = threadIdx.x; i < N; i += blockDim.x) A[(size_t)i * N + i] -= c;
  __syncthreads();
  for (int j = 0; j < N; ++j) {
    if (threadIdx.x == 0) {
      double d = A[(size_t)j * N + j];
      if (d == 0.0) d = 1e-300;
      if (d < 0.0) ++cnt;
      dj = d;
    }
    __syncthreads();
    const double invd = 1.0 / dj;
    // trailing update A_ik -= A_ij A_kj / d_j for j < k <= i (lower), one warp per row
    const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int i = j + 1 + (int)(threadIdx.x >> 5); i < N; i += nw) {
      const double aij = A[(size_t)i * N + j] * invd;
      for (int k = j + 1 + lane; k <= i; k += 32) A[(size_t)i * N + k] -= aij * A[(size_t)k * N + j];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) *neg = cnt;
}

kqr_status rpcholesky_setup(Handle* h, const double* uniforms) {
  const int64_t n = h->n;
  int r0 = h->opt.rank0 > 0 ? h->opt.rank0 : (int)std::ceil(std::sqrt((double)n));
  if (r0 > n) r0 = (int)n;
  if (r0 > 1024) r0 = 1024;
  h->r0 = r0;
  cudaStream_t st = h->stream;
  cudaError_t e;
  const size_t fbytes = sizeof(double) * (size_t)r0 * n;
  double* F64 = (double*)dev_alloc(h, fbytes);
  double* d = (double*)dev_alloc(h, sizeof(double) * n);
  double* csum = (double*)dev_alloc(h, sizeof(double) * (kPivChunks + 8));
  int* bad = (int*)dev_alloc(h, sizeof(int) * 2);
  auto cleanup = [&]() {
    dev_free(h, F64); dev_free(h, d); dev_free(h, csum); dev_free(h, bad);
  };
  if (!F64 || !d || !csum || !bad) {
    cleanup();
    return fail(h, KQR_OOM, "RPCholesky workspace");
  }
  // Pivot uniforms: given, or a splitmix64 stream from the seed.
  std::vector<double> u(r0);
  if (uniforms) {
    for (int t = 0; t < r0; ++t) u[t] = uniforms[t];
  } else {
    uint64_t x = h->opt.seed;
    for (int t = 0; t < r0; ++t) {
      x += 0x9E3779B97F4A7C15ull;
      uint64_t z = x;
      z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
      z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
      z ^= z >> 31;
      u[t] = (double)(z >> 11) * (1.0 / 9007199254740992.0);
    }
  }
  const int64_t chunk = (n + kPivChunks - 1) / kPivChunks;
  const int nchunks = (int)((n + chunk - 1) / chunk);
  const int rchunks = (int)((n + kRpcChunk - 1) / kRpcChunk);
  double* u_dev = (double*)dev_alloc(h, sizeof(double) * (r0 + 1));
  double* rsum = (double*)dev_alloc(h, sizeof(double) * (rchunks + 1));
  long long* piv_all = (long long*)dev_alloc(h, sizeof(long long) * (r0 + 1));
  int* state = (int*)dev_alloc(h, sizeof(int) * 4);
  auto cleanup2 = [&]() { dev_free(h, u_dev); dev_free(h, rsum); dev_free(h, piv_all); dev_free(h, state); };
  if (!u_dev || !rsum || !piv_all || !state) {
    cleanup2();
    cleanup();
    return fail(h, KQR_OOM, "RPCholesky workspace");
  }
  const size_t smem = sizeof(double) * ((size_t)r0 + h->p);
  if (smem > 48 * 1024 &&
      (e = cudaFuncSetAttribute(rpc_step_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess) {
    cleanup2();
    cleanup();
    return cuda_fail(h, e, "RPCholesky shared memory (p too large)");
  }
  // All r0 steps are queued back to back; the device decides the pivots and when to stop.
  if ((e = cudaMemcpyAsync(u_dev, u.data(), sizeof(double) * r0, cudaMemcpyHostToDevice, st)) != cudaSuccess ||
      (e = cudaMemsetAsync(state, 0, sizeof(int) * 4, st)) != cudaSuccess ||
      (e = cudaMemsetAsync(piv_all, 0xff, sizeof(long long) * (r0 + 1), st)) != cudaSuccess) {
    cleanup2();
    cleanup();
    return cuda_fail(h, e, "RPCholesky start");
  }
  rpc_init_kernel<<<rchunks, kRpcThreads, 0, st>>>(d, n, rchunks, rsum, u_dev, r0, piv_all, state);
  h->launches++;
  for (int t = 0; t < r0; ++t) {
    rpc_step_kernel<<<rchunks, kRpcThreads, smem, st>>>(h->xc64, h->ldn, (int)h->p, h->gamma,
                                                        h->kind == KQR_LAPLACIAN, F64, d, n, t, r0, rchunks, rsum,
                                                        u_dev, piv_all, state);
    h->launches++;
  }
  int hstate[4] = {0, 0, 0, 0};
  std::vector<long long> hpiv(r0 + 1);
  if ((e = cudaGetLastError()) != cudaSuccess ||
      (e = cudaMemcpyAsync(hstate, state, sizeof(int) * 4, cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
      (e = cudaMemcpyAsync(hpiv.data(), piv_all, sizeof(long long) * (r0 + 1), cudaMemcpyDeviceToHost, st)) !=
          cudaSuccess ||
      (e = cudaStreamSynchronize(st)) != cudaSuccess) {
    cleanup2();
    cleanup();
    return cuda_fail(h, e, "RPCholesky steps");
  }
  cleanup2();
  h->pivots.clear();
  const int t = hstate[1];
  for (int q = 0; q < t; ++q) h->pivots.push_back(hpiv[q]);
  const int rr0 = t;  // columns actually produced
  h->r0 = rr0;
  int r = rr0;
  if (h->opt.adaptive_rank && rr0 > 1) {
    // Rank heuristic on F0^T F0 (rr0 x rr0).
    double* A = (double*)dev_alloc(h, sizeof(double) * (size_t)rr0 * rr0 + sizeof(double) * (2 * rr0 + 4));
    if (!A) {
      cleanup();
      return fail(h, KQR_OOM, "rank heuristic workspace");
    }
    double* xw = A + (size_t)rr0 * rr0;
    double* yw = xw + rr0;
    double* lam1 = yw + rr0;
    core_gram<double>(h, F64, rr0, false, nullptr, A, st);
    power_iter_kernel<<<1, 512, 0, st>>>(A, rr0, xw, yw, 2000, lam1);
    h->launches++;
    double hl1 = 0.0;
    if ((e = cudaMemcpyAsync(&hl1, lam1, sizeof(double), cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
        (e = cudaStreamSynchronize(st)) != cudaSuccess) {
      dev_free(h, A);
      cleanup();
      return cuda_fail(h, e, "power iteration");
    }
    core_gram<double>(h, F64, rr0, false, nullptr, A, st);
    inertia_kernel<<<1, 1024, 0, st>>>(A, rr0, h->opt.xi * hl1, bad + 1);
    h->launches++;
    int neg = 0;
    if ((e = cudaMemcpyAsync(&neg, bad + 1, sizeof(int), cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
        (e = cudaStreamSynchronize(st)) != cudaSuccess) {
      dev_free(h, A);
      cleanup();
      return cuda_fail(h, e, "inertia");
    }
    dev_free(h, A);
    const int above = rr0 - neg;           // eigenvalues > xi lambda_1
    r = above + 1 <= rr0 ? above + 1 : rr0;
  }
  h->r = r;
  dev_free(h, h->F32); dev_free(h, h->dres); dev_free(h, h->core); dev_free(h, h->tvec); dev_free(h, h->Linv);
  h->core_valid = false;
  h->F32 = (float*)dev_alloc(h, sizeof(float) * ((size_t)r * n + 1));
  h->dres = (double*)dev_alloc(h, sizeof(double) * n);
  const int N = r + 1;
  h->core = (double*)dev_alloc(h, sizeof(double) * 3 * (size_t)N * N);
  h->tvec = (double*)dev_alloc(h, sizeof(double) * 2 * N);
  h->Linv = (double*)dev_alloc(h, sizeof(double) * n);
  if (!h->F32 || !h->dres || !h->core || !h->tvec || !h->Linv) {
    cleanup();
    return fail(h, KQR_OOM, "preconditioner buffers");
  }
  if (r > 0) {
    to_float_kernel<<<grid_for((int64_t)r * n), 256, 0, st>>>(F64, h->F32, (int64_t)r * n);
    h->launches++;
  }
  dres_kernel<<<grid_for(n), 256, 0, st>>>(h->F32, r, n, h->dres);
  h->launches++;
  // Floor the residual diagonal at 0.1 of its mean: it is 0 at the pivots, and
  // L + dres must stay away from 0 for a well-conditioned Woodbury core.
  chunk_sum_kernel<<<nchunks, 256, 0, st>>>(h->dres, n, chunk, csum);
  h->launches++;
  std::vector<double> hsum(nchunks);
  if ((e = cudaMemcpyAsync(hsum.data(), csum, sizeof(double) * nchunks, cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
      (e = cudaStreamSynchronize(st)) != cudaSuccess) {
    cleanup();
    return cuda_fail(h, e, "residual diagonal");
  }
  double tot = 0.0;
  for (double v : hsum) tot += v;
  h->dres_mean = tot / (double)n;
  floor_kernel<<<grid_for(n), 256, 0, st>>>(h->dres, n, 0.1 * tot / (double)n);
  h->launches++;
  e = cudaStreamSynchronize(st);
  cleanup();
  if (e != cudaSuccess) return cuda_fail(h, e, "RPCholesky finish");
  return KQR_OK;
}

}  // namespace kqr
