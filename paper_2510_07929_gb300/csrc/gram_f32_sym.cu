// Symmetric FP32 Gram product u = K v (one right-hand side).
//
// K is symmetric, so each off-diagonal 128 x 128 tile K_IJ (J > I) is formed
// once and used twice: u_I += K_IJ v_J (row sums) and u_J += K_IJ^T v_I
// (column sums).  Diagonal tiles give row sums only.  This halves the kernel
// entries formed per product (n^2/2 + O(n) instead of n^2).
//
// Work units are (row tile I, column tiles [J0, J1)) with J0 >= I, about 64
// per resident CTA, listed in a table built once per problem; a CTA TMA-loads
// its row tile once and double-buffers the column tiles as in the plain
// kernel.  Column sums are reduced across the 16 row groups of the CTA through
// shared memory (double-buffered by tile parity) and added to the output with
// FP32 atomics, as are the unit's row sums at the end; the order of those
// additions is not fixed, so results vary in the last bits between runs.
#include <vector>

#include "kqr_internal.h"
#include "ptx.cuh"

namespace kqr {

enum { SYM_RBF = 0, SYM_LAP = 1 };

template <int KIND>
__global__ void __launch_bounds__(kThreads, 2)
    gram_f32_sym_kernel(const __grid_constant__ CUtensorMap tm, const float* __restrict__ nrm,
                        const float* __restrict__ v32, const int4* __restrict__ units, float* __restrict__ acc, int p,
                        int* __restrict__ err) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  float* XI = reinterpret_cast<float*>(smem_raw);
  float* XJ0 = XI + p * kTile;
  float* XJ1 = XJ0 + p * kTile;
  float* colred = XJ1 + p * kTile;        // 2 buffers x 4 row-group warps x 128 columns
  float* rowred = colred + 2 * 4 * kTile; // 2 column-group warps x 128 rows
  uint64_t* bars = reinterpret_cast<uint64_t*>(rowred + 2 * kTile);

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int ty = (warp >> 1) * 4 + (lane >> 3);
  const int tx = (warp & 1) * 8 + (lane & 7);
  const int4 unit = units[blockIdx.x];
  const int row0 = unit.x * kTile;
  const int jt0 = unit.y, jt1 = unit.z;
  const uint32_t bytes = (uint32_t)p * kTile * 4u;

  if (tid == 0) {
    mbar_init(&bars[0], 1);
    mbar_init(&bars[1], 1);
    mbar_init(&bars[2], 1);
    fence_mbar_init();
  }
  __syncthreads();
  if (tid == 0) {
    mbar_arrive_expect_tx(&bars[0], bytes);
    tma_load_2d(XI, &tm, row0, 0, &bars[0]);
    mbar_arrive_expect_tx(&bars[1], bytes);
    tma_load_2d(XJ0, &tm, jt0 * kTile, 0, &bars[1]);
  }
  float va[8], ni[8];
#pragma unroll
  for (int a = 0; a < 8; ++a) {
    va[a] = __ldg(v32 + row0 + ty * 8 + a);
    ni[a] = (KIND == SYM_RBF) ? __ldg(nrm + row0 + ty * 8 + a) : 0.f;
  }
  float racc[8];
#pragma unroll
  for (int a = 0; a < 8; ++a) racc[a] = 0.f;
  if (!mbar_wait_bounded(&bars[0], 0, err)) return;

  for (int t = jt0; t < jt1; ++t) {
    const int q = t - jt0;
    const int s = q & 1;
    float* XJ = s ? XJ1 : XJ0;
    if (tid == 0 && t + 1 < jt1) {
      const int ns = (q + 1) & 1;
      mbar_arrive_expect_tx(&bars[1 + ns], bytes);
      tma_load_2d(ns ? XJ1 : XJ0, &tm, (t + 1) * kTile, 0, &bars[1 + ns]);
    }
    const int col0 = t * kTile + tx * 8;
    float vb[8], nj[8];
#pragma unroll
    for (int b = 0; b < 8; ++b) {
      vb[b] = __ldg(v32 + col0 + b);
      nj[b] = (KIND == SYM_RBF) ? __ldg(nrm + col0 + b) : 0.f;
    }
    if (!mbar_wait_bounded(&bars[1 + s], (uint32_t)((q >> 1) & 1), err)) return;

    float d[8][8];
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
      for (int b = 0; b < 8; ++b) d[a][b] = 0.f;
#pragma unroll 2
    for (int k = 0; k < p; ++k) {
      const float4 a0 = *reinterpret_cast<const float4*>(XI + k * kTile + ty * 8);
      const float4 a1 = *reinterpret_cast<const float4*>(XI + k * kTile + ty * 8 + 4);
      const float4 b0 = *reinterpret_cast<const float4*>(XJ + k * kTile + tx * 8);
      const float4 b1 = *reinterpret_cast<const float4*>(XJ + k * kTile + tx * 8 + 4);
      const float xa[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      const float xb[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
      for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int b = 0; b < 8; ++b) {
          if (KIND == SYM_LAP)
            d[a][b] += fabsf(xa[a] - xb[b]);
          else
            d[a][b] = fmaf(xa[a], xb[b], d[a][b]);
        }
    }
    float cs[8];
#pragma unroll
    for (int b = 0; b < 8; ++b) cs[b] = 0.f;
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
      for (int b = 0; b < 8; ++b) {
        const float arg = (KIND == SYM_LAP) ? -d[a][b] : fmaf(2.f, d[a][b], -(ni[a] + nj[b]));
        const float e = ex2_approx(arg);
        racc[a] = fmaf(e, vb[b], racc[a]);
        cs[b] = fmaf(e, va[a], cs[b]);
      }
    const bool offdiag = (t != unit.x);   // uniform over the CTA
    float* cr = colred + s * (4 * kTile);
    if (offdiag) {
      // column sums: reduce over the 4 row groups of the warp, then the 4 row-group warps
#pragma unroll
      for (int b = 0; b < 8; ++b) {
        cs[b] += __shfl_xor_sync(0xffffffffu, cs[b], 8);
        cs[b] += __shfl_xor_sync(0xffffffffu, cs[b], 16);
      }
      if ((lane >> 3) == 0) {
#pragma unroll
        for (int b = 0; b < 8; ++b) cr[(warp >> 1) * kTile + tx * 8 + b] = cs[b];
      }
    }
    __syncthreads();
    if (offdiag && tid < kTile) {
      const float c = cr[tid] + cr[kTile + tid] + cr[2 * kTile + tid] + cr[3 * kTile + tid];
      atomicAdd(acc + t * kTile + tid, c);
    }
  }

  // row sums: reduce over the 8 lanes of a row group, then the 2 column-group warps
#pragma unroll
  for (int a = 0; a < 8; ++a) {
    float v = racc[a];
    v += __shfl_xor_sync(0xffffffffu, v, 1);
    v += __shfl_xor_sync(0xffffffffu, v, 2);
    v += __shfl_xor_sync(0xffffffffu, v, 4);
    racc[a] = v;
  }
  if ((lane & 7) == 0) {
#pragma unroll
    for (int a = 0; a < 8; ++a) rowred[(warp & 1) * kTile + ty * 8 + a] = racc[a];
  }
  __syncthreads();
  if (tid < kTile) atomicAdd(acc + row0 + tid, rowred[tid] + rowred[kTile + tid]);
}

// v (FP64, n) -> v32 [ldn] zero padded; acc [ldn] zeroed; optional sum of v.
__global__ void sym_prep_kernel(const double* __restrict__ V, float* __restrict__ v32, float* __restrict__ acc,
                                int64_t n, int64_t ldn, double* __restrict__ sum_out) {
  double s = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < ldn; i += (int64_t)gridDim.x * blockDim.x) {
    const double x = i < n ? V[i] : 0.0;
    v32[i] = (float)x;
    acc[i] = 0.f;
    s += x;
  }
  if (sum_out) {
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    __shared__ double ws[32];
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += ws[w];
      atomicAdd(sum_out, t);
    }
  }
}

// out = acc (+ gam sum_p + L p), dot_out += p . out, raw_out = acc.
__global__ void sym_finish_kernel(const float* __restrict__ acc, int64_t n, double* __restrict__ out, GramEpilogue ep) {
  double dot = 0.0;
  const double sump = ep.sum_p ? *ep.sum_p : 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double s = (double)acc[i];
    if (ep.raw_out) ep.raw_out[i] = s;
    if (ep.L) s += (ep.gam_dev ? *ep.gam_dev : ep.gam) * sump + ep.L[i] * ep.pvec[i];
    out[i] = s;
    if (ep.dot_out) dot += ep.pvec[i] * s;
  }
  if (ep.dot_out) {
    for (int o = 16; o > 0; o >>= 1) dot += __shfl_xor_sync(0xffffffffu, dot, o);
    __shared__ double ws[32];
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = dot;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += ws[w];
      atomicAdd(ep.dot_out, t);
    }
  }
}

static size_t sym_smem_bytes(int p) {
  return ((size_t)3 * p * kTile + 2 * 4 * kTile + 2 * kTile) * sizeof(float) + 4 * sizeof(uint64_t);
}

// Work-unit table: for each row tile I, column tiles [J0, J1) with I <= J0,
// chunks of C tiles, C chosen for ~64 units per resident CTA.
cudaError_t sym_units_ensure(Handle* h) {
  const int T = (int)(h->ldn / kTile);
  if (h->sym_units && h->sym_T == T) return cudaSuccess;
  const int64_t pairs = (int64_t)T * (T + 1) / 2;
  const int64_t target = (int64_t)64 * 2 * h->num_sms;
  int C = (int)((pairs + target - 1) / target);
  if (C < 1) C = 1;
  std::vector<int4> u;
  for (int I = 0; I < T; ++I)
    for (int J0 = I; J0 < T; J0 += C) u.push_back(make_int4(I, J0, J0 + C < T ? J0 + C : T, 0));
  dev_free(h, h->sym_units);
  h->sym_units = (int4*)dev_alloc(h, u.size() * sizeof(int4));
  if (!h->sym_units) return cudaErrorMemoryAllocation;
  h->sym_nunits = (int)u.size();
  h->sym_T = T;
  return cudaMemcpy(h->sym_units, u.data(), u.size() * sizeof(int4), cudaMemcpyHostToDevice);
}

cudaError_t gram_f32_sym(Handle* h, const double* V, double* U, const GramEpilogue* ep, cudaStream_t st) {
  cudaError_t e = sym_units_ensure(h);
  if (e != cudaSuccess) return e;
  const size_t need = (size_t)h->ldn * sizeof(float) * 2;   // v32 + acc
  if (h->v32_cap < need) {
    dev_free(h, h->v32);
    h->v32 = (float*)dev_alloc(h, need);
    h->v32_cap = h->v32 ? need : 0;
    if (!h->v32) return cudaErrorMemoryAllocation;
  }
  float* v32 = h->v32;
  float* acc = h->v32 + h->ldn;
  GramEpilogue none;
  const GramEpilogue& g = ep ? *ep : none;
  double* sum_out = g.sum_p ? const_cast<double*>(g.sum_p) : nullptr;
  if (sum_out && (e = cudaMemsetAsync(sum_out, 0, sizeof(double), st)) != cudaSuccess) return e;
  sym_prep_kernel<<<grid_for(h->ldn), 256, 0, st>>>(V, v32, acc, h->n, h->ldn, sum_out);
  h->launches++;
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  const size_t smem = sym_smem_bytes((int)h->p);
  prof_mark(h, 0, true, st);
  if (h->kind == KQR_LAPLACIAN) {
    e = cudaFuncSetAttribute(gram_f32_sym_kernel<SYM_LAP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    gram_f32_sym_kernel<SYM_LAP><<<h->sym_nunits, kThreads, smem, st>>>(h->tm_xs32, h->nrm32, v32, h->sym_units, acc,
                                                                        (int)h->p, h->err_flag);
  } else {
    e = cudaFuncSetAttribute(gram_f32_sym_kernel<SYM_RBF>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    gram_f32_sym_kernel<SYM_RBF><<<h->sym_nunits, kThreads, smem, st>>>(h->tm_xs32, h->nrm32, v32, h->sym_units, acc,
                                                                        (int)h->p, h->err_flag);
  }
  prof_mark(h, 0, false, st);
  h->launches++;
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (g.dot_out && (e = cudaMemsetAsync(g.dot_out, 0, sizeof(double), st)) != cudaSuccess) return e;
  sym_finish_kernel<<<grid_for(h->n), 256, 0, st>>>(acc, h->n, U, g);
  h->launches++;
  return cudaGetLastError();
}

}  // namespace kqr

namespace kqr {

// v -> FP32 copy and zeroed FP32 accumulator (and 1^T v into *sum_out if given),
// for products that accumulate with atomics (symmetric tiles, stored K).
cudaError_t sym_prep(Handle* h, const double* V, float* v32, float* acc, double* sum_out, cudaStream_t st) {
  cudaError_t e;
  if (sum_out && (e = cudaMemsetAsync(sum_out, 0, sizeof(double), st)) != cudaSuccess) return e;
  sym_prep_kernel<<<grid_for(h->ldn), 256, 0, st>>>(V, v32, acc, h->n, h->ldn, sum_out);
  h->launches++;
  return cudaGetLastError();
}

// out = acc (+ the CG operator's terms of g), as at the end of gram_f32_sym.
cudaError_t sym_finish(Handle* h, const float* acc, double* U, const GramEpilogue& g, cudaStream_t st) {
  cudaError_t e;
  if (g.dot_out && (e = cudaMemsetAsync(g.dot_out, 0, sizeof(double), st)) != cudaSuccess) return e;
  sym_finish_kernel<<<grid_for(h->n), 256, 0, st>>>(acc, h->n, U, g);
  h->launches++;
  return cudaGetLastError();
}

}  // namespace kqr
