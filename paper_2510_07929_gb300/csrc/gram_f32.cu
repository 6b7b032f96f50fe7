// FP32 Gram products U = K V with kernel entries formed on the fly in tiles.
//
// K_ij = k(x_i, x_j) of Sec. 1 (text after eq. (1.1)).  X is stored centred,
// feature-major ([p][ldn]) and pre-scaled so that
//   Laplacian: K_ij = exp2(-sum_k |xs_ik - xs_jk|),       xs = gamma log2(e) (x - mean)
//   RBF:       K_ij = exp2(2 xs_i.xs_j - |xs_i|^2 - |xs_j|^2), xs = sqrt(gamma log2(e)) (x - mean)
// (centring is exact for these translation-invariant kernels).  A CTA owns a
// 128-row block; it TMA-loads that block once and then double-buffers
// 128-column tiles of X through shared memory.  Each of its 256 threads keeps
// an 8 x 8 block of distances in registers (2 FP32 ops per feature for L1, one
// FFMA per feature for the dot product), then applies ex2 and accumulates
// e_ij V_j into per-row sums, so the kernel matrix never leaves registers.
// Column tiles are split over gridDim.y; per-split row sums go to a scratch
// buffer and a second kernel adds them in FP64 (deterministic order).
#include <cstdio>

#include "kqr_internal.h"
#include "ptx.cuh"

namespace kqr {

enum { KIND_RBF = 0, KIND_LAP = 1 };

template <int KIND, int M>
__global__ void __launch_bounds__(kThreads, (M <= 2) ? 2 : 1)
    gram_f32_kernel(const __grid_constant__ CUtensorMap tm, const float* __restrict__ nrm,
                    const float* __restrict__ v32, float* __restrict__ part, int p, int ldn,
                    int tiles_per_split, int col_tiles, int* __restrict__ err) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  float* XI = reinterpret_cast<float*>(smem_raw);
  float* XJ0 = XI + p * kTile;
  float* XJ1 = XJ0 + p * kTile;
  float* red = XJ1 + p * kTile;  // 2 x 128 x M floats for the final row reduction
  uint64_t* bars = reinterpret_cast<uint64_t*>(red + 2 * kTile * M);

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int ty = (warp >> 1) * 4 + (lane >> 3);  // row group 0..15
  const int tx = (warp & 1) * 8 + (lane & 7);    // column group 0..15
  const int row0 = blockIdx.x * kTile;
  const int split = blockIdx.y;
  const int jt0 = split * tiles_per_split;
  const int jt1 = min(col_tiles, jt0 + tiles_per_split);
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
    if (jt0 < jt1) {
      mbar_arrive_expect_tx(&bars[1], bytes);
      tma_load_2d(XJ0, &tm, jt0 * kTile, 0, &bars[1]);
    }
  }

  float ni[8];
  if (KIND == KIND_RBF) {
    const float4 q0 = *reinterpret_cast<const float4*>(nrm + row0 + ty * 8);
    const float4 q1 = *reinterpret_cast<const float4*>(nrm + row0 + ty * 8 + 4);
    ni[0] = q0.x; ni[1] = q0.y; ni[2] = q0.z; ni[3] = q0.w;
    ni[4] = q1.x; ni[5] = q1.y; ni[6] = q1.z; ni[7] = q1.w;
  }
  float racc[8][M];
#pragma unroll
  for (int a = 0; a < 8; ++a)
#pragma unroll
    for (int c = 0; c < M; ++c) racc[a][c] = 0.f;

  if (!mbar_wait_bounded(&bars[0], 0, err)) return;

  for (int t = jt0; t < jt1; ++t) {
    const int q = t - jt0;
    const int s = q & 1;
    float* XJ = s ? XJ1 : XJ0;
    if (tid == 0 && t + 1 < jt1) {
      // Buffer (q + 1) & 1 was last read in iteration q - 1, which every
      // thread left through the __syncthreads() at its end.
      const int ns = (q + 1) & 1;
      mbar_arrive_expect_tx(&bars[1 + ns], bytes);
      tma_load_2d(ns ? XJ1 : XJ0, &tm, (t + 1) * kTile, 0, &bars[1 + ns]);
    }
    const int col0 = t * kTile + tx * 8;
    float vb[8][M];
#pragma unroll
    for (int b = 0; b < 8; ++b)
#pragma unroll
      for (int c = 0; c < M; ++c) vb[b][c] = __ldg(v32 + (size_t)(col0 + b) * M + c);
    float nj[8];
    if (KIND == KIND_RBF) {
#pragma unroll
      for (int b = 0; b < 8; ++b) nj[b] = __ldg(nrm + col0 + b);
    }
    if (!mbar_wait_bounded(&bars[1 + s], (uint32_t)((q >> 1) & 1), err)) return;

    float acc[8][8];
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
      for (int b = 0; b < 8; ++b) acc[a][b] = 0.f;

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
          if (KIND == KIND_LAP)
            acc[a][b] += fabsf(xa[a] - xb[b]);
          else
            acc[a][b] = fmaf(xa[a], xb[b], acc[a][b]);
        }
    }
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
      for (int b = 0; b < 8; ++b) {
        const float arg = (KIND == KIND_LAP) ? -acc[a][b] : fmaf(2.f, acc[a][b], -(ni[a] + nj[b]));
        const float e = ex2_approx(arg);
#pragma unroll
        for (int c = 0; c < M; ++c) racc[a][c] = fmaf(e, vb[b][c], racc[a][c]);
      }
    __syncthreads();
  }

  // Row sums: reduce over the 8 lanes of a row group, then over the 2 warps.
#pragma unroll
  for (int a = 0; a < 8; ++a)
#pragma unroll
    for (int c = 0; c < M; ++c) {
      float v = racc[a][c];
      v += __shfl_xor_sync(0xffffffffu, v, 1);
      v += __shfl_xor_sync(0xffffffffu, v, 2);
      v += __shfl_xor_sync(0xffffffffu, v, 4);
      racc[a][c] = v;
    }
  const int wc = warp & 1;
  if ((lane & 7) == 0) {
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
      for (int c = 0; c < M; ++c) red[((wc * 16 + ty) * 8 + a) * M + c] = racc[a][c];
  }
  __syncthreads();
  for (int idx = tid; idx < kTile * M; idx += kThreads) {
    const int row = idx / M, c = idx % M;
    const int g = row >> 3, a = row & 7;
    const float s0 = red[((0 * 16 + g) * 8 + a) * M + c];
    const float s1 = red[((1 * 16 + g) * 8 + a) * M + c];
    part[((size_t)split * ldn + row0 + row) * M + c] = s0 + s1;
  }
}

// V (FP64, n x m) -> v32 (FP32, ldn x M, zero padded); optionally sum of V[:, 0].
__global__ void to_f32_kernel(const double* __restrict__ V, float* __restrict__ v32, int64_t n, int64_t ldn,
                              int m, int M, double* __restrict__ sum_out) {
  double s = 0.0;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < ldn * M;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = idx / M;
    const int c = (int)(idx % M);
    const double x = (i < n && c < m) ? V[i * m + c] : 0.0;
    v32[idx] = (float)x;
    if (c == 0) s += x;
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

__global__ void gram_reduce_kernel(const float* __restrict__ part, int splits, int64_t ldn, int M, int m,
                                   int64_t n, double* __restrict__ out, GramEpilogue ep) {
  double dot = 0.0;
  const double sump = ep.sum_p ? *ep.sum_p : 0.0;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < n * m;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t row = idx / m;
    const int c = (int)(idx % m);
    double s = 0.0;
    for (int sp = 0; sp < splits; ++sp) s += (double)part[((size_t)sp * ldn + row) * M + c];
    if (ep.raw_out) ep.raw_out[idx] = s;
    if (ep.L) s += (ep.gam_dev ? *ep.gam_dev : ep.gam) * sump + ep.L[row] * ep.pvec[row];
    out[idx] = s;
    if (ep.dot_out) dot += ep.pvec[row] * s;
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

static size_t f32_smem_bytes(int p, int M) {
  return ((size_t)3 * p * kTile + (size_t)2 * kTile * M) * sizeof(float) + 4 * sizeof(uint64_t);
}

template <int KIND, int M>
static cudaError_t launch_tiles(Handle* h, int splits, int tiles_per_split, cudaStream_t st) {
  const int row_tiles = (int)(h->ldn / kTile);
  const int col_tiles = row_tiles;
  const size_t smem = f32_smem_bytes((int)h->p, M);
  auto kern = gram_f32_kernel<KIND, M>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  dim3 grid(row_tiles, splits);
  prof_mark(h, 0, true, st);
  kern<<<grid, kThreads, smem, st>>>(h->tm_xs32, h->nrm32, h->v32, h->part, (int)h->p, (int)h->ldn,
                                     tiles_per_split, col_tiles, h->err_flag);
  prof_mark(h, 0, false, st);
  h->launches++;
  return cudaGetLastError();
}

template <int M>
static cudaError_t launch_kind(Handle* h, int splits, int tps, cudaStream_t st) {
  return h->kind == KQR_LAPLACIAN ? launch_tiles<KIND_LAP, M>(h, splits, tps, st)
                                  : launch_tiles<KIND_RBF, M>(h, splits, tps, st);
}

static cudaError_t ensure(Handle* h, void** buf, size_t* cap, size_t bytes) {
  if (*cap >= bytes) return cudaSuccess;
  dev_free(h, *buf);
  *buf = dev_alloc(h, bytes);
  *cap = *buf ? bytes : 0;
  return *buf ? cudaSuccess : cudaErrorMemoryAllocation;
}

// Number of column splits: about 8 waves of resident CTAs, at most one split per tile.
static void pick_splits(Handle* h, int resident_per_sm, int* splits, int* tps) {
  const int row_tiles = (int)(h->ldn / kTile);
  const int col_tiles = row_tiles;
  const int target = 8 * resident_per_sm * h->num_sms;
  int s = (target + row_tiles - 1) / row_tiles;
  if (s < 1) s = 1;
  if (s > col_tiles) s = col_tiles;
  *tps = (col_tiles + s - 1) / s;
  *splits = (col_tiles + *tps - 1) / *tps;
}

cudaError_t gram_f32(Handle* h, const double* V, double* U, int m, const GramEpilogue* ep, cudaStream_t st) {
  if (m == 1 && h->kstore) return gram_stored(h, V, U, ep, st);
  if (h->kind == KQR_RBF && h->opt.rbf_tensor_cores) return gram_rbf_tc(h, V, U, m, true, ep, st);
  if (m == 1 && h->opt.symmetric_gram) return gram_f32_sym(h, V, U, ep, st);
  const int M = m <= 1 ? 1 : (m <= 2 ? 2 : (m <= 4 ? 4 : 8));
  int splits, tps;
  pick_splits(h, M <= 2 ? 2 : 1, &splits, &tps);
  cudaError_t e = ensure(h, (void**)&h->v32, &h->v32_cap, (size_t)h->ldn * M * sizeof(float) * 2);
  if (e != cudaSuccess) return e;
  e = ensure(h, (void**)&h->part, &h->part_cap, (size_t)splits * h->ldn * M * sizeof(float));
  if (e != cudaSuccess) return e;
  double* sum_out = (ep && ep->sum_p) ? const_cast<double*>(ep->sum_p) : nullptr;
  if (sum_out) {
    e = cudaMemsetAsync(sum_out, 0, sizeof(double), st);
    if (e != cudaSuccess) return e;
  }
  to_f32_kernel<<<grid_for(h->ldn * M), 256, 0, st>>>(V, h->v32, h->n, h->ldn, m, M, sum_out);
  h->launches++;
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  switch (M) {
    case 1: e = launch_kind<1>(h, splits, tps, st); break;
    case 2: e = launch_kind<2>(h, splits, tps, st); break;
    case 4: e = launch_kind<4>(h, splits, tps, st); break;
    default: e = launch_kind<8>(h, splits, tps, st); break;
  }
  if (e != cudaSuccess) return e;
  GramEpilogue none;
  const GramEpilogue& g = ep ? *ep : none;
  if (g.dot_out) {
    e = cudaMemsetAsync(g.dot_out, 0, sizeof(double), st);
    if (e != cudaSuccess) return e;
  }
  gram_reduce_kernel<<<grid_for(h->n * m), 256, 0, st>>>(h->part, splits, h->ldn, M, m, h->n, U, g);
  h->launches++;
  return cudaGetLastError();
}

// Same product as gram_f32 (no CG epilogue), with the FP32 copy of V and the
// per-split partial sums placed in caller-provided scratch instead of handle
// buffers.  *need receives the scratch bytes this (n, m) requires; when cap is
// smaller nothing is launched and cudaErrorInvalidValue is returned.
template <int KIND, int M>
static cudaError_t launch_tiles_into(Handle* h, int splits, int tiles_per_split, const float* v32, float* part,
                                     cudaStream_t st) {
  const int row_tiles = (int)(h->ldn / kTile);
  const size_t smem = f32_smem_bytes((int)h->p, M);
  auto kern = gram_f32_kernel<KIND, M>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<dim3(row_tiles, splits), kThreads, smem, st>>>(h->tm_xs32, h->nrm32, v32, part, (int)h->p, (int)h->ldn,
                                                        tiles_per_split, row_tiles, h->err_flag);
  h->launches++;
  return cudaGetLastError();
}

template <int M>
static cudaError_t launch_kind_into(Handle* h, int splits, int tps, const float* v32, float* part, cudaStream_t st) {
  return h->kind == KQR_LAPLACIAN ? launch_tiles_into<KIND_LAP, M>(h, splits, tps, v32, part, st)
                                  : launch_tiles_into<KIND_RBF, M>(h, splits, tps, v32, part, st);
}

cudaError_t gram_f32_scratch(Handle* h, const double* V, double* U, int m, unsigned char* scratch, size_t cap,
                             size_t* need, cudaStream_t st) {
  const int M = m <= 1 ? 1 : (m <= 2 ? 2 : (m <= 4 ? 4 : 8));
  int splits, tps;
  pick_splits(h, M <= 2 ? 2 : 1, &splits, &tps);
  const size_t vbytes = ((size_t)h->ldn * M * sizeof(float) + 255) / 256 * 256;
  const size_t pbytes = (size_t)splits * h->ldn * M * sizeof(float);
  *need = vbytes + pbytes;
  if (*need > cap) return cudaErrorInvalidValue;
  float* v32 = reinterpret_cast<float*>(scratch);
  float* part = reinterpret_cast<float*>(scratch + vbytes);
  // to_f32_kernel writes all ldn * M entries and the tile kernel writes every
  // (split, row) partial, so nothing read here is left over from an earlier call.
  to_f32_kernel<<<grid_for(h->ldn * M), 256, 0, st>>>(V, v32, h->n, h->ldn, m, M, nullptr);
  h->launches++;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  switch (M) {
    case 1: e = launch_kind_into<1>(h, splits, tps, v32, part, st); break;
    case 2: e = launch_kind_into<2>(h, splits, tps, v32, part, st); break;
    case 4: e = launch_kind_into<4>(h, splits, tps, v32, part, st); break;
    default: e = launch_kind_into<8>(h, splits, tps, v32, part, st); break;
  }
  if (e != cudaSuccess) return e;
  GramEpilogue none;
  gram_reduce_kernel<<<grid_for(h->n * m), 256, 0, st>>>(part, splits, h->ldn, M, m, h->n, U, none);
  h->launches++;
  return cudaGetLastError();
}

}  // namespace kqr
