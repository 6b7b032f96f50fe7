// Stored-K Gram product u = K v (one right-hand side) for kernel matrices
// whose packed upper triangle fits in device memory.
//
// The products inside CG ((2.1), (3.1)) multiply the same K (Sec. 1 kernel
// entries) hundreds of times.  When the upper triangle fits in HBM, forming
// each entry once and streaming it afterwards is cheaper than forming it on
// the fly every product: a product then reads 4 bytes per stored entry,
// n(n+1)/2 entries, and is bound by HBM bandwidth.
//
// Layout: the upper-triangle tile pairs (I, J >= I) of 128 x 128 FP32 tiles,
// in row-major order of (I, J), each tile row-major and contiguous (64 KB).
// Tile t of row tile I starts at ks_row_start(I) = I T - I (I - 1) / 2 with
// T = ldn / 128.  Entries with a row or column index >= n are stored as 0.
//
// Fill (once per problem): one CTA per tile, FP32 arithmetic identical to the
// on-the-fly CUDA-core tiles (exp2 of -L1 or of 2 xs_i.xs_j - |xs_i|^2 - |xs_j|^2).
//
// Product: a persistent kernel, one CTA per SM, each CTA a contiguous range of
// tiles.  Warp 8 streams the range through shared memory in 16 KB chunks
// (32 rows x 128 columns) with bulk copies (cp.async.bulk) into an 8-stage
// ring guarded by mbarriers (full: bytes landed; empty: the 8 consumer warps
// released it).  Warp w of the 8 consumer warps takes rows 4w..4w+3 of every
// chunk, lane l columns 4l..4l+3: each stored entry gives one FFMA into its
// row's sum (K_IJ v_J) and, off the diagonal, one into its column's sum
// (K_IJ^T v_I).  Row sums stay in registers while the row tile I is
// unchanged and go to the output with FP32 atomics when it changes; column
// sums are reduced over the 8 warps in shared memory and added with FP32
// atomics per tile.  Every wait is bounded; after a timeout the CTA records
// the error, stops issuing copies, keeps its barrier sequence (no warp is
// left waiting at a named barrier) and, before exiting, waits (bounded) for
// the copies it issued.
#include <cmath>
#include <vector>

#include "kqr_internal.h"
#include "ptx.cuh"

namespace kqr {

cudaError_t sym_prep(Handle* h, const double* V, float* v32, float* acc, double* sum_out, cudaStream_t st);
cudaError_t sym_finish(Handle* h, const float* acc, double* U, const GramEpilogue& g, cudaStream_t st);

constexpr int kKsTileFloats = kTile * kTile;                     // 16384 floats = 64 KB
constexpr int kKsChunkRows = 32;
constexpr int kKsChunkFloats = kKsChunkRows * kTile;            // 4096 floats
constexpr uint32_t kKsChunkBytes = kKsChunkFloats * 4u;          // 16 KB
constexpr int kKsChunksPerTile = kTile / kKsChunkRows;          // 4
constexpr int kKsStages = 8;
constexpr int kKsConsumerWarps = 8;
constexpr int kKsThreads = (kKsConsumerWarps + 1) * 32;          // + the copy warp

__host__ __device__ inline int64_t ks_row_start(int64_t I, int64_t T) { return I * T - I * (I - 1) / 2; }

__host__ __device__ inline void ks_decode(int64_t t, int64_t T, int* I, int* J) {
  const double b = 2.0 * (double)T + 1.0;
  int64_t i = (int64_t)floor((b - sqrt(b * b - 8.0 * (double)t)) * 0.5);
  if (i < 0) i = 0;
  if (i > T - 1) i = T - 1;
  while (i + 1 < T && ks_row_start(i + 1, T) <= t) ++i;
  while (i > 0 && ks_row_start(i, T) > t) --i;
  *I = (int)i;
  *J = (int)(i + (t - ks_row_start(i, T)));
}

__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void consumer_sync() { asm volatile("bar.sync 1, 256;" ::: "memory"); }

enum { KS_RBF = 0, KS_LAP = 1 };

// One CTA per stored tile t = blockIdx.x: K_IJ entries in FP32, zero outside n x n.
template <int KIND>
__global__ void __launch_bounds__(256) kstore_fill_kernel(const float* __restrict__ xs32, const float* __restrict__ nrm,
                                                          int p, int64_t ldn, int64_t n, int64_t T,
                                                          float* __restrict__ K) {
  extern __shared__ __align__(16) float ks_smem[];
  float* XI = ks_smem;
  float* XJ = ks_smem + p * kTile;
  const int64_t t = blockIdx.x;
  int I, J;
  ks_decode(t, T, &I, &J);
  for (int e = threadIdx.x; e < p * kTile; e += blockDim.x) {
    const int k = e / kTile, c = e % kTile;
    XI[e] = xs32[(size_t)k * ldn + (size_t)I * kTile + c];
    XJ[e] = xs32[(size_t)k * ldn + (size_t)J * kTile + c];
  }
  __syncthreads();
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int ty = (warp >> 1) * 4 + (lane >> 3);
  const int tx = (warp & 1) * 8 + (lane & 7);
  float d[8][8];
#pragma unroll
  for (int a = 0; a < 8; ++a)
#pragma unroll
    for (int b = 0; b < 8; ++b) d[a][b] = 0.f;
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
        if (KIND == KS_LAP)
          d[a][b] += fabsf(xa[a] - xb[b]);
        else
          d[a][b] = fmaf(xa[a], xb[b], d[a][b]);
      }
  }
  float* out = K + (size_t)t * kKsTileFloats;
  const int64_t col0 = (int64_t)J * kTile + tx * 8;
#pragma unroll
  for (int a = 0; a < 8; ++a) {
    const int r = ty * 8 + a;
    const int64_t row = (int64_t)I * kTile + r;
    const float ni = (KIND == KS_RBF) ? nrm[row] : 0.f;
    float e[8];
#pragma unroll
    for (int b = 0; b < 8; ++b) {
      const float arg = (KIND == KS_LAP) ? -d[a][b] : fmaf(2.f, d[a][b], -(ni + nrm[col0 + b]));
      e[b] = (row < n && col0 + b < n) ? ex2_approx(arg) : 0.f;
    }
    float4* o = reinterpret_cast<float4*>(out + r * kTile + tx * 8);
    o[0] = make_float4(e[0], e[1], e[2], e[3]);
    o[1] = make_float4(e[4], e[5], e[6], e[7]);
  }
}

// Symmetric streaming product over the stored tiles; sched[b] = (t0, t1, I0, J0)
// is CTA b's tile range and the (I, J) of its first tile.
__global__ void __launch_bounds__(kKsThreads, 1)
    kstore_gemv_kernel(const float* __restrict__ K, const float* __restrict__ v32, float* __restrict__ acc,
                       const int4* __restrict__ sched, int T, int* __restrict__ err) {
  extern __shared__ __align__(128) unsigned char ks_raw[];
  float* stages = reinterpret_cast<float*>(ks_raw);                              // kKsStages x 4096
  float* colred = stages + kKsStages * kKsChunkFloats;                           // [2][8][128]
  uint64_t* full = reinterpret_cast<uint64_t*>(colred + 2 * kKsConsumerWarps * kTile);
  uint64_t* empty = full + kKsStages;
  volatile int* abort_flag = reinterpret_cast<volatile int*>(empty + kKsStages);

  const int4 sc = sched[blockIdx.x];
  const int t0 = sc.x, t1 = sc.y;
  const int nchunks = (t1 - t0) * kKsChunksPerTile;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < kKsStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], kKsConsumerWarps);
    }
    *abort_flag = 0;
    fence_mbar_init();
  }
  __syncthreads();

  if (warp == kKsConsumerWarps) {
    // ---- copy warp: one thread streams the CTA's chunks into the ring
    if (lane == 0) {
      const float* src = K + (size_t)t0 * kKsTileFloats;
      int issued = 0;
      for (int c = 0; c < nchunks; ++c) {
        const int s = c % kKsStages;
        if (c >= kKsStages && !mbar_wait_bounded(&empty[s], (uint32_t)(((c / kKsStages) - 1) & 1), err)) {
          *abort_flag = 1;
          break;
        }
        if (*abort_flag) break;
        mbar_arrive_expect_tx(&full[s], kKsChunkBytes);
        bulk_load(stages + s * kKsChunkFloats, src + (size_t)c * kKsChunkFloats, kKsChunkBytes, &full[s]);
        issued = c + 1;
      }
      // The CTA must not exit with a copy in flight: wait (bounded) for the
      // last copy issued on every stage (consumers normally have already).
      const int first = issued > kKsStages ? issued - kKsStages : 0;
      for (int c = first; c < issued; ++c)
        (void)mbar_wait_bounded(&full[c % kKsStages], (uint32_t)((c / kKsStages) & 1), err);
    }
    return;
  }

  // ---- consumer warps 0..7
  int I = sc.z, J = sc.w;
  float vi[16];                       // v over this warp's 16 rows of row tile I
  float4 vj = make_float4(0.f, 0.f, 0.f, 0.f);
  float rp[16];
  float col[4];
  float row_acc = 0.f;                // lane's row (lane >> 1 of the warp's 16) summed over tiles of this I
  int parity = 0;                     // colred buffer, flipped per off-diagonal tile
  bool aborted = false;
  auto load_vi = [&](int Irow) {
#pragma unroll
    for (int r = 0; r < 16; ++r) vi[r] = __ldg(v32 + (size_t)Irow * kTile + (r >> 2) * kKsChunkRows + 4 * warp + (r & 3));
  };
  const int ntiles = t1 - t0;
  if (ntiles > 0) load_vi(I);
  for (int tl = 0; tl < ntiles; ++tl) {
#pragma unroll
    for (int r = 0; r < 16; ++r) rp[r] = 0.f;
#pragma unroll
    for (int j = 0; j < 4; ++j) col[j] = 0.f;
    vj = __ldg(reinterpret_cast<const float4*>(v32 + (size_t)J * kTile) + lane);
#pragma unroll
    for (int q = 0; q < kKsChunksPerTile; ++q) {
      const int c = tl * kKsChunksPerTile + q;
      const int s = c % kKsStages;
      if (!aborted && *abort_flag) aborted = true;
      if (!aborted && !mbar_wait_bounded(&full[s], (uint32_t)((c / kKsStages) & 1), err)) {
        *abort_flag = 1;
        aborted = true;
      }
      if (!aborted) {
        const float* ch = stages + s * kKsChunkFloats;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const float4 e = *reinterpret_cast<const float4*>(ch + (4 * warp + k) * kTile + 4 * lane);
          float r = rp[q * 4 + k];
          r = fmaf(e.x, vj.x, r);
          r = fmaf(e.y, vj.y, r);
          r = fmaf(e.z, vj.z, r);
          r = fmaf(e.w, vj.w, r);
          rp[q * 4 + k] = r;
          const float a = vi[q * 4 + k];
          col[0] = fmaf(e.x, a, col[0]);
          col[1] = fmaf(e.y, a, col[1]);
          col[2] = fmaf(e.z, a, col[2]);
          col[3] = fmaf(e.w, a, col[3]);
        }
      }
      __syncwarp();
      if (lane == 0 && !aborted) mbar_arrive(&empty[s]);
    }
    // row sums of the warp's 16 rows: reduce-scatter over the 32 lanes; lanes
    // l and l ^ 1 end with the full sum of row r = l >> 1 (rows r of rp are
    // tile rows (r >> 2) * 32 + 4 * warp + (r & 3)).
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const bool up = lane & 16;
      const float keep = up ? rp[i + 8] : rp[i], send = up ? rp[i] : rp[i + 8];
      rp[i] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const bool up = lane & 8;
      const float keep = up ? rp[i + 4] : rp[i], send = up ? rp[i] : rp[i + 4];
      rp[i] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
    }
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      const bool up = lane & 4;
      const float keep = up ? rp[i + 2] : rp[i], send = up ? rp[i] : rp[i + 2];
      rp[i] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
    }
    {
      const bool up = lane & 2;
      const float keep = up ? rp[1] : rp[0], send = up ? rp[0] : rp[1];
      rp[0] = keep + __shfl_xor_sync(0xffffffffu, send, 2);
    }
    rp[0] += __shfl_xor_sync(0xffffffffu, rp[0], 1);
    row_acc += rp[0];
    if (J != I) {
      float* cr = colred + parity * (kKsConsumerWarps * kTile);
      *reinterpret_cast<float4*>(cr + warp * kTile + 4 * lane) = make_float4(col[0], col[1], col[2], col[3]);
      consumer_sync();
      if (threadIdx.x < kTile && !aborted) {
        float sum = 0.f;
#pragma unroll
        for (int w = 0; w < kKsConsumerWarps; ++w) sum += cr[w * kTile + threadIdx.x];
        atomicAdd(acc + (size_t)J * kTile + threadIdx.x, sum);
      }
      parity ^= 1;
    }
    const bool last = (tl == ntiles - 1);
    const int nI = (J + 1 < T) ? I : I + 1;
    const int nJ = (J + 1 < T) ? J + 1 : I + 1;
    if (last || nI != I) {
      if ((lane & 1) == 0 && !aborted) {
        const int r = lane >> 1;
        atomicAdd(acc + (size_t)I * kTile + (r >> 2) * kKsChunkRows + 4 * warp + (r & 3), row_acc);
      }
      row_acc = 0.f;
      if (!last) load_vi(nI);
    }
    I = nI;
    J = nJ;
  }
}

constexpr size_t kStoreL2Bytes = (size_t)64 << 20;   // stored tiles up to this size stay in L2

size_t kstore_bytes(int64_t ldn) {
  const int64_t T = ldn / kTile;
  return (size_t)(T * (T + 1) / 2) * kKsTileFloats * sizeof(float);
}

static size_t kstore_smem() {
  return (size_t)kKsStages * kKsChunkBytes + (size_t)2 * kKsConsumerWarps * kTile * sizeof(float) +
         2 * kKsStages * sizeof(uint64_t) + 16;
}

kqr_status kstore_setup(Handle* h) {
  const int mode = h->opt.gram_store;
  if (mode == 0 || h->kstore) return KQR_OK;
  const size_t bytes = kstore_bytes(h->ldn);
  size_t free_b = 0, total_b = 0;
  cudaError_t e = cudaMemGetInfo(&free_b, &total_b);
  if (e != cudaSuccess) return cuda_fail(h, e, "cudaMemGetInfo");
  if (mode == 2 && bytes > free_b / 2) return KQR_OK;   // automatic: only when it fits comfortably
  // automatic: once the stored tiles no longer fit in L2, the symmetric tcgen05 RBF tiles
  // (p <= 32, one 128-byte atom per row) form K faster than a stored K streams from HBM
  // (0.48 against 0.74 ms at n = 50000)
  if (mode == 2 && h->kind == KQR_RBF && h->opt.rbf_tensor_cores && h->opt.symmetric_gram && h->p <= 32 &&
      bytes > kStoreL2Bytes)
    return KQR_OK;
  const int64_t T = h->ldn / kTile;
  const int64_t ntiles = T * (T + 1) / 2;
  if (ntiles > (int64_t)INT32_MAX / kKsChunksPerTile) return mode == 1 ? fail(h, KQR_INVALID_ARG, "K too large to store") : KQR_OK;
  float* K = (float*)dev_alloc(h, bytes);
  if (!K) {
    if (mode == 1) return fail(h, KQR_OOM, "stored K: " + std::to_string(bytes) + " bytes");
    cudaGetLastError();
    return KQR_OK;
  }
  // per-CTA tile ranges of the product
  const int G = h->num_sms > 0 ? h->num_sms : 1;
  std::vector<int4> sched(G);
  for (int b = 0; b < G; ++b) {
    const int64_t a = ntiles * b / G, c = ntiles * (b + 1) / G;
    int I = 0, J = 0;
    if (a < ntiles) ks_decode(a, T, &I, &J);
    sched[b] = make_int4((int)a, (int)c, I, J);
  }
  int4* dsched = (int4*)dev_alloc(h, sizeof(int4) * G);
  if (!dsched) {
    dev_free(h, K);
    if (mode == 1) return fail(h, KQR_OOM, "stored K schedule");
    return KQR_OK;
  }
  cudaStream_t st = h->stream;
  if ((e = cudaMemcpyAsync(dsched, sched.data(), sizeof(int4) * G, cudaMemcpyHostToDevice, st)) != cudaSuccess) {
    dev_free(h, K);
    dev_free(h, dsched);
    return cuda_fail(h, e, "stored K schedule");
  }
  const size_t fill_smem = (size_t)2 * h->p * kTile * sizeof(float);
  if (h->kind == KQR_LAPLACIAN) {
    e = cudaFuncSetAttribute(kstore_fill_kernel<KS_LAP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fill_smem);
    if (e == cudaSuccess)
      kstore_fill_kernel<KS_LAP><<<(unsigned)ntiles, 256, fill_smem, st>>>(h->xs32, h->nrm32, (int)h->p, h->ldn, h->n,
                                                                           T, K);
  } else {
    e = cudaFuncSetAttribute(kstore_fill_kernel<KS_RBF>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fill_smem);
    if (e == cudaSuccess)
      kstore_fill_kernel<KS_RBF><<<(unsigned)ntiles, 256, fill_smem, st>>>(h->xs32, h->nrm32, (int)h->p, h->ldn, h->n,
                                                                           T, K);
  }
  h->launches++;
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaFuncSetAttribute(kstore_gemv_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)kstore_smem());
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    dev_free(h, K);
    dev_free(h, dsched);
    return cuda_fail(h, e, "stored K fill");
  }
  h->kstore = K;
  h->kstore_bytes = bytes;
  h->kstore_sched = dsched;
  h->kstore_grid = G;
  return KQR_OK;
}

void kstore_free(Handle* h) {
  dev_free(h, h->kstore);
  dev_free(h, h->kstore_sched);
  h->kstore = nullptr;
  h->kstore_sched = nullptr;
  h->kstore_bytes = 0;
}

cudaError_t gram_stored(Handle* h, const double* V, double* U, const GramEpilogue* ep, cudaStream_t st) {
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
  cudaError_t e = sym_prep(h, V, v32, acc, g.sum_p ? const_cast<double*>(g.sum_p) : nullptr, st);
  if (e != cudaSuccess) return e;
  prof_mark(h, 2, true, st);
  kstore_gemv_kernel<<<h->kstore_grid, kKsThreads, kstore_smem(), st>>>(h->kstore, v32, acc, h->kstore_sched,
                                                                       (int)(h->ldn / kTile), h->err_flag);
  prof_mark(h, 2, false, st);
  h->launches++;
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  return sym_finish(h, acc, U, g, st);
}

}  // namespace kqr
