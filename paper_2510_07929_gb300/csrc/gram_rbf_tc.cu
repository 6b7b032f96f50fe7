// RBF Gram product U = K V with the cross term on the tcgen05 tensor cores.
//
// K_ij = exp2(2 xs_i . xs_j - |xs_i|^2 - |xs_j|^2) (Sec. 1 RBF kernel, with
// xs = sqrt(gamma log2 e)(x - mean)).  The 128 x 128 tile of dot products
// xs_I xs_J^T is a dense contraction over p: it runs as tcgen05.mma kind::tf32
// (M = N = 128, K = 8 per instruction) from shared-memory tiles that TMA loads
// with the 128-byte swizzle, into an FP32 accumulator in tensor memory (two
// 128-column buffers, so the MMAs of tile q overlap the epilogue of tile q-1).
// FP32 accuracy comes from splitting xs = hi + lo into TF32 parts and summing
// hi.hi + hi.lo + lo.hi (the lo.lo term is below FP32 rounding); one term
// (hi.hi) gives the TF32 product.
//
// One CTA = 8 warps = 256 threads; thread t serves TMEM lane t mod 128 (row
// t mod 128 of the tile) over column half t / 128, reads its 64 accumulators
// with tcgen05.ld and accumulates exp2(...) v_j in registers (four independent
// chains per right-hand side, so the FFMAs do not serialise); the two halves
// of a row are added once at the end.  Thread 0 issues the TMA copies and the
// MMAs.  Column tiles are split over
// gridDim.y; per-split row sums are added in FP64 by a second kernel.
// Every mbarrier wait is bounded; on a timeout the CTA records the error,
// stops issuing work and frees its tensor memory.
#include <algorithm>
#include <vector>

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "kqr_internal.h"
#include "ptx.cuh"

namespace kqr {

__device__ __forceinline__ void tmem_alloc(uint32_t* dst, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst)), "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// D[tmem] (+)= A[smem] B[smem]^T, tf32 inputs, FP32 accumulate.
__device__ __forceinline__ void umma_tf32(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                          uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

// D[tmem] (+)= A[smem] B[smem]^T, kind::f16: bf16 or fp16 inputs as the instruction
// descriptor says (A and B of the same type), FP32 accumulate.
__device__ __forceinline__ void umma_f16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                          uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void umma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

// 32 consecutive FP32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// Shared-memory matrix descriptor: K-major operand in the canonical 128-byte
// swizzled layout (8-row groups 1024 bytes apart), tcgen05 version bits 0b001.
__device__ __forceinline__ uint64_t umma_desc_sw128(const void* p) {
  const uint32_t a = smem_u32(p);
  uint64_t d = (uint64_t)((a & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;              // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(1024 >> 4) << 32;    // stride byte offset
  d |= (uint64_t)1 << 46;              // fixed 0b001
  d |= (uint64_t)2 << 61;              // 128-byte swizzle
  return d;
}

constexpr uint32_t kAtomBytes = 128 * 128;   // 128 rows x 128 bytes (32 tf32 of K)

template <int M, int NTERMS>
__global__ void __launch_bounds__(256, 1)
    gram_rbf_tc_kernel(const __grid_constant__ CUtensorMap tm_hi, const __grid_constant__ CUtensorMap tm_lo,
                       const float* __restrict__ nrm, const float* __restrict__ v32, float* __restrict__ part,
                       int ksteps, int katoms, int ldn, int tiles_per_split, int col_tiles, int fold_rows,
                       int* __restrict__ err) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* base = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                                         ~static_cast<uintptr_t>(1023));
  const uint32_t tb = (uint32_t)katoms * kAtomBytes;   // one operand tile
  unsigned char* XIh = base;
  unsigned char* XIl = XIh + tb;
  unsigned char* XJh[2] = {XIl + tb, XIl + 3 * tb};
  unsigned char* XJl[2] = {XIl + 2 * tb, XIl + 4 * tb};
  float* s_nrm = reinterpret_cast<float*>(XIl + 5 * tb);   // [2][128]
  float* s_v = s_nrm + 2 * 128;                             // [2][128 * M]
  float* s_red = s_v + 2 * 128 * M;                         // [128 * M] second-half row sums
  uint64_t* bars = reinterpret_cast<uint64_t*>(s_red + 128 * M);  // 0: XI, 1-2: stages, 3-4: MMA buffers
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 5);
  int* abort_flag = reinterpret_cast<int*>(tmem_slot + 1);

  const int tid = threadIdx.x, warp = tid >> 5;
  const int row = tid & 127, half = tid >> 7;
  const int row0 = blockIdx.x * 128;
  const int split = blockIdx.y;
  const int jt0 = split * tiles_per_split;
  const int jt1 = min(col_tiles, jt0 + tiles_per_split);
  const int nt = jt1 - jt0;
  const uint32_t load_bytes = (NTERMS == 3 ? 2u : 1u) * tb;

  if (warp == 0) {
    tmem_alloc(tmem_slot, 256);
    tmem_relinquish();
  }
  if (tid == 0) {
    for (int i = 0; i < 5; ++i) mbar_init(&bars[i], 1);
    *abort_flag = 0;
    fence_mbar_init();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  auto load_tile = [&](unsigned char* dh, unsigned char* dl, int row, uint64_t* bar) {
    mbar_arrive_expect_tx(bar, load_bytes);
    for (int a = 0; a < katoms; ++a) {
      tma_load_2d(dh + a * kAtomBytes, &tm_hi, a * 32, row, bar);
      if (NTERMS == 3) tma_load_2d(dl + a * kAtomBytes, &tm_lo, a * 32, row, bar);
    }
  };
  if (tid == 0) {
    load_tile(XIh, XIl, row0, &bars[0]);
    if (nt > 0) load_tile(XJh[0], XJl[0], jt0 * 128, &bars[1]);
    if (nt > 1) load_tile(XJh[1], XJl[1], (jt0 + 1) * 128, &bars[2]);
  }
  // K_ij = exp2(2 g_ij - n_j) exp2(-n_i): with fold_rows the row factor exp2(-n_i)
  // multiplies the finished row sums instead of every entry (the host enables it
  // only when max n_i is small enough that exp2(2 g - n_j) <= exp2(n_i) cannot overflow).
  const float ni = nrm[row0 + row];
  const float ni_in = fold_rows ? 0.f : ni;
  float racc[M][4];
#pragma unroll
  for (int c = 0; c < M; ++c)
#pragma unroll
    for (int u = 0; u < 4; ++u) racc[c][u] = 0.f;
  // kind::tf32, FP32 accumulate, A and B K-major, N = 128, M = 128
  // FP32 accumulate, A and B K-major, N = 128, M = 128; operands TF32 (kind::tf32) or bf16 (kind::f16)
  const uint32_t idesc = (1u << 4) | (NTERMS == 0 ? (1u << 7) | (1u << 10) : (2u << 7) | (2u << 10)) |
                         ((128u >> 3) << 17) | ((128u >> 4) << 24);

  for (int q = 0; q <= nt; ++q) {
    if (q < nt && tid < 128) {
      const int col = (jt0 + q) * 128 + tid;
      s_nrm[(q & 1) * 128 + tid] = __ldg(nrm + col);
#pragma unroll
      for (int c = 0; c < M; ++c) s_v[(q & 1) * 128 * M + tid * M + c] = __ldg(v32 + (size_t)col * M + c);
    }
    if (q < nt && tid == 0) {
      bool ok = true;
      if (q == 0) ok = mbar_wait_bounded(&bars[0], 0, err);
      if (ok) ok = mbar_wait_bounded(&bars[1 + (q & 1)], (uint32_t)((q >> 1) & 1), err);
      if (ok) {
        tc_fence_after();
        const uint32_t d = tmem + (uint32_t)((q & 1) * 128);
        const unsigned char* bh = XJh[q & 1];
        const unsigned char* bl = XJl[q & 1];
        for (int k = 0; k < ksteps; ++k) {
          const uint32_t off = (uint32_t)(k >> 2) * kAtomBytes + (uint32_t)(k & 3) * 32u;
          if (NTERMS == 0) umma_f16(d, umma_desc_sw128(XIh + off), umma_desc_sw128(bh + off), idesc, k > 0 ? 1u : 0u);
          else umma_tf32(d, umma_desc_sw128(XIh + off), umma_desc_sw128(bh + off), idesc, k > 0 ? 1u : 0u);
          if (NTERMS == 3) {
            umma_tf32(d, umma_desc_sw128(XIh + off), umma_desc_sw128(bl + off), idesc, 1u);
            umma_tf32(d, umma_desc_sw128(XIl + off), umma_desc_sw128(bh + off), idesc, 1u);
          }
        }
        umma_commit(&bars[3 + (q & 1)]);
      } else {
        *abort_flag = 1;
      }
    }
    if (q >= 1) {
      const int pq = q - 1;
      const int b = pq & 1;
      if (mbar_wait_bounded(&bars[3 + b], (uint32_t)((pq >> 1) & 1), err)) {
        tc_fence_after();
        const uint32_t tbase = tmem + (uint32_t)(b * 128 + half * 64) + ((uint32_t)((warp & 3) * 32) << 16);
        const float* nj = s_nrm + b * 128 + half * 64;
        const float* vj = s_v + (b * 128 + half * 64) * M;
#pragma unroll 1
        for (int c4 = 0; c4 < 2; ++c4) {
          float g[32];
          tmem_ld32(tbase + (uint32_t)(c4 * 32), g);
#pragma unroll
          for (int j4 = 0; j4 < 8; ++j4) {
            const float4 n4 = *reinterpret_cast<const float4*>(nj + c4 * 32 + j4 * 4);
            const float nn[4] = {n4.x + ni_in, n4.y + ni_in, n4.z + ni_in, n4.w + ni_in};
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              const int jj = j4 * 4 + u;
              const int col = c4 * 32 + jj;
              const float e = ex2_approx(fmaf(2.f, g[jj], -nn[u]));
#pragma unroll
              for (int c = 0; c < M; ++c) racc[c][u] = fmaf(e, vj[col * M + c], racc[c][u]);
            }
          }
        }
      } else {
        *abort_flag = 1;
      }
      tc_fence_before();
    }
    __syncthreads();
    if (*abort_flag) break;
    // Stage (q + 1) & 1 held tile q - 1, whose MMAs completed above: refill it with tile q + 1.
    if (tid == 0 && q >= 1 && q + 1 < nt) load_tile(XJh[(q + 1) & 1], XJl[(q + 1) & 1], (jt0 + q + 1) * 128, &bars[1 + ((q + 1) & 1)]);
  }
  float rs[M];
  const float rowf = fold_rows ? ex2_approx(-ni) : 1.f;
#pragma unroll
  for (int c = 0; c < M; ++c) rs[c] = ((racc[c][0] + racc[c][1]) + (racc[c][2] + racc[c][3])) * rowf;
  if (half == 1) {
#pragma unroll
    for (int c = 0; c < M; ++c) s_red[row * M + c] = rs[c];
  }
  tc_fence_before();
  __syncthreads();
  if (half == 0) {
#pragma unroll
    for (int c = 0; c < M; ++c) part[((size_t)split * ldn + row0 + row) * M + c] = rs[c] + s_red[row * M + c];
  }
  if (warp == 0) tmem_dealloc(tmem, 256);
}

// xs32 (feature-major [p][ldn]) -> row-major TF32 parts [ldn][Kp], zero padded.
__global__ void tf32_split_kernel(const float* __restrict__ xs32, int64_t ldn, int p, int Kp, float* __restrict__ hi,
                                  float* __restrict__ lo) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < ldn * Kp; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / Kp;
    const int k = (int)(e % Kp);
    const float x = k < p ? xs32[(size_t)k * ldn + i] : 0.f;
    uint32_t h, l;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(h) : "f"(x));
    const float r = x - __uint_as_float(h);
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(l) : "f"(r));
    hi[e] = __uint_as_float(h);
    lo[e] = __uint_as_float(l);
  }
}

__global__ void tc_to_f32_kernel(const double* __restrict__ V, float* __restrict__ v32, int64_t n, int64_t ldn, int m,
                                 int M, double* __restrict__ sum_out) {
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

// out = sum of split partials (+ gam sum_p + L p for the CG operator); dot_out += p . out.
__global__ void tc_reduce_kernel(const float* __restrict__ part, int splits, int64_t ldn, int M, int m, int64_t n,
                                 double* __restrict__ out, GramEpilogue ep) {
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

static size_t tc_smem(int katoms, int M) {
  return 1024 + (size_t)6 * katoms * kAtomBytes + (2 * 128 + 3 * 128 * (size_t)M) * sizeof(float) + 5 * 8 + 16;
}

bool make_tmap_rowmajor_sw128(CUtensorMap* tm, void* base, int64_t ldn, int Kp);

// Prepares the TF32 row-major copies and their tensor maps (once per problem).
cudaError_t rbf_tc_prepare(Handle* h) {
  if (h->tc_hi) return cudaSuccess;
  const int Kp = h->p <= 32 ? 32 : 64;
  const size_t bytes = (size_t)h->ldn * Kp * sizeof(float);
  h->tc_hi = (float*)dev_alloc(h, bytes);
  h->tc_lo = (float*)dev_alloc(h, bytes);
  if (!h->tc_hi || !h->tc_lo) return cudaErrorMemoryAllocation;
  h->tc_Kp = Kp;
  // Fold the row factor exp2(-n_i) out of the entries when every n_i < 60:
  // then exp2(2 g - n_j) <= exp2(n_i) < 2^60 stays finite in FP32.
  {
    std::vector<float> nrm((size_t)h->ldn);
    cudaError_t e2 = cudaMemcpy(nrm.data(), h->nrm32, nrm.size() * sizeof(float), cudaMemcpyDeviceToHost);
    if (e2 != cudaSuccess) return e2;
    float mx = 0.f;
    for (float v : nrm) mx = v > mx ? v : mx;
    h->tc_fold_rows = mx < 60.f ? 1 : 0;
  }
  tf32_split_kernel<<<grid_for(h->ldn * Kp), 256, 0, h->stream>>>(h->xs32, h->ldn, (int)h->p, Kp, h->tc_hi, h->tc_lo);
  h->launches++;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (!make_tmap_rowmajor_sw128(&h->tm_tc_hi, h->tc_hi, h->ldn, Kp) ||
      !make_tmap_rowmajor_sw128(&h->tm_tc_lo, h->tc_lo, h->ldn, Kp))
    return cudaErrorInvalidValue;
  return cudaStreamSynchronize(h->stream);
}

// xs32 (feature-major [p][ldn]) -> the fp16 operands of the symmetric FP32-class tiles,
// row-major [ldn][W] halves: per row A' = [hi | hi | lo] and B' = [hi | lo | hi] over the
// p features (hi = fp16 round-to-nearest of x, lo = that of x - hi), zero beyond 3p.
// A'_j . B'_i = hi_j.hi_i + hi_j.lo_i + lo_j.hi_i, the three-term product of the TF32
// form with the same 11-bit parts, as one contraction of length 3p.
__global__ void f16_split_kernel(const float* __restrict__ xs32, int64_t ldn, int p, int W, __half* __restrict__ a,
                                 __half* __restrict__ b) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < ldn * W; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / W;
    const int k = (int)(e % W);
    __half va = __float2half_rn(0.f), vb = va;
    if (k < 3 * p) {
      const int seg = k / p;
      const float x = xs32[(size_t)(k % p) * ldn + i];
      const __half hi = __float2half_rn(x);
      const __half lo = __float2half_rn(x - __half2float(hi));
      va = seg == 2 ? lo : hi;
      vb = seg == 1 ? lo : hi;
    }
    a[e] = va;
    b[e] = vb;
  }
}

// Prepares the fp16 operands of the symmetric FP32-class tiles (once per problem).  Used
// only with folded row factors (every n_i < 60, so |xs| < 8: far inside the fp16 range; a
// lo part below 2^-14 loses bits as a subnormal, an absolute error of at most 2^-25 per
// part, below FP32 rounding of the cross term) and 3p <= 128.
static cudaError_t rbf_f16_prepare(Handle* h) {
  if (h->tc_a16) return cudaSuccess;
  const int katoms = (int)((3 * h->p + 63) / 64);
  const int W = 64 * katoms;
  const size_t bytes = (size_t)h->ldn * W * sizeof(__half);
  h->tc_a16 = (float*)dev_alloc(h, bytes);
  h->tc_b16 = (float*)dev_alloc(h, bytes);
  if (!h->tc_a16 || !h->tc_b16) return cudaErrorMemoryAllocation;
  h->tc16_katoms = katoms;
  f16_split_kernel<<<grid_for(h->ldn * W), 256, 0, h->stream>>>(h->xs32, h->ldn, (int)h->p, W,
                                                                 reinterpret_cast<__half*>(h->tc_a16),
                                                                 reinterpret_cast<__half*>(h->tc_b16));
  h->launches++;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  // a row of W halves is W / 2 FP32 words: the same 128-byte swizzled boxes as the TF32 parts
  if (!make_tmap_rowmajor_sw128(&h->tm_tc_a16, h->tc_a16, h->ldn, W / 2) ||
      !make_tmap_rowmajor_sw128(&h->tm_tc_b16, h->tc_b16, h->ldn, W / 2))
    return cudaErrorInvalidValue;
  return cudaStreamSynchronize(h->stream);
}

template <int M, int NT>
static cudaError_t launch_tc(Handle* h, int splits, int tps, int ksteps, cudaStream_t st) {
  const int katoms = NT == 0 ? 1 : h->tc_Kp / 32;
  const size_t smem = tc_smem(katoms, M);
  auto kern = gram_rbf_tc_kernel<M, NT>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int row_tiles = (int)(h->ldn / kTile);
  prof_mark(h, 0, true, st);
  kern<<<dim3(row_tiles, splits), 256, smem, st>>>(NT == 0 ? h->tm_tc_bf : h->tm_tc_hi, h->tm_tc_lo, h->nrm32,
                                                   h->v32, h->part, ksteps,
                                                   katoms, (int)h->ldn, tps, row_tiles, h->tc_fold_rows,
                                                   h->err_flag);
  prof_mark(h, 0, false, st);
  h->launches++;
  return cudaGetLastError();
}

// row-major bf16 copy [ldn][64] of xs32 (feature-major), round to nearest, zero padded.
__global__ void bf16_copy_kernel(const float* __restrict__ xs32, int64_t ldn, int p,
                                 __nv_bfloat16* __restrict__ out) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < ldn * 64; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / 64;
    const int k = (int)(e % 64);
    out[e] = __float2bfloat16_rn(k < p ? xs32[(size_t)k * ldn + i] : 0.f);
  }
}

bool make_tmap_rowmajor_bf16_sw128(CUtensorMap* tm, void* base, int64_t ldn);

static cudaError_t rbf_bf16_prepare(Handle* h) {
  if (h->tc_bf) return cudaSuccess;
  h->tc_bf = (__nv_bfloat16*)dev_alloc(h, (size_t)h->ldn * 64 * sizeof(__nv_bfloat16));
  if (!h->tc_bf) return cudaErrorMemoryAllocation;
  bf16_copy_kernel<<<grid_for(h->ldn * 64), 256, 0, h->stream>>>(h->xs32, h->ldn, (int)h->p, h->tc_bf);
  h->launches++;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (!make_tmap_rowmajor_bf16_sw128(&h->tm_tc_bf, h->tc_bf, h->ldn)) return cudaErrorInvalidValue;
  return cudaStreamSynchronize(h->stream);
}

// U = K V on the tensor cores; nt = 3: FP32 class (TF32 hi.hi + hi.lo + lo.hi), 1: TF32 (hi.hi),
// 0: bf16 (one term, K = 16 per instruction).
static cudaError_t rbf_tc_product(Handle* h, const double* V, double* U, int m, int nt, const GramEpilogue* ep,
                                  cudaStream_t st) {
  cudaError_t e = rbf_tc_prepare(h);
  if (e != cudaSuccess) return e;
  if (nt == 0 && (e = rbf_bf16_prepare(h)) != cudaSuccess) return e;
  const int M = m <= 1 ? 1 : (m <= 2 ? 2 : (m <= 4 ? 4 : 8));
  const int row_tiles = (int)(h->ldn / kTile), col_tiles = row_tiles;
  const int katoms = nt == 0 ? 1 : h->tc_Kp / 32;
  const int resident = tc_smem(katoms, M) * 2 <= 228 * 1024 ? 2 : 1;
  const int target = 8 * resident * h->num_sms;
  int s = (target + row_tiles - 1) / row_tiles;
  if (s < 1) s = 1;
  if (s > col_tiles) s = col_tiles;
  const int tps = (col_tiles + s - 1) / s;
  const int splits = (col_tiles + tps - 1) / tps;
  const size_t vb = (size_t)h->ldn * M * sizeof(float) * 2;
  if (h->v32_cap < vb) {
    dev_free(h, h->v32);
    h->v32 = (float*)dev_alloc(h, vb);
    h->v32_cap = h->v32 ? vb : 0;
    if (!h->v32) return cudaErrorMemoryAllocation;
  }
  const size_t pb = (size_t)splits * h->ldn * M * sizeof(float);
  if (h->part_cap < pb) {
    dev_free(h, h->part);
    h->part = (float*)dev_alloc(h, pb);
    h->part_cap = h->part ? pb : 0;
    if (!h->part) return cudaErrorMemoryAllocation;
  }
  GramEpilogue none;
  const GramEpilogue& g = ep ? *ep : none;
  double* sum_out = g.sum_p ? const_cast<double*>(g.sum_p) : nullptr;
  if (sum_out && (e = cudaMemsetAsync(sum_out, 0, sizeof(double), st)) != cudaSuccess) return e;
  tc_to_f32_kernel<<<grid_for(h->ldn * M), 256, 0, st>>>(V, h->v32, h->n, h->ldn, m, M, sum_out);
  h->launches++;
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  const int ksteps = nt == 0 ? (int)((h->p + 15) / 16) : (int)((h->p + 7) / 8);
  if (nt == 0) {
    switch (M) {
      case 1: e = launch_tc<1, 0>(h, splits, tps, ksteps, st); break;
      case 2: e = launch_tc<2, 0>(h, splits, tps, ksteps, st); break;
      case 4: e = launch_tc<4, 0>(h, splits, tps, ksteps, st); break;
      default: e = launch_tc<8, 0>(h, splits, tps, ksteps, st); break;
    }
  } else if (nt == 3) {
    switch (M) {
      case 1: e = launch_tc<1, 3>(h, splits, tps, ksteps, st); break;
      case 2: e = launch_tc<2, 3>(h, splits, tps, ksteps, st); break;
      case 4: e = launch_tc<4, 3>(h, splits, tps, ksteps, st); break;
      default: e = launch_tc<8, 3>(h, splits, tps, ksteps, st); break;
    }
  } else {
    switch (M) {
      case 1: e = launch_tc<1, 1>(h, splits, tps, ksteps, st); break;
      case 2: e = launch_tc<2, 1>(h, splits, tps, ksteps, st); break;
      case 4: e = launch_tc<4, 1>(h, splits, tps, ksteps, st); break;
      default: e = launch_tc<8, 1>(h, splits, tps, ksteps, st); break;
    }
  }
  if (e != cudaSuccess) return e;
  if (g.dot_out && (e = cudaMemsetAsync(g.dot_out, 0, sizeof(double), st)) != cudaSuccess) return e;
  tc_reduce_kernel<<<grid_for(h->n * m), 256, 0, st>>>(h->part, splits, h->ldn, M, m, h->n, U, g);
  h->launches++;
  return cudaGetLastError();
}

// ---- symmetric tiles for one right-hand side ------------------------------------------
// K is symmetric, so each off-diagonal 128 x 128 tile K_JI (J > I) is formed once on the
// tensor cores and used twice: u_J += K_JI v_I and u_I += K_JI^T v_J.  A work unit is a
// row tile I and a run of column tiles J in [J0, J1) with J0 >= I.  The MMA computes
// D = X_J X_I^T, so TMEM lane l is row j = J*128 + l and TMEM column c is i = I*128 + c.
//
// Operands (NTERMS): 3 = TF32 parts hi.hi + hi.lo + lo.hi, three MMAs per K = 8 step;
// 16 = the same three products from fp16 parts concatenated along K (A' = [hi | hi | lo]
// for J, B' = [hi | lo | hi] for I), one chain of ceil(3p / 16) MMAs of K = 16.  The MMAs
// of a tile accumulate into one TMEM buffer and so run one after another; the short
// chain of the fp16 form is what makes it faster; 1 = TF32 hi.hi alone (the TF32 product).
//
// One CTA = 8 warps, two CTAs per SM; warp w reads TMEM lanes 32 (w mod 4) .. + 31 (the
// lanes its warp may access) over the 64 columns 64 (w / 4) .. + 63.  Per element a thread
// forms e = exp2(2 xs_j.xs_i - n_j [- n_i]) and adds e w_i to its row j's sum (a register
// sum: u_J needs no exchange between threads) and e v_j to column i's sum, which stays in
// a register across all tiles of the unit (I is fixed), so the exchange across the warp's
// 32 rows happens once per unit.  With FOLD (every n < 60) exp2(-n_i) is folded into
// w_i = v_i exp2(-n_i) and into the column results.
//
// No CTA-wide barrier inside the tile loop: thread 0 issues the TMA copies and MMAs; a
// copy refills a stage once the MMAs that read it have completed (mma_done), an MMA
// reuses a TMEM buffer once all 8 warps have read it out (tmem_free, one arrival per
// warp).  Row sums go to the output with FP32 atomics per tile, column sums per unit.
// Every wait is bounded; on a timeout the CTA records the error, drains its own copies
// and MMAs (bounded) and frees its tensor memory.
constexpr int kSymWarps = 8;
constexpr int kSymCols = 64;  // columns of tile I per warp: two 32-column TMEM loads
constexpr int kSymBufs = 2;   // TMEM accumulator buffers of 128 columns (two CTAs per SM)

// nstage X_J stages; the MMAs of tile q are issued nstage / 2 iterations before its
// epilogue, and the copy of tile q + nstage is issued as soon as the MMAs of tile q have
// completed.
template <int NTERMS, bool FOLD>
__global__ void __launch_bounds__(kSymWarps * 32, 2)
    gram_rbf_tc_sym_kernel(const __grid_constant__ CUtensorMap tm_hi, const __grid_constant__ CUtensorMap tm_lo,
                           const float* __restrict__ nrm, const float* __restrict__ v32, const int4* __restrict__ units,
                           float* __restrict__ acc, int ksteps, int katoms, int nstage, int* __restrict__ err) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* base = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                                         ~static_cast<uintptr_t>(1023));
  const uint32_t tb = (uint32_t)katoms * kAtomBytes;
  unsigned char* XIh = base;
  unsigned char* XIl = XIh + tb;
  // stage s: hi part at base + (2 + 2 s) tb, lo part right after it
  float* s_w = reinterpret_cast<float*>(base + (size_t)(2 + 2 * nstage) * tb);   // [128] column factors of tile I
  float* s_ni = s_w + 128;                                                       // [128] n_i of tile I (without FOLD)
  uint64_t* bars = reinterpret_cast<uint64_t*>(s_ni + 128);
  uint64_t* full_i = &bars[0];
  uint64_t* full_j = &bars[1];                   // [nstage] X_J stage landed
  uint64_t* mma_done = &bars[1 + 4];             // [kSymBufs] MMAs of TMEM buffer b completed
  uint64_t* tmem_free = &bars[1 + 4 + kSymBufs]; // [kSymBufs] all warps have read TMEM buffer b
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 1 + 4 + 2 * kSymBufs);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  // thread 0's bookkeeping, in shared memory to spare registers: the latest tile whose copy,
  // and the latest whose MMAs, may still be in flight
  int* load_pending = reinterpret_cast<int*>(tmem_slot + 2);
  int* mma_pending = load_pending + 1;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int lq = warp & 3, cq = warp >> 2;
  const int4 unit = units[blockIdx.x];
  const int ti = unit.x;
  const int jt0 = unit.y, jt1 = unit.z;
  const int nt = jt1 - jt0;
  const int look = nstage / 2;
  const uint32_t load_bytes = (NTERMS == 3 ? 2u : 1u) * tb;

  if (warp == 0) {
    tmem_alloc(tmem_slot, 128 * kSymBufs);
    tmem_relinquish();
  }
  if (tid == 0) {
    mbar_init(full_i, 1);
    for (int s = 0; s < nstage; ++s) mbar_init(&full_j[s], 1);
    for (int b = 0; b < kSymBufs; ++b) {
      mbar_init(&mma_done[b], 1);
      mbar_init(&tmem_free[b], kSymWarps);
    }
    *abort_flag = 0;
    fence_mbar_init();
  }
  if (tid < 128) {
    const float n_i = nrm[ti * 128 + tid];
    s_w[tid] = v32[ti * 128 + tid] * (FOLD ? ex2_approx(-n_i) : 1.f);
    s_ni[tid] = n_i;
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  auto stage_hi = [&](int s) { return base + (size_t)(2 + 2 * s) * tb; };
  auto load_tile = [&](int t) {   // tile t of the unit into stage t mod nstage
    const int s = t % nstage;
    unsigned char* dh = stage_hi(s);
    mbar_arrive_expect_tx(&full_j[s], load_bytes);
    for (int a = 0; a < katoms; ++a) {
      tma_load_2d(dh + a * kAtomBytes, &tm_hi, a * 32, (jt0 + t) * 128, &full_j[s]);
      if (NTERMS == 3) tma_load_2d(dh + tb + a * kAtomBytes, &tm_lo, a * 32, (jt0 + t) * 128, &full_j[s]);
    }
  };
  if (tid == 0) {
    *load_pending = -1;
    *mma_pending = -1;
    mbar_arrive_expect_tx(full_i, load_bytes);
    for (int a = 0; a < katoms; ++a) {
      // with fp16 operands tm_hi maps A' (the J rows) and tm_lo maps B' (the I rows)
      tma_load_2d(XIh + a * kAtomBytes, NTERMS == 16 ? &tm_lo : &tm_hi, a * 32, ti * 128, full_i);
      if (NTERMS == 3) tma_load_2d(XIl + a * kAtomBytes, &tm_lo, a * 32, ti * 128, full_i);
    }
    for (int t = 0; t < nstage && t < nt; ++t) {
      load_tile(t);
      *load_pending = t;
    }
  }
  // FP32 accumulate, A and B K-major, N = 128, M = 128; operands TF32 (format 2) or fp16 (0)
  const uint32_t idesc = (1u << 4) | (NTERMS == 16 ? 0u : (2u << 7) | (2u << 10)) | ((128u >> 3) << 17) |
                         ((128u >> 4) << 24);
  float cacc[kSymCols];   // column sums of tile I over this warp's 32 rows, across the unit's tiles
#pragma unroll
  for (int c = 0; c < kSymCols; ++c) cacc[c] = 0.f;
  bool ok = true;   // warp-uniform: every wait of this warp succeeded
  // this thread's row of the next epilogue tile, loaded one tile ahead
  const int jrow = jt0 * 128 + lq * 32 + lane;
  float n_nx = __ldg(nrm + jrow);
  float v_nx = jt0 == ti ? 0.f : __ldg(v32 + jrow);   // the diagonal tile gives row sums only

  for (int q = 0; q < nt + look; ++q) {
    if (tid == 0 && q < nt) {
      const int s = q % nstage, b = q % kSymBufs;
      bool w_ok = true;
      if (q == 0) w_ok = mbar_wait_bounded(full_i, 0, err);
      if (w_ok) w_ok = mbar_wait_bounded(&full_j[s], (uint32_t)((q / nstage) & 1), err);
      // TMEM buffer b last held tile q - kSymBufs: every warp must have read it out
      if (w_ok && q >= kSymBufs)
        w_ok = mbar_wait_bounded(&tmem_free[b], (uint32_t)((q / kSymBufs - 1) & 1), err);
      if (w_ok) {
        tc_fence_after();
        const uint32_t d = tmem + (uint32_t)(b * 128);
        const unsigned char* ah = stage_hi(s);
        const unsigned char* al = ah + tb;
        for (int k = 0; k < ksteps; ++k) {
          const uint32_t off = (uint32_t)(k >> 2) * kAtomBytes + (uint32_t)(k & 3) * 32u;
          if (NTERMS == 16) umma_f16(d, umma_desc_sw128(ah + off), umma_desc_sw128(XIh + off), idesc, k > 0 ? 1u : 0u);
          else umma_tf32(d, umma_desc_sw128(ah + off), umma_desc_sw128(XIh + off), idesc, k > 0 ? 1u : 0u);
          if (NTERMS == 3) {
            umma_tf32(d, umma_desc_sw128(ah + off), umma_desc_sw128(XIl + off), idesc, 1u);
            umma_tf32(d, umma_desc_sw128(al + off), umma_desc_sw128(XIh + off), idesc, 1u);
          }
        }
        umma_commit(&mma_done[b]);
        *mma_pending = q;
      } else {
        *abort_flag = 1;
      }
    }
    if (q >= look) {
      const int pq = q - look, b = pq % kSymBufs;
      const float n_j = n_nx, v_j = v_nx;
      if (pq + 1 < nt) {
        n_nx = __ldg(nrm + jrow + (pq + 1) * 128);
        v_nx = jt0 + pq + 1 == ti ? 0.f : __ldg(v32 + jrow + (pq + 1) * 128);
      }
      const bool landed = __all_sync(
          0xffffffffu, *abort_flag == 0 && mbar_wait_bounded(&mma_done[b], (uint32_t)((pq / kSymBufs) & 1), err));
      if (!landed) {
        ok = false;
        *abort_flag = 1;
        break;
      }
      tc_fence_after();
      // the MMAs of tile pq have completed, so its stage is free: refill it with tile pq + nstage
      if (tid == 0 && pq + nstage < nt) {
        load_tile(pq + nstage);
        *load_pending = pq + nstage;
      }
      float racc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
      for (int h = 0; h < kSymCols / 32; ++h) {
      float g[32];
      tmem_ld32(tmem + (uint32_t)(b * 128 + cq * kSymCols + h * 32) + ((uint32_t)(lq * 32) << 16), g);
      if (h == kSymCols / 32 - 1) {
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&tmem_free[b]);
      }
      const float* wq = s_w + cq * kSymCols + h * 32;
      const float* nq = s_ni + cq * kSymCols + h * 32;
#pragma unroll
      for (int c4 = 0; c4 < 8; ++c4) {
        const float4 w4 = *reinterpret_cast<const float4*>(wq + c4 * 4);
        const float ww[4] = {w4.x, w4.y, w4.z, w4.w};
        float nn[4] = {n_j, n_j, n_j, n_j};
        if (!FOLD) {
          const float4 n4 = *reinterpret_cast<const float4*>(nq + c4 * 4);
          nn[0] += n4.x;
          nn[1] += n4.y;
          nn[2] += n4.z;
          nn[3] += n4.w;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int c = c4 * 4 + u;
          const float e = ex2_approx(fmaf(2.f, g[c], -nn[u]));
          racc[u] = fmaf(e, ww[u], racc[u]);
          cacc[h * 32 + c] = fmaf(e, v_j, cacc[h * 32 + c]);
        }
      }
      }
      atomicAdd(acc + jrow + pq * 128, (racc[0] + racc[1]) + (racc[2] + racc[3]));
    }
  }
  // column sums: reduce-scatter each 32 column partials over the warp's 32 rows, so that
  // lane l ends with column cq kSymCols + 32 h + l of tile I
  if (__all_sync(0xffffffffu, ok && *abort_flag == 0)) {
#pragma unroll
    for (int h = 0; h < kSymCols / 32; ++h) {
      float* ch = cacc + h * 32;
#pragma unroll
      for (int w = 16; w >= 1; w >>= 1) {
        const bool up = (lane & w) != 0;
#pragma unroll
        for (int i = 0; i < w; ++i) {
          const float keep = up ? ch[i + w] : ch[i], send = up ? ch[i] : ch[i + w];
          ch[i] = keep + __shfl_xor_sync(0xffffffffu, send, w);
        }
      }
      const int col = cq * kSymCols + h * 32 + lane;
      const float f = FOLD ? ex2_approx(-s_ni[col]) : 1.f;
      atomicAdd(acc + ti * 128 + col, ch[0] * f);
    }
  }
  if (tid == 0 && *abort_flag) {
    // a wait gave up: let this CTA's own copies and MMAs finish (bounded) before it frees
    // its tensor memory and exits; copies go out in tile order, so each stage's latest is
    // one of the last nstage tiles issued, and the last commit covers every earlier MMA
    mbar_wait_bounded(full_i, 0, err);
    const int lp = *load_pending, mp = *mma_pending;
    for (int t = lp; t >= 0 && t > lp - nstage; --t)
      mbar_wait_bounded(&full_j[t % nstage], (uint32_t)((t / nstage) & 1), err);
    if (mp >= 0) mbar_wait_bounded(&mma_done[mp % kSymBufs], (uint32_t)((mp / kSymBufs) & 1), err);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, 128 * kSymBufs);
}

static int tc_sym_stages(int) { return 2; }

static size_t tc_sym_smem(int katoms) {
  return 1024 + (size_t)(2 + 2 * tc_sym_stages(katoms)) * katoms * kAtomBytes + 256 * sizeof(float) +
         (1 + 4 + 2 * kSymBufs) * sizeof(uint64_t) + 32;
}

cudaError_t sym_prep(Handle* h, const double* V, float* v32, float* acc, double* sum_out, cudaStream_t st);

// Work units of the symmetric tensor-core tiles: (row tile I, column tiles [J0, J1)) with
// I <= J0, about 8 per SM (one CTA resident), so that each CTA's TMA/MMA pipeline runs over
// tens of tiles; the longest units come first, for the block scheduler's tail.
static cudaError_t tc_sym_units_ensure(Handle* h) {
  const int T = (int)(h->ldn / kTile);
  if (h->tc_sym_units && h->tc_sym_T == T) return cudaSuccess;
  const int64_t pairs = (int64_t)T * (T + 1) / 2;
  const int64_t target = (int64_t)8 * h->num_sms;
  int C = (int)((pairs + target - 1) / target);
  if (C < 1) C = 1;
  std::vector<int4> u;
  for (int I = 0; I < T; ++I)
    for (int J0 = I; J0 < T; J0 += C) u.push_back(make_int4(I, J0, J0 + C < T ? J0 + C : T, 0));
  std::stable_sort(u.begin(), u.end(), [](const int4& a, const int4& b) { return a.z - a.y > b.z - b.y; });
  dev_free(h, h->tc_sym_units);
  h->tc_sym_units = (int4*)dev_alloc(h, u.size() * sizeof(int4));
  if (!h->tc_sym_units) return cudaErrorMemoryAllocation;
  h->tc_sym_nunits = (int)u.size();
  h->tc_sym_T = T;
  return cudaMemcpy(h->tc_sym_units, u.data(), u.size() * sizeof(int4), cudaMemcpyHostToDevice);
}
cudaError_t sym_finish(Handle* h, const float* acc, double* U, const GramEpilogue& g, cudaStream_t st);

// m = 1 RBF product on symmetric tensor-core tiles; nt = 3: FP32 class (fp16 parts when
// the row factors fold and 3p <= 128, else TF32 parts), 1: TF32.
static cudaError_t rbf_tc_sym_product(Handle* h, const double* V, double* U, int nt, const GramEpilogue* ep,
                                      cudaStream_t st) {
  cudaError_t e = rbf_tc_prepare(h);
  if (e != cudaSuccess) return e;
  if ((e = tc_sym_units_ensure(h)) != cudaSuccess) return e;
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
  if ((e = sym_prep(h, V, v32, acc, g.sum_p ? const_cast<double*>(g.sum_p) : nullptr, st)) != cudaSuccess) return e;
  const bool f16 = nt == 3 && h->tc_fold_rows && 3 * h->p <= 128;
  if (f16 && (e = rbf_f16_prepare(h)) != cudaSuccess) return e;
  const int katoms = f16 ? h->tc16_katoms : h->tc_Kp / 32;
  const int ksteps = f16 ? (int)((3 * h->p + 15) / 16) : (int)((h->p + 7) / 8);
  const size_t smem = tc_sym_smem(katoms);
  auto kern = f16 ? gram_rbf_tc_sym_kernel<16, true>
                  : nt == 3 ? (h->tc_fold_rows ? gram_rbf_tc_sym_kernel<3, true> : gram_rbf_tc_sym_kernel<3, false>)
                            : (h->tc_fold_rows ? gram_rbf_tc_sym_kernel<1, true> : gram_rbf_tc_sym_kernel<1, false>);
  if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
    return e;
  prof_mark(h, 0, true, st);
  kern<<<h->tc_sym_nunits, kSymWarps * 32, smem, st>>>(f16 ? h->tm_tc_a16 : h->tm_tc_hi, f16 ? h->tm_tc_b16 : h->tm_tc_lo,
                                                       h->nrm32, v32, h->tc_sym_units, acc, ksteps, katoms,
                                                       tc_sym_stages(katoms), h->err_flag);
  prof_mark(h, 0, false, st);
  h->launches++;
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  return sym_finish(h, acc, U, g, st);
}

cudaError_t gram_rbf_tc(Handle* h, const double* V, double* U, int m, bool three_terms, const GramEpilogue* ep,
                        cudaStream_t st) {
  if (m == 1 && h->opt.symmetric_gram) return rbf_tc_sym_product(h, V, U, three_terms ? 3 : 1, ep, st);
  return rbf_tc_product(h, V, U, m, three_terms ? 3 : 1, ep, st);
}

cudaError_t gram_rbf_tc_bf16(Handle* h, const double* V, double* U, int m, cudaStream_t st) {
  return rbf_tc_product(h, V, U, m, 0, nullptr, st);
}

}  // namespace kqr
