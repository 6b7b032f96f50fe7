// Symmetric FP64-class Laplacian Gram product u = K v (one right-hand side).
//
// Same arithmetic as gram_lap_high_kernel (exact int32 fixed-point L1
// distances, table-driven double-float exp2, double-float accumulation), but
// each off-diagonal tile K_IJ (J > I) is formed once and used for both
// u_I += K_IJ v_J and u_J += K_IJ^T v_I, over the work units of the
// symmetric FP32 product.  Per tile, a thread's 8-row column partials are
// summed in double-float, converted to FP64, reduced over the CTA's row
// groups and added to the output with FP64 atomics (order not fixed: results
// vary in the last FP64 bits between runs).
#include "kqr_internal.h"
#include "ptx.cuh"

namespace kqr {

cudaError_t sym_units_ensure(Handle* h);

constexpr int kTBs = kExpTableBits;
constexpr float kLn2HiS = 0.693147182464599609375f;
constexpr float kLn2LoS = -1.904654323148236e-09f;

// 2^-(A 2^-G + lo) as a double-float (k_hi, k_lo); A >= 0 exact, |lo| small.
__device__ __forceinline__ void df_exp2_neg(int Ai, float lo, int G, int shift_f, int mask_f, int mask_r, float scaleG,
                                            const float2* tab, float& k_hi, float& k_lo) {
  const int eint = Ai >> G;
  const int kidx = (Ai >> shift_f) & mask_f;
  const int rem = Ai & mask_r;
  const float rem_f = __fsub_rn(__int_as_float(rem | 0x4B000000), 8388608.f);
  const float ap = __fmul_rn(rem_f, scaleG);
  const float r_hi = __fadd_rn(ap, lo);
  const float bb = __fsub_rn(r_hi, ap);
  const float r_lo = __fadd_rn(__fsub_rn(ap, __fsub_rn(r_hi, bb)), __fsub_rn(lo, bb));
  const float x_hi = __fmul_rn(r_hi, kLn2HiS);
  float x_lo = fmaf(r_hi, kLn2HiS, -x_hi);
  x_lo = fmaf(r_hi, kLn2LoS, x_lo);
  x_lo = fmaf(r_lo, kLn2HiS, x_lo);
  const float tail = __fmul_rn(__fmul_rn(x_hi, x_hi), fmaf(x_hi, fmaf(x_hi, 1.f / 24.f, -1.f / 6.f), 0.5f));
  const float P_hi = __fsub_rn(1.f, x_hi);
  const float P_lo = __fadd_rn(__fsub_rn(__fsub_rn(__fsub_rn(1.f, P_hi), x_hi), x_lo), tail);
  const float2 T = tab[kidx];
  float kh = __fmul_rn(T.x, P_hi);
  float kl = fmaf(T.x, P_hi, -kh);
  kl = fmaf(T.x, P_lo, kl);
  kl = fmaf(T.y, P_hi, kl);
  const float sc = (eint < 100) ? __int_as_float((127 - eint) << 23) : 0.f;
  k_hi = __fmul_rn(kh, sc);
  k_lo = __fmul_rn(kl, sc);
}

// (s_hi, s_lo) += (k_hi, k_lo) (v_hi, v_lo), TwoSum on the leading terms.
__device__ __forceinline__ void df_acc(float& s_hi, float& s_lo, float k_hi, float k_lo, float v_hi, float v_lo) {
  const float p_hi = __fmul_rn(k_hi, v_hi);
  float p_lo = fmaf(k_hi, v_hi, -p_hi);
  p_lo = fmaf(k_hi, v_lo, p_lo);
  p_lo = fmaf(k_lo, v_hi, p_lo);
  const float sum = __fadd_rn(s_hi, p_hi);
  const float bv = __fsub_rn(sum, s_hi);
  const float e2 = __fadd_rn(__fsub_rn(s_hi, __fsub_rn(sum, bv)), __fsub_rn(p_hi, bv));
  s_hi = sum;
  s_lo = __fadd_rn(s_lo, __fadd_rn(e2, p_lo));
}

__global__ void __launch_bounds__(kThreads, 1)
    gram_lap_high_sym_kernel(const __grid_constant__ CUtensorMap tm_h, const __grid_constant__ CUtensorMap tm_l,
                             const float2* __restrict__ vhl, const float2* __restrict__ table,
                             const int4* __restrict__ units, double* __restrict__ acc, int p, int G, int one,
                             int* __restrict__ err) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int tile_elems = p * kTile;
  int32_t* HI = reinterpret_cast<int32_t*>(smem_raw);
  float* LI = reinterpret_cast<float*>(HI + tile_elems);
  int32_t* HJ[2];
  float* LJ[2];
  HJ[0] = reinterpret_cast<int32_t*>(LI + tile_elems);
  LJ[0] = reinterpret_cast<float*>(HJ[0] + tile_elems);
  HJ[1] = reinterpret_cast<int32_t*>(LJ[0] + tile_elems);
  LJ[1] = reinterpret_cast<float*>(HJ[1] + tile_elems);
  float2* tab = reinterpret_cast<float2*>(LJ[1] + tile_elems);
  double* colred = reinterpret_cast<double*>(tab + (1 << kTBs));  // 2 x 4 x 128
  double* rowred = colred + 2 * 4 * kTile;                        // 2 x 128
  uint64_t* bars = reinterpret_cast<uint64_t*>(rowred + 2 * kTile);

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int ty = (warp >> 1) * 4 + (lane >> 3);
  const int tx = (warp & 1) * 8 + (lane & 7);
  const int4 unit = units[blockIdx.x];
  const int row0 = unit.x * kTile;
  const int jt0 = unit.y, jt1 = unit.z;
  const uint32_t bytes = (uint32_t)tile_elems * 4u;

  for (int i = tid; i < (1 << kTBs); i += kThreads) tab[i] = table[i];
  if (tid == 0) {
    mbar_init(&bars[0], 1);
    mbar_init(&bars[1], 1);
    mbar_init(&bars[2], 1);
    fence_mbar_init();
  }
  __syncthreads();
  if (tid == 0) {
    mbar_arrive_expect_tx(&bars[0], 2 * bytes);
    tma_load_2d(HI, &tm_h, row0, 0, &bars[0]);
    tma_load_2d(LI, &tm_l, row0, 0, &bars[0]);
    mbar_arrive_expect_tx(&bars[1], 2 * bytes);
    tma_load_2d(HJ[0], &tm_h, jt0 * kTile, 0, &bars[1]);
    tma_load_2d(LJ[0], &tm_l, jt0 * kTile, 0, &bars[1]);
  }
  float vah[8], val[8], s_hi[8], s_lo[8];
#pragma unroll
  for (int a = 0; a < 8; ++a) {
    const float2 w = __ldg(vhl + row0 + ty * 8 + a);
    vah[a] = w.x;
    val[a] = w.y;
    s_hi[a] = s_lo[a] = 0.f;
  }
  const float scaleG = __int_as_float((127 - G) << 23);
  const int mone = -one, two = one + one;
  const int shift_f = G - kTBs;
  const int mask_f = (1 << kTBs) - 1;
  const int mask_r = (1 << shift_f) - 1;
  if (!mbar_wait_bounded(&bars[0], 0, err)) return;

  for (int t = jt0; t < jt1; ++t) {
    const int q = t - jt0;
    const int s = q & 1;
    if (tid == 0 && t + 1 < jt1) {
      const int ns = (q + 1) & 1;
      mbar_arrive_expect_tx(&bars[1 + ns], 2 * bytes);
      tma_load_2d(HJ[ns], &tm_h, (t + 1) * kTile, 0, &bars[1 + ns]);
      tma_load_2d(LJ[ns], &tm_l, (t + 1) * kTile, 0, &bars[1 + ns]);
    }
    const int col0 = t * kTile + tx * 8;
    float vbh[8], vbl[8];
#pragma unroll
    for (int b = 0; b < 8; ++b) {
      const float2 w = __ldg(vhl + col0 + b);
      vbh[b] = w.x;
      vbl[b] = w.y;
    }
    if (!mbar_wait_bounded(&bars[1 + s], (uint32_t)((q >> 1) & 1), err)) return;
    const int32_t* HJs = HJ[s];
    const float* LJs = LJ[s];

    int A[8][8];
    float Lo[8][8];
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
      for (int b = 0; b < 8; ++b) {
        A[a][b] = 0;
        Lo[a][b] = 0.f;
      }
    for (int k = 0; k < p; ++k) {
      const int4 h0 = *reinterpret_cast<const int4*>(HI + k * kTile + ty * 8);
      const int4 h1 = *reinterpret_cast<const int4*>(HI + k * kTile + ty * 8 + 4);
      const float4 l0 = *reinterpret_cast<const float4*>(LI + k * kTile + ty * 8);
      const float4 l1 = *reinterpret_cast<const float4*>(LI + k * kTile + ty * 8 + 4);
      const int4 g0 = *reinterpret_cast<const int4*>(HJs + k * kTile + tx * 8);
      const int4 g1 = *reinterpret_cast<const int4*>(HJs + k * kTile + tx * 8 + 4);
      const float4 m0 = *reinterpret_cast<const float4*>(LJs + k * kTile + tx * 8);
      const float4 m1 = *reinterpret_cast<const float4*>(LJs + k * kTile + tx * 8 + 4);
      const int ha[8] = {h0.x, h0.y, h0.z, h0.w, h1.x, h1.y, h1.z, h1.w};
      const float la[8] = {l0.x, l0.y, l0.z, l0.w, l1.x, l1.y, l1.z, l1.w};
      const int hb[8] = {g0.x, g0.y, g0.z, g0.w, g1.x, g1.y, g1.z, g1.w};
      const float lb[8] = {m0.x, m0.y, m0.z, m0.w, m1.x, m1.y, m1.z, m1.w};
      // Integer adds are written as multiply-adds by the run-time constant `one`
      // (= 1) so that they issue on the FMA pipe, which the float part leaves
      // mostly idle, instead of the integer ALU pipe (the bottleneck otherwise).
#pragma unroll
      for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int b = 0; b < 8; ++b) {
          const int dH = hb[b] * mone + ha[a];
          A[a][b] = abs(dH) * one + A[a][b];
          const float dl = la[a] - lb[b];
          const int dlb = __float_as_int(dl);
          const int key = dH * two + (dlb >> 31);
          Lo[a][b] += __int_as_float(dlb ^ (key & (int)0x80000000));
        }
    }
    // Entries as double-float, in place of the distance registers.
    float Kh[8][8], Kl[8][8];
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
      for (int b = 0; b < 8; ++b) df_exp2_neg(A[a][b], Lo[a][b], G, shift_f, mask_f, mask_r, scaleG, tab, Kh[a][b], Kl[a][b]);
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
      for (int b = 0; b < 8; ++b) df_acc(s_hi[a], s_lo[a], Kh[a][b], Kl[a][b], vbh[b], vbl[b]);

    const bool offdiag = (t != unit.x);
    double* cr = colred + s * (4 * kTile);
    if (offdiag) {
#pragma unroll
      for (int b = 0; b < 8; ++b) {
        float c_hi = 0.f, c_lo = 0.f;
#pragma unroll
        for (int a = 0; a < 8; ++a) df_acc(c_hi, c_lo, Kh[a][b], Kl[a][b], vah[a], val[a]);
        double c = (double)c_hi + (double)c_lo;
        c += __shfl_xor_sync(0xffffffffu, c, 8);
        c += __shfl_xor_sync(0xffffffffu, c, 16);
        if ((lane >> 3) == 0) cr[(warp >> 1) * kTile + tx * 8 + b] = c;
      }
    }
    __syncthreads();
    if (offdiag && tid < kTile) atomicAdd(acc + t * kTile + tid, cr[tid] + cr[kTile + tid] + cr[2 * kTile + tid] +
                                                                     cr[3 * kTile + tid]);
  }

#pragma unroll
  for (int a = 0; a < 8; ++a) {
    double v = (double)s_hi[a] + (double)s_lo[a];
    v += __shfl_xor_sync(0xffffffffu, v, 1);
    v += __shfl_xor_sync(0xffffffffu, v, 2);
    v += __shfl_xor_sync(0xffffffffu, v, 4);
    if ((lane & 7) == 0) rowred[(warp & 1) * kTile + ty * 8 + a] = v;
  }
  __syncthreads();
  if (tid < kTile) atomicAdd(acc + row0 + tid, rowred[tid] + rowred[kTile + tid]);
}

// v (FP64, n) -> (hi, lo) floats [ldn] zero padded; acc [ldn] zeroed.
__global__ void high_sym_prep_kernel(const double* __restrict__ v, float2* __restrict__ vhl, double* __restrict__ acc,
                                     int64_t n, int64_t ldn) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < ldn; i += (int64_t)gridDim.x * blockDim.x) {
    const double x = i < n ? v[i] : 0.0;
    const float hi = (float)x;
    vhl[i] = make_float2(hi, (float)(x - (double)hi));
    acc[i] = 0.0;
  }
}

__global__ void high_sym_copy_kernel(const double* __restrict__ acc, double* __restrict__ out, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = acc[i];
}

static size_t high_sym_smem(int p) {
  return (size_t)6 * p * kTile * 4 + (size_t)(1 << kTBs) * sizeof(float2) + (size_t)(2 * 4 + 2) * kTile * sizeof(double) +
         4 * sizeof(uint64_t);
}

cudaError_t gram_high_sym(Handle* h, const double* V, double* U, cudaStream_t st) {
  cudaError_t e = sym_units_ensure(h);
  if (e != cudaSuccess) return e;
  const size_t need = (size_t)h->ldn * (sizeof(float2) + sizeof(double));
  if (h->v32_cap < need) {
    dev_free(h, h->v32);
    h->v32 = (float*)dev_alloc(h, need);
    h->v32_cap = h->v32 ? need : 0;
    if (!h->v32) return cudaErrorMemoryAllocation;
  }
  float2* vhl = reinterpret_cast<float2*>(h->v32);
  double* acc = reinterpret_cast<double*>(vhl + h->ldn);
  high_sym_prep_kernel<<<grid_for(h->ldn), 256, 0, st>>>(V, vhl, acc, h->n, h->ldn);
  h->launches++;
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  const size_t smem = high_sym_smem((int)h->p);
  e = cudaFuncSetAttribute(gram_lap_high_sym_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  prof_mark(h, 1, true, st);
  gram_lap_high_sym_kernel<<<h->sym_nunits, kThreads, smem, st>>>(h->tm_hq, h->tm_hl, vhl, h->exp_table,
                                                                  h->sym_units, acc, (int)h->p, h->grid_G, 1,
                                                                  h->err_flag);
  prof_mark(h, 1, false, st);
  h->launches++;
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  high_sym_copy_kernel<<<grid_for(h->n), 256, 0, st>>>(acc, U, h->n);
  h->launches++;
  return cudaGetLastError();
}

}  // namespace kqr
