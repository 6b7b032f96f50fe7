// FP64-class Gram products u = K v (gradients of eq. (2.3) and the Sec. 4
// KKT residual need K alpha to ~1e-13 relative: errors there are multiplied by
// 1/lambda).
//
// Laplacian, on the FP32/INT32 pipes (FP64 throughput of this part is a small
// fraction of FP32):
//   xs = gamma log2(e) (x - mean) = hq 2^-G + hl,  hq int32, |hl| <= 2^-(G+1) float,
//   G chosen per problem so that sum_k |hq_ik - hq_jk| < 2^31.
//   |xs_ik - xs_jk| = |dH 2^-G + dl| with dH = hq_ik - hq_jk (exact int) and
//   dl = hl_ik - hl_jk; since |dl| <= 2^-G, the sign of the difference is the
//   sign of dH when dH != 0 and the sign of dl otherwise.  So
//   E_ij = sum_k |xs_ik - xs_jk| = A 2^-G + Lo,  A = sum |dH| (exact int32),
//   Lo = sum sign * dl (FP32, |Lo| <= p 2^-G).
//   K_ij = 2^-E = 2^-floor * T[f] * exp(-r ln 2): T a 1024-entry double-float
//   table of 2^(-k/1024), r < 2^-10 handled by a degree-4 Taylor polynomial
//   whose two leading terms are kept in double-float (Tang's table method).
//   Row sums of K_ij v_j are double-float (TwoSum accumulation), then FP64.
// RBF: the same fixed-point scheme on squared differences (p <= kRbfEmuMaxP), else
// plain FP64 entries and sums.
#include <cmath>

#include "kqr_internal.h"
#include "ptx.cuh"

namespace kqr {

constexpr int kTB = kExpTableBits;
constexpr float kLn2Hi = 0.693147182464599609375f;          // float(ln 2)
constexpr float kLn2Lo = -1.904654323148236e-09f;          // ln 2 - kLn2Hi

__global__ void __launch_bounds__(kThreads, 1)
    gram_lap_high_kernel(const __grid_constant__ CUtensorMap tm_h, const __grid_constant__ CUtensorMap tm_l,
                         const float2* __restrict__ vhl, const float2* __restrict__ table, double* __restrict__ part,
                         int p, int ldn, int G, int tiles_per_split, int col_tiles, int* __restrict__ err) {
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
  double* red = reinterpret_cast<double*>(tab + (1 << kTB));  // 2 x 128 doubles
  uint64_t* bars = reinterpret_cast<uint64_t*>(red + 2 * kTile);

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int ty = (warp >> 1) * 4 + (lane >> 3);
  const int tx = (warp & 1) * 8 + (lane & 7);
  const int row0 = blockIdx.x * kTile;
  const int split = blockIdx.y;
  const int jt0 = split * tiles_per_split;
  const int jt1 = min(col_tiles, jt0 + tiles_per_split);
  const uint32_t bytes = (uint32_t)tile_elems * 4u;

  for (int i = tid; i < (1 << kTB); i += kThreads) tab[i] = table[i];
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
    if (jt0 < jt1) {
      mbar_arrive_expect_tx(&bars[1], 2 * bytes);
      tma_load_2d(HJ[0], &tm_h, jt0 * kTile, 0, &bars[1]);
      tma_load_2d(LJ[0], &tm_l, jt0 * kTile, 0, &bars[1]);
    }
  }
  float s_hi[8], s_lo[8];
#pragma unroll
  for (int a = 0; a < 8; ++a) s_hi[a] = s_lo[a] = 0.f;
  const float scaleG = __int_as_float((127 - G) << 23);   // 2^-G
  const int shift_f = G - kTB;
  const int mask_f = (1 << kTB) - 1;
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
    float vh[8], vl[8];
#pragma unroll
    for (int b = 0; b < 8; ++b) {
      const float2 w = __ldg(vhl + col0 + b);
      vh[b] = w.x;
      vl[b] = w.y;
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
#pragma unroll
      for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int b = 0; b < 8; ++b) {
          const int dH = ha[a] - hb[b];
          A[a][b] += abs(dH);
          const float dl = la[a] - lb[b];
          const int dlb = __float_as_int(dl);
          // key < 0 exactly when the true difference is negative: dH <= -1, or dH == 0 and dl < 0.
          const int key = (dH << 1) + (dlb >> 31);
          Lo[a][b] += __int_as_float(dlb ^ (key & (int)0x80000000));
        }
    }
    // exp2(-E) in double-float and accumulation of K_ij v_j.
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
      for (int b = 0; b < 8; ++b) {
        const int Ai = A[a][b];
        const int eint = Ai >> G;
        const int kidx = (Ai >> shift_f) & mask_f;
        const int rem = Ai & mask_r;                                   // < 2^(G - 10) <= 2^23
        const float rem_f = __fsub_rn(__int_as_float(rem | 0x4B000000), 8388608.f);  // exact
        const float ap = __fmul_rn(rem_f, scaleG);                     // exact (power of two)
        const float lo = Lo[a][b];
        // r = ap + lo, TwoSum
        const float r_hi = __fadd_rn(ap, lo);
        const float bb = __fsub_rn(r_hi, ap);
        const float r_lo = __fadd_rn(__fsub_rn(ap, __fsub_rn(r_hi, bb)), __fsub_rn(lo, bb));
        // x = r ln2 (double-float)
        const float x_hi = __fmul_rn(r_hi, kLn2Hi);
        float x_lo = fmaf(r_hi, kLn2Hi, -x_hi);
        x_lo = fmaf(r_hi, kLn2Lo, x_lo);
        x_lo = fmaf(r_lo, kLn2Hi, x_lo);
        // e^-x = 1 - x + x^2 (1/2 - x/6 + x^2/24)
        const float tail = __fmul_rn(__fmul_rn(x_hi, x_hi), fmaf(x_hi, fmaf(x_hi, 1.f / 24.f, -1.f / 6.f), 0.5f));
        const float P_hi = __fsub_rn(1.f, x_hi);
        const float P_lo = __fadd_rn(__fsub_rn(__fsub_rn(__fsub_rn(1.f, P_hi), x_hi), x_lo), tail);
        const float2 T = tab[kidx];
        float K_hi = __fmul_rn(T.x, P_hi);
        float K_lo = fmaf(T.x, P_hi, -K_hi);
        K_lo = fmaf(T.x, P_lo, K_lo);
        K_lo = fmaf(T.y, P_hi, K_lo);
        const float sc = (eint < 100) ? __int_as_float((127 - eint) << 23) : 0.f;
        K_hi = __fmul_rn(K_hi, sc);
        K_lo = __fmul_rn(K_lo, sc);
        // (s_hi, s_lo) += K v_j
        const float p_hi = __fmul_rn(K_hi, vh[b]);
        float p_lo = fmaf(K_hi, vh[b], -p_hi);
        p_lo = fmaf(K_hi, vl[b], p_lo);
        p_lo = fmaf(K_lo, vh[b], p_lo);
        const float sum = __fadd_rn(s_hi[a], p_hi);
        const float bv = __fsub_rn(sum, s_hi[a]);
        const float e2 = __fadd_rn(__fsub_rn(s_hi[a], __fsub_rn(sum, bv)), __fsub_rn(p_hi, bv));
        s_hi[a] = sum;
        s_lo[a] = __fadd_rn(s_lo[a], __fadd_rn(e2, p_lo));
      }
    __syncthreads();
  }

  // Reduce the 16 column groups of each row in FP64, write per-split partials.
  double r8[8];
#pragma unroll
  for (int a = 0; a < 8; ++a) {
    double v = (double)s_hi[a] + (double)s_lo[a];
    v += __shfl_xor_sync(0xffffffffu, v, 1);
    v += __shfl_xor_sync(0xffffffffu, v, 2);
    v += __shfl_xor_sync(0xffffffffu, v, 4);
    r8[a] = v;
  }
  __syncthreads();
  const int wc = warp & 1;
  if ((lane & 7) == 0) {
#pragma unroll
    for (int a = 0; a < 8; ++a) red[wc * kTile + ty * 8 + a] = r8[a];
  }
  __syncthreads();
  if (tid < kTile) part[(size_t)split * ldn + row0 + tid] = red[tid] + red[kTile + tid];
}

// RBF, FP64-class on the FP32/INT32 pipes (p <= kRbfEmuMaxP):
//   xs = sqrt(gamma log2 e)(x - mean) = hq 2^-G + hl as for the Laplacian, with G
//   chosen so that sum_k (hq_ik - hq_jk)^2 < 2^62.  With dH = hq_ik - hq_jk (exact
//   int), dl = hl_ik - hl_jk and dx = xs32_ik - xs32_jk (the FP32 coordinates),
//   (dH 2^-G + dl)^2 = dH^2 2^-2G + (2 (dH 2^-G + dl) - dl) dl, so
//   D_ij = sum_k (xs_ik - xs_jk)^2 = Q 2^-2G + W,  Q = sum dH^2 (exact int64),
//   W = sum (2 dx - dl) dl (FP32; replacing dH 2^-G + dl by dx costs
//   2 |dx| 2^-24 |dl| <= 2^-(G+22) |dx| per feature, far below D's FP64-class error).
//   K_ij = 2^-D by the same table method as the Laplacian, the sub-table part
//   r = (Q mod 2^(2G-10)) 2^-2G + W carried in double-float.
// Thread tile 8 rows x 4 columns (the int64 sums need the registers); a 128-column
// TMA tile is processed as two 64-column halves.
__global__ void __launch_bounds__(kThreads, 1)
    gram_rbf_emu_kernel(const __grid_constant__ CUtensorMap tm_h, const __grid_constant__ CUtensorMap tm_l,
                        const __grid_constant__ CUtensorMap tm_x, const float2* __restrict__ vhl,
                        const float2* __restrict__ table, double* __restrict__ part, int p, int ldn, int G,
                        int tiles_per_split, int col_tiles, int* __restrict__ err) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int tile_elems = p * kTile;
  int32_t* HI = reinterpret_cast<int32_t*>(smem_raw);
  float* LI = reinterpret_cast<float*>(HI + tile_elems);
  float* XI = LI + tile_elems;
  int32_t* HJ[2];
  float* LJ[2];
  float* XJ[2];
  HJ[0] = reinterpret_cast<int32_t*>(XI + tile_elems);
  LJ[0] = reinterpret_cast<float*>(HJ[0] + tile_elems);
  XJ[0] = LJ[0] + tile_elems;
  HJ[1] = reinterpret_cast<int32_t*>(XJ[0] + tile_elems);
  LJ[1] = reinterpret_cast<float*>(HJ[1] + tile_elems);
  XJ[1] = LJ[1] + tile_elems;
  float2* tab = reinterpret_cast<float2*>(XJ[1] + tile_elems);
  double* red = reinterpret_cast<double*>(tab + (1 << kTB));  // 2 x 128 doubles
  uint64_t* bars = reinterpret_cast<uint64_t*>(red + 2 * kTile);

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int ty = (warp >> 1) * 4 + (lane >> 3);
  const int tx = (warp & 1) * 8 + (lane & 7);
  const int row0 = blockIdx.x * kTile;
  const int split = blockIdx.y;
  const int jt0 = split * tiles_per_split;
  const int jt1 = min(col_tiles, jt0 + tiles_per_split);
  const uint32_t bytes = (uint32_t)tile_elems * 4u;

  for (int i = tid; i < (1 << kTB); i += kThreads) tab[i] = table[i];
  if (tid == 0) {
    mbar_init(&bars[0], 1);
    mbar_init(&bars[1], 1);
    mbar_init(&bars[2], 1);
    fence_mbar_init();
  }
  __syncthreads();
  if (tid == 0) {
    mbar_arrive_expect_tx(&bars[0], 3 * bytes);
    tma_load_2d(HI, &tm_h, row0, 0, &bars[0]);
    tma_load_2d(LI, &tm_l, row0, 0, &bars[0]);
    tma_load_2d(XI, &tm_x, row0, 0, &bars[0]);
    if (jt0 < jt1) {
      mbar_arrive_expect_tx(&bars[1], 3 * bytes);
      tma_load_2d(HJ[0], &tm_h, jt0 * kTile, 0, &bars[1]);
      tma_load_2d(LJ[0], &tm_l, jt0 * kTile, 0, &bars[1]);
      tma_load_2d(XJ[0], &tm_x, jt0 * kTile, 0, &bars[1]);
    }
  }
  float s_hi[8], s_lo[8];
#pragma unroll
  for (int a = 0; a < 8; ++a) s_hi[a] = s_lo[a] = 0.f;
  const int sh = 2 * G - kTB;                                   // bits below the table index
  const long long mask_r = (1LL << sh) - 1;
  const int mask_f = (1 << kTB) - 1;
  const float scaleA = __int_as_float((127 + 23 - 2 * G) << 23);  // 2^(23 - 2G)
  const float scaleB = __int_as_float((127 - 2 * G) << 23);       // 2^-2G

  if (!mbar_wait_bounded(&bars[0], 0, err)) return;

  for (int t = jt0; t < jt1; ++t) {
    const int q = t - jt0;
    const int s = q & 1;
    if (tid == 0 && t + 1 < jt1) {
      const int ns = (q + 1) & 1;
      mbar_arrive_expect_tx(&bars[1 + ns], 3 * bytes);
      tma_load_2d(HJ[ns], &tm_h, (t + 1) * kTile, 0, &bars[1 + ns]);
      tma_load_2d(LJ[ns], &tm_l, (t + 1) * kTile, 0, &bars[1 + ns]);
      tma_load_2d(XJ[ns], &tm_x, (t + 1) * kTile, 0, &bars[1 + ns]);
    }
    if (!mbar_wait_bounded(&bars[1 + s], (uint32_t)((q >> 1) & 1), err)) return;
    const int32_t* HJs = HJ[s];
    const float* LJs = LJ[s];
    const float* XJs = XJ[s];
#pragma unroll 1
    for (int half = 0; half < 2; ++half) {
      const int cj = half * 64 + tx * 4;             // column within the tile
      const int col0 = t * kTile + cj;
      float vh[4], vl[4];
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        const float2 w = __ldg(vhl + col0 + b);
        vh[b] = w.x;
        vl[b] = w.y;
      }
      long long Q[8][4];
      float W[8][4];
#pragma unroll
      for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          Q[a][b] = 0;
          W[a][b] = 0.f;
        }
      for (int k = 0; k < p; ++k) {
        const int4 h0 = *reinterpret_cast<const int4*>(HI + k * kTile + ty * 8);
        const int4 h1 = *reinterpret_cast<const int4*>(HI + k * kTile + ty * 8 + 4);
        const float4 l0 = *reinterpret_cast<const float4*>(LI + k * kTile + ty * 8);
        const float4 l1 = *reinterpret_cast<const float4*>(LI + k * kTile + ty * 8 + 4);
        const float4 x0 = *reinterpret_cast<const float4*>(XI + k * kTile + ty * 8);
        const float4 x1 = *reinterpret_cast<const float4*>(XI + k * kTile + ty * 8 + 4);
        const int4 g0 = *reinterpret_cast<const int4*>(HJs + k * kTile + cj);
        const float4 m0 = *reinterpret_cast<const float4*>(LJs + k * kTile + cj);
        const float4 y0 = *reinterpret_cast<const float4*>(XJs + k * kTile + cj);
        const int ha[8] = {h0.x, h0.y, h0.z, h0.w, h1.x, h1.y, h1.z, h1.w};
        const float la[8] = {l0.x, l0.y, l0.z, l0.w, l1.x, l1.y, l1.z, l1.w};
        const float xa[8] = {x0.x, x0.y, x0.z, x0.w, x1.x, x1.y, x1.z, x1.w};
        const int hb[4] = {g0.x, g0.y, g0.z, g0.w};
        const float lb[4] = {m0.x, m0.y, m0.z, m0.w};
        const float xb[4] = {y0.x, y0.y, y0.z, y0.w};
#pragma unroll
        for (int a = 0; a < 8; ++a)
#pragma unroll
          for (int b = 0; b < 4; ++b) {
            const int dH = ha[a] - hb[b];
            Q[a][b] += (long long)dH * (long long)dH;
            const float dl = la[a] - lb[b];
            const float dx = xa[a] - xb[b];
            W[a][b] = fmaf(fmaf(2.f, dx, -dl), dl, W[a][b]);
          }
      }
#pragma unroll
      for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          const long long Qv = Q[a][b];
          const long long qi = Qv >> (2 * G);
          const int eint = qi > 1000 ? 1000 : (int)qi;
          const int kidx = (int)(Qv >> sh) & mask_f;
          const long long rem = Qv & mask_r;                       // < 2^(2G - 10) <= 2^46
          const int ra = (int)(rem >> 23), rb = (int)(rem & 0x7FFFFF);
          const float pa = __fmul_rn(__fsub_rn(__int_as_float(ra | 0x4B000000), 8388608.f), scaleA);  // exact
          const float pb = __fmul_rn(__fsub_rn(__int_as_float(rb | 0x4B000000), 8388608.f), scaleB);  // exact
          // (t_hi, t_lo) = pa + pb exactly (TwoSum), then r = t + W
          const float t_hi = __fadd_rn(pa, pb);
          const float tb = __fsub_rn(t_hi, pa);
          const float t_lo = __fadd_rn(__fsub_rn(pa, __fsub_rn(t_hi, tb)), __fsub_rn(pb, tb));
          const float w = W[a][b];
          const float r_hi = __fadd_rn(t_hi, w);
          const float bb = __fsub_rn(r_hi, t_hi);
          const float r_lo = __fadd_rn(__fadd_rn(__fsub_rn(t_hi, __fsub_rn(r_hi, bb)), __fsub_rn(w, bb)), t_lo);
          // x = r ln2 (double-float)
          const float x_hi = __fmul_rn(r_hi, kLn2Hi);
          float x_lo = fmaf(r_hi, kLn2Hi, -x_hi);
          x_lo = fmaf(r_hi, kLn2Lo, x_lo);
          x_lo = fmaf(r_lo, kLn2Hi, x_lo);
          // e^-x = 1 - x + x^2 (1/2 - x/6 + x^2/24)
          const float tail = __fmul_rn(__fmul_rn(x_hi, x_hi), fmaf(x_hi, fmaf(x_hi, 1.f / 24.f, -1.f / 6.f), 0.5f));
          const float P_hi = __fsub_rn(1.f, x_hi);
          const float P_lo = __fadd_rn(__fsub_rn(__fsub_rn(__fsub_rn(1.f, P_hi), x_hi), x_lo), tail);
          const float2 T = tab[kidx];
          float K_hi = __fmul_rn(T.x, P_hi);
          float K_lo = fmaf(T.x, P_hi, -K_hi);
          K_lo = fmaf(T.x, P_lo, K_lo);
          K_lo = fmaf(T.y, P_hi, K_lo);
          const float sc = (eint < 100) ? __int_as_float((127 - eint) << 23) : 0.f;
          K_hi = __fmul_rn(K_hi, sc);
          K_lo = __fmul_rn(K_lo, sc);
          const float p_hi = __fmul_rn(K_hi, vh[b]);
          float p_lo = fmaf(K_hi, vh[b], -p_hi);
          p_lo = fmaf(K_hi, vl[b], p_lo);
          p_lo = fmaf(K_lo, vh[b], p_lo);
          const float sum = __fadd_rn(s_hi[a], p_hi);
          const float bv = __fsub_rn(sum, s_hi[a]);
          const float e2 = __fadd_rn(__fsub_rn(s_hi[a], __fsub_rn(sum, bv)), __fsub_rn(p_hi, bv));
          s_hi[a] = sum;
          s_lo[a] = __fadd_rn(s_lo[a], __fadd_rn(e2, p_lo));
        }
    }
    __syncthreads();
  }

  double r8[8];
#pragma unroll
  for (int a = 0; a < 8; ++a) {
    double v = (double)s_hi[a] + (double)s_lo[a];
    v += __shfl_xor_sync(0xffffffffu, v, 1);
    v += __shfl_xor_sync(0xffffffffu, v, 2);
    v += __shfl_xor_sync(0xffffffffu, v, 4);
    r8[a] = v;
  }
  __syncthreads();
  const int wc = warp & 1;
  if ((lane & 7) == 0) {
#pragma unroll
    for (int a = 0; a < 8; ++a) red[wc * kTile + ty * 8 + a] = r8[a];
  }
  __syncthreads();
  if (tid < kTile) part[(size_t)split * ldn + row0 + tid] = red[tid] + red[kTile + tid];
}

static size_t rbf_emu_smem(int p) {
  return (size_t)9 * p * kTile * 4 + (size_t)(1 << kTB) * sizeof(float2) + 2 * kTile * sizeof(double) +
         4 * sizeof(uint64_t);
}

// RBF, FP64: entries exp(-gamma ||x_i - x_j||^2) from the centred FP64 copy.
__global__ void __launch_bounds__(kThreads, 1)
    gram_rbf_high_kernel(const double* __restrict__ xc, const double* __restrict__ v, double* __restrict__ part,
                         int p, int ldn, double gamma, int tiles_per_split, int col_tiles) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  double* XI = reinterpret_cast<double*>(smem_raw);
  double* XJ = XI + p * kTile;
  double* red = XJ + p * kTile;  // 2 x 128 doubles
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int ty = (warp >> 1) * 4 + (lane >> 3);
  const int tx = (warp & 1) * 8 + (lane & 7);
  const int row0 = blockIdx.x * kTile;
  const int split = blockIdx.y;
  const int jt0 = split * tiles_per_split;
  const int jt1 = min(col_tiles, jt0 + tiles_per_split);
  for (int i = tid; i < p * kTile; i += kThreads) XI[i] = xc[(size_t)(i / kTile) * ldn + row0 + (i % kTile)];
  double racc[8];
#pragma unroll
  for (int a = 0; a < 8; ++a) racc[a] = 0.0;
  for (int t = jt0; t < jt1; ++t) {
    __syncthreads();
    for (int i = tid; i < p * kTile; i += kThreads)
      XJ[i] = xc[(size_t)(i / kTile) * ldn + t * kTile + (i % kTile)];
    __syncthreads();
    double acc[8][8];
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
      for (int b = 0; b < 8; ++b) acc[a][b] = 0.0;
    for (int k = 0; k < p; ++k) {
      double xa[8], xb[8];
#pragma unroll
      for (int a = 0; a < 8; ++a) xa[a] = XI[k * kTile + ty * 8 + a];
#pragma unroll
      for (int b = 0; b < 8; ++b) xb[b] = XJ[k * kTile + tx * 8 + b];
#pragma unroll
      for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int b = 0; b < 8; ++b) {
          const double d = xa[a] - xb[b];
          acc[a][b] = fma(d, d, acc[a][b]);
        }
    }
    const int col0 = t * kTile + tx * 8;
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
      for (int b = 0; b < 8; ++b) racc[a] = fma(exp(-gamma * acc[a][b]), v[col0 + b], racc[a]);
  }
#pragma unroll
  for (int a = 0; a < 8; ++a) {
    double vv = racc[a];
    vv += __shfl_xor_sync(0xffffffffu, vv, 1);
    vv += __shfl_xor_sync(0xffffffffu, vv, 2);
    vv += __shfl_xor_sync(0xffffffffu, vv, 4);
    racc[a] = vv;
  }
  __syncthreads();
  const int wc = warp & 1;
  if ((lane & 7) == 0) {
#pragma unroll
    for (int a = 0; a < 8; ++a) red[wc * kTile + ty * 8 + a] = racc[a];
  }
  __syncthreads();
  if (tid < kTile) part[(size_t)split * ldn + row0 + tid] = red[tid] + red[kTile + tid];
}

// v (FP64, n) -> (hi, lo) floats [ldn], zero padded.
__global__ void split_hilo_kernel(const double* __restrict__ v, float2* __restrict__ out, int64_t n, int64_t ldn) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < ldn; i += (int64_t)gridDim.x * blockDim.x) {
    const double x = i < n ? v[i] : 0.0;
    const float hi = (float)x;
    out[i] = make_float2(hi, (float)(x - (double)hi));
  }
}

__global__ void pad_copy_kernel(const double* __restrict__ v, double* __restrict__ out, int64_t n, int64_t ldn) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < ldn; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = i < n ? v[i] : 0.0;
}

__global__ void sum_splits_kernel(const double* __restrict__ part, int splits, int64_t ldn, int64_t n,
                                  double* __restrict__ out, int stride) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int sp = 0; sp < splits; ++sp) s += part[(size_t)sp * ldn + i];
    out[i * stride] = s;
  }
}

__global__ void gather_col_kernel(const double* __restrict__ V, double* __restrict__ out, int64_t n, int m, int c) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = V[i * m + c];
}

static size_t lap_high_smem(int p) {
  return (size_t)6 * p * kTile * 4 + (size_t)(1 << kTB) * sizeof(float2) + 2 * kTile * sizeof(double) +
         4 * sizeof(uint64_t);
}

cudaError_t gram_high(Handle* h, const double* V, double* U, int m, cudaStream_t st) {
  if (m == 1 && h->kind == KQR_LAPLACIAN && h->opt.symmetric_gram) return gram_high_sym(h, V, U, st);
  const int row_tiles = (int)(h->ldn / kTile), col_tiles = row_tiles;
  const int target = 8 * h->num_sms;
  int s = (target + row_tiles - 1) / row_tiles;
  if (s < 1) s = 1;
  if (s > col_tiles) s = col_tiles;
  const int tps = (col_tiles + s - 1) / s;
  const int splits = (col_tiles + tps - 1) / tps;
  const size_t part_bytes = (size_t)splits * h->ldn * sizeof(double);
  if (h->part_cap < part_bytes) {
    dev_free(h, h->part);
    h->part = (float*)dev_alloc(h, part_bytes);
    h->part_cap = h->part ? part_bytes : 0;
    if (!h->part) return cudaErrorMemoryAllocation;
  }
  const size_t vbytes = (size_t)h->ldn * sizeof(double) * 2;
  if (h->v32_cap < vbytes) {
    dev_free(h, h->v32);
    h->v32 = (float*)dev_alloc(h, vbytes);
    h->v32_cap = h->v32 ? vbytes : 0;
    if (!h->v32) return cudaErrorMemoryAllocation;
  }
  double* part = reinterpret_cast<double*>(h->part);
  cudaError_t e = cudaSuccess;
  for (int c = 0; c < m; ++c) {
    // Column c of V, contiguous and padded: reuse the last solver slot as staging.
    const double* vcol = V;
    if (m > 1) {
      double* stage = vec(h, V_TMP2);
      gather_col_kernel<<<grid_for(h->n), 256, 0, st>>>(V, stage, h->n, m, c);
      h->launches++;
      vcol = stage;
    }
    if (h->kind == KQR_LAPLACIAN) {
      float2* vhl = reinterpret_cast<float2*>(h->v32);
      split_hilo_kernel<<<grid_for(h->ldn), 256, 0, st>>>(vcol, vhl, h->n, h->ldn);
      h->launches++;
      const size_t smem = lap_high_smem((int)h->p);
      e = cudaFuncSetAttribute(gram_lap_high_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
      prof_mark(h, 1, true, st);
      gram_lap_high_kernel<<<dim3(row_tiles, splits), kThreads, smem, st>>>(
          h->tm_hq, h->tm_hl, vhl, h->exp_table, part, (int)h->p, (int)h->ldn, h->grid_G, tps, col_tiles,
          h->err_flag);
      prof_mark(h, 1, false, st);
      h->launches++;
    } else if (h->hq) {
      float2* vhl = reinterpret_cast<float2*>(h->v32);
      split_hilo_kernel<<<grid_for(h->ldn), 256, 0, st>>>(vcol, vhl, h->n, h->ldn);
      h->launches++;
      const size_t smem = rbf_emu_smem((int)h->p);
      e = cudaFuncSetAttribute(gram_rbf_emu_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
      prof_mark(h, 1, true, st);
      gram_rbf_emu_kernel<<<dim3(row_tiles, splits), kThreads, smem, st>>>(
          h->tm_hq, h->tm_hl, h->tm_xs32, vhl, h->exp_table, part, (int)h->p, (int)h->ldn, h->grid_G, tps,
          col_tiles, h->err_flag);
      prof_mark(h, 1, false, st);
      h->launches++;
    } else {
      double* vpad = reinterpret_cast<double*>(h->v32);
      pad_copy_kernel<<<grid_for(h->ldn), 256, 0, st>>>(vcol, vpad, h->n, h->ldn);
      h->launches++;
      const size_t smem = ((size_t)2 * h->p * kTile + 2 * kTile) * sizeof(double);
      e = cudaFuncSetAttribute(gram_rbf_high_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
      prof_mark(h, 1, true, st);
      gram_rbf_high_kernel<<<dim3(row_tiles, splits), kThreads, smem, st>>>(h->xc64, vpad, part, (int)h->p,
                                                                           (int)h->ldn, h->gamma, tps, col_tiles);
      prof_mark(h, 1, false, st);
      h->launches++;
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    sum_splits_kernel<<<grid_for(h->n), 256, 0, st>>>(part, splits, h->ldn, h->n, U + c, m);
    h->launches++;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace kqr
