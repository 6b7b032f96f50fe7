// Batched multi-right-hand-side RBF Gram products U_b = K_b V_b over B
// independent problems of different sizes, for fitting a grid of (tau, lambda)
// pairs on many data sets at once: every pair's solver needs products with
// the same K_b (Sec. 3: the Newton and ADMM systems all multiply by K), so a
// block of up to 64 right-hand sides shares each Gram tile.
//
// Both contractions run on the tcgen05 tensor cores (kind::tf32, FP32
// accumulation in tensor memory):
//   S = XS_I XS_J^T        (128 x 64 tile, K = p, from TMA tiles, 128-byte swizzle)
//   P = exp2(2 S - n_i - n_j) = K_IJ   (epilogue warps: TMEM -> registers -> TMEM, or
//                                        shared memory with KQR_BATCH_P_IN_SMEM)
//   U_I += P V_J           (128 x 64 accumulator, K = 64 Gram columns)
// with XS = sqrt(gamma log2 e)(x - mean_b) rounded to TF32 and n = |XS|^2 of
// the rounded rows (so the tile is the RBF kernel at those rows, and stays
// positive semidefinite), P rounded to TF32 (nearest) and V rounded to TF32.
//
// Work item = (problem, 128-row tile); its 64-column steps stream X_J and V_J
// through TMA rings of 4 and 5 stages.  Items are sorted by length and dealt
// round-robin to one persistent CTA per SM.  Warp roles (320 threads): warp 0
// issues TMA copies, warp 1 owns tensor memory and issues the MMAs, warps 2-9
// are the epilogue in two groups of four that take alternate steps (thread =
// TMEM lane = row), so two tiles are exponentiated at once.  Tensor memory: four S buffers and two U accumulators (64 columns
// each); the first MMAs run two steps ahead of the second ones, so the epilogue
// finds its next S tile computed, and the read-out of item i overlaps item i + 1.
// Every wait is bounded; a timeout sets the error flag and an abort flag that
// ends every role's loop, after which the CTA drains its copies and MMAs and
// frees its tensor memory.
#include <algorithm>
#include <cmath>
#include <vector>

#include "kqr_internal.h"
#include "ptx.cuh"

namespace kqr {

namespace {

constexpr int kBM = 128;      // rows per work item (TMEM lanes)
constexpr int kBN = 64;       // Gram columns per step = K of the second MMA
constexpr int kBR = 64;       // right-hand sides = N of the second MMA
constexpr int kXStages = 4;                 // X_J ring (released after the first MMA)
constexpr int kVStages = 5;                 // V_J ring (released after the second MMA)
constexpr int kSBufs = 4;                   // S tiles in tensor memory
constexpr int kLookahead = 2;               // first MMAs issued ahead of the second ones
constexpr int kEpiWarps = 8;                // two groups of four, alternate steps
constexpr int kBatchThreads = 64 + 32 * kEpiWarps;
constexpr uint32_t kXIBytes = kBM * 128;    // 128 rows x 128 B (32 TF32 features, zero padded)
constexpr uint32_t kXJBytes = kBN * 128;    // 64 rows x 128 B
constexpr uint32_t kVAtom = kBR * 128;      // 64 right-hand sides x 32 columns
constexpr uint32_t kVBytes = 2 * kVAtom;      // bytes the TMA copies of V_J bring
constexpr uint32_t kNrmBytes = kBN * 4;       // the 64 column norms of the step (bulk copy)
constexpr uint32_t kVStride = kVBytes + 1024; // V_J atoms, then the norms (keeps 1024-byte alignment)
constexpr uint32_t kPAtom = kBM * 128;      // 128 rows x 32 columns
constexpr uint32_t kPBytes = 2 * kPAtom;
constexpr uint32_t kOffXI = 0;
constexpr uint32_t kOffXJ = kOffXI + 2 * kXIBytes;
constexpr uint32_t kOffV = kOffXJ + kXStages * kXJBytes;
constexpr uint32_t kOffP = kOffV + kVStages * kVStride;
constexpr uint32_t kOffBar = kOffP + 2 * kPBytes;
constexpr int kNumBars = 2 + 2 + 2 * kXStages + 2 * kVStages + 2 * kSBufs + 2 + 2 + 2 + 2 + 1;
constexpr size_t kBatchSmem = 1024 + kOffBar + kNumBars * 8 + 16;
constexpr uint32_t kUCol = 64 * kSBufs;     // first TMEM column of the U accumulators
constexpr uint32_t kPCol = kUCol + 128;     // first TMEM column of the P tiles (P kept in tensor memory)

__device__ __forceinline__ void tmem_alloc_b(uint32_t* dst, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst)), "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tmem_relinquish_b() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc_b(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

// D[tmem] (+)= A[tmem] B[smem]^T, tf32, A held in tensor memory (row i in lane i, K along columns).
__device__ __forceinline__ void mma_tf32_ta(uint32_t d_tmem, uint32_t a_tmem, uint64_t bdesc, uint32_t idesc,
                                            uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n\t}" ::"r"(d_tmem),
      "r"(a_tmem), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

// Issue a load of 32 consecutive 32-bit columns of this thread's TMEM lane (no wait).
__device__ __forceinline__ void tmem_ld32_nowait(uint32_t taddr, uint32_t* r) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// Issue a store of 32 consecutive 32-bit columns of this thread's TMEM lane (no wait).
__device__ __forceinline__ void tmem_st32_nowait(uint32_t taddr, const uint32_t* v) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], "
      "{%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16, "
      "%17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31, %32};" ::"r"(taddr),
      "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]), "r"(v[8]),
      "r"(v[9]), "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]), "r"(v[15]), "r"(v[16]),
      "r"(v[17]), "r"(v[18]), "r"(v[19]), "r"(v[20]), "r"(v[21]), "r"(v[22]), "r"(v[23]), "r"(v[24]),
      "r"(v[25]), "r"(v[26]), "r"(v[27]), "r"(v[28]), "r"(v[29]), "r"(v[30]), "r"(v[31])
      : "memory");
}

// Untiled bulk copy global -> shared (16-byte aligned addresses, size a multiple of 16).
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(reinterpret_cast<uint64_t>(src)), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void tmem_load32(uint32_t taddr, float* v) {
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

// K-major operand in the canonical 128-byte swizzled layout (8-row groups 1024 B apart).
__device__ __forceinline__ uint64_t desc_sw128(uint32_t saddr) {
  uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)(1024 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}

__device__ __forceinline__ uint32_t tf32_rna(float x) {
  uint32_t h;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(h) : "f"(x));
  return h;
}

// Bounded wait that also gives up as soon as another role has aborted.
__device__ __forceinline__ bool bwait(uint64_t* bar, uint32_t parity, volatile int* abort_flag, int* err) {
  for (uint32_t i = 0; i < (1u << 22); ++i) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((i & 255u) == 255u && *abort_flag) return false;
  }
  *abort_flag = 1;
  atomicExch(err, 1);
  return false;
}

// Drain wait: bounded, ignores the abort flag.
__device__ __forceinline__ void dwait(uint64_t* bar, uint32_t parity) {
  for (uint32_t i = 0; i < (1u << 22); ++i)
    if (mbar_try_wait(bar, parity)) return;
}

struct MmaStep {
  int stage, ub, item_seq, first, last;
};

}  // namespace

// items[i] = {row0 (padded row of the tile), col0 (padded first row of its problem),
//             nt (64-column steps), nvalid (rows < n_b in the tile)}; out0[i] = output row of row0.
template <bool PT>
__global__ void __launch_bounds__(kBatchThreads, 1)
    batch_kv_kernel(const __grid_constant__ CUtensorMap tm_xi, const __grid_constant__ CUtensorMap tm_xj,
                    const __grid_constant__ CUtensorMap tm_v, const float* __restrict__ nrm,
                    const int4* __restrict__ items, const int* __restrict__ out0, int n_items, int ksteps,
                    double* __restrict__ out, int m, int* __restrict__ err) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* base = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                                         ~static_cast<uintptr_t>(1023));
  const uint32_t sbase = smem_u32(base);
  uint64_t* bars = reinterpret_cast<uint64_t*>(base + kOffBar);
  uint64_t* xi_full = bars;
  uint64_t* xi_empty = bars + 2;
  uint64_t* xl_full = bars + 4;
  uint64_t* xl_empty = xl_full + kXStages;
  uint64_t* vl_full = xl_empty + kXStages;
  uint64_t* vl_empty = vl_full + kVStages;
  uint64_t* s_full = vl_empty + kVStages;
  uint64_t* s_empty = s_full + kSBufs;
  uint64_t* p_full = s_empty + kSBufs;
  uint64_t* p_empty = p_full + 2;
  uint64_t* u_full = p_empty + 2;
  uint64_t* u_empty = u_full + 2;
  uint64_t* drain = u_empty + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + kNumBars);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (warp == 1) {
    tmem_alloc_b(tmem_slot, 512);
    tmem_relinquish_b();
  }
  if (tid == 0) {
    for (int i = 0; i < 2; ++i) {
      mbar_init(&xi_full[i], 1);
      mbar_init(&xi_empty[i], 1);
      mbar_init(&p_full[i], kEpiWarps / 2);
      mbar_init(&p_empty[i], 1);
      mbar_init(&u_full[i], 1);
      mbar_init(&u_empty[i], kEpiWarps / 2);
    }
    for (int i = 0; i < kSBufs; ++i) {
      mbar_init(&s_full[i], 1);
      mbar_init(&s_empty[i], kEpiWarps / 2);
    }
    for (int i = 0; i < kXStages; ++i) {
      mbar_init(&xl_full[i], 1);
      mbar_init(&xl_empty[i], 1);
    }
    for (int i = 0; i < kVStages; ++i) {
      mbar_init(&vl_full[i], 1);
      mbar_init(&vl_empty[i], 1);
    }
    mbar_init(drain, 1);
    *abort_flag = 0;
    fence_mbar_init();
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tmem_slot;
  // kind::tf32, FP32 accumulate, A and B K-major, M = 128, N = 64 (both MMAs)
  const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((64u >> 3) << 17) | ((128u >> 4) << 24);

  if (warp == 0) {
    // ---- TMA producer ----
    if (lane == 0) {
      int q = 0, seq = 0;
      bool ok = true;
      for (int it = blockIdx.x; it < n_items && ok; it += gridDim.x) {
        const int4 I = items[it];
        const int xb = seq & 1;
        if (!bwait(&xi_empty[xb], ((seq >> 1) & 1) ^ 1, abort_flag, err)) break;
        mbar_arrive_expect_tx(&xi_full[xb], kXIBytes);
        tma_load_2d(base + kOffXI + xb * kXIBytes, &tm_xi, 0, I.x, &xi_full[xb]);
        ++seq;
        for (int j = 0; j < I.z; ++j) {
          const int xs = q % kXStages, vs = q % kVStages;
          const int c0 = I.y + j * kBN;
          if (!bwait(&xl_empty[xs], ((q / kXStages) & 1) ^ 1, abort_flag, err)) {
            ok = false;
            break;
          }
          mbar_arrive_expect_tx(&xl_full[xs], kXJBytes);
          tma_load_2d(base + kOffXJ + xs * kXJBytes, &tm_xj, 0, c0, &xl_full[xs]);
          if (!bwait(&vl_empty[vs], ((q / kVStages) & 1) ^ 1, abort_flag, err)) {
            ok = false;
            ++q;                         // the X_J copy of this step is in flight
            break;
          }
          mbar_arrive_expect_tx(&vl_full[vs], kVBytes + kNrmBytes);
          tma_load_2d(base + kOffV + vs * kVStride, &tm_v, c0, 0, &vl_full[vs]);
          tma_load_2d(base + kOffV + vs * kVStride + kVAtom, &tm_v, c0 + 32, 0, &vl_full[vs]);
          bulk_load(base + kOffV + vs * kVStride + kVBytes, nrm + c0, kNrmBytes, &vl_full[vs]);
          ++q;
        }
      }
      // Drain: every copy this thread issued has landed before the CTA exits.
      for (int k = (seq > 2 ? seq - 2 : 0); k < seq; ++k) dwait(&xi_full[k & 1], (k >> 1) & 1);
      for (int k = (q > kXStages ? q - kXStages : 0); k < q; ++k) dwait(&xl_full[k % kXStages], (k / kXStages) & 1);
      for (int k = (q > kVStages ? q - kVStages : 0); k < q; ++k) dwait(&vl_full[k % kVStages], (k / kVStages) & 1);
    }
  } else if (warp == 1) {
    // ---- MMA issuer: first MMAs run kLookahead steps ahead of the second ones ----
    if (lane == 0) {
      int q = 0, q2 = 0, seq = 0;
      MmaStep rec[kSBufs];
      bool ok = true;
      auto second = [&](const MmaStep& ps, int qq) -> bool {
        const int pb = qq & 1;
        if (!bwait(&p_full[pb], (qq >> 1) & 1, abort_flag, err)) return false;
        if (!bwait(&vl_full[ps.stage], (qq / kVStages) & 1, abort_flag, err)) return false;
        if (ps.first && !bwait(&u_empty[ps.ub], ((ps.item_seq >> 1) & 1) ^ 1, abort_flag, err)) return false;
        fence_after();
        const uint32_t d = tmem + kUCol + (uint32_t)(ps.ub * 64);
        const uint32_t pa = sbase + kOffP + pb * kPBytes;
        const uint32_t va = sbase + kOffV + ps.stage * kVStride;
#pragma unroll
        for (int k = 0; k < kBN / 8; ++k) {
          const uint32_t ka = (uint32_t)(k >> 2), kb = (uint32_t)(k & 3) * 32u;
          if (PT)
            mma_tf32_ta(d, tmem + kPCol + (uint32_t)(pb * 64 + k * 8), desc_sw128(va + ka * kVAtom + kb), idesc,
                        (ps.first && k == 0) ? 0u : 1u);
          else
            mma_tf32(d, desc_sw128(pa + ka * kPAtom + kb), desc_sw128(va + ka * kVAtom + kb), idesc,
                     (ps.first && k == 0) ? 0u : 1u);
        }
        mma_commit(&p_empty[pb]);
        mma_commit(&vl_empty[ps.stage]);
        if (ps.last) mma_commit(&u_full[ps.ub]);
        return true;
      };
      for (int it = blockIdx.x; it < n_items && ok; it += gridDim.x, ++seq) {
        const int4 I = items[it];
        const int xb = seq & 1;
        if (!bwait(&xi_full[xb], (seq >> 1) & 1, abort_flag, err)) {
          ok = false;
          break;
        }
        const uint32_t xa = sbase + kOffXI + xb * kXIBytes;
        for (int j = 0; j < I.z; ++j) {
          const int xs = q % kXStages, sb = q % kSBufs;
          if (!bwait(&xl_full[xs], (q / kXStages) & 1, abort_flag, err) ||
              !bwait(&s_empty[sb], ((q / kSBufs) & 1) ^ 1, abort_flag, err)) {
            ok = false;
            break;
          }
          fence_after();
          const uint32_t ja = sbase + kOffXJ + xs * kXJBytes;
          const uint32_t d = tmem + (uint32_t)(sb * 64);
          for (int k = 0; k < ksteps; ++k)
            mma_tf32(d, desc_sw128(xa + (uint32_t)k * 32u), desc_sw128(ja + (uint32_t)k * 32u), idesc, k > 0 ? 1u : 0u);
          mma_commit(&s_full[sb]);
          mma_commit(&xl_empty[xs]);
          if (j == I.z - 1) mma_commit(&xi_empty[xb]);
          rec[sb] = {q % kVStages, seq & 1, seq, j == 0 ? 1 : 0, j == I.z - 1 ? 1 : 0};
          ++q;
          while (ok && q2 < q - kLookahead) {
            if (!second(rec[q2 % kSBufs], q2)) ok = false;
            ++q2;
          }
        }
      }
      while (ok && q2 < q) {
        if (!second(rec[q2 % kSBufs], q2)) ok = false;
        ++q2;
      }
      // Drain: all MMAs issued by this thread have completed.
      mma_commit(drain);
      dwait(drain, 0);
    }
  } else {
    // ---- epilogue: two groups of four warps take alternate steps (group g the steps
    // q with q mod 2 = g), so two Gram tiles are exponentiated at once; in a group,
    // thread = TMEM lane = row, and each warp covers all 64 columns in two halves.
    const int lg = warp & 3;                  // TMEM lane group this warp may access
    const int grp = (warp - 2) >> 2;
    const int r = lg * 32 + lane;
    const uint32_t lane_off = (uint32_t)(lg * 32) << 16;
    int q = 0, seq = 0;
    bool ok = true;
    for (int it = blockIdx.x; it < n_items && ok; it += gridDim.x, ++seq) {
      const int4 I = items[it];
      const float ni = __ldg(nrm + I.x + r);
      const int q_last = q + I.z - 1;
      for (int j = 0; j < I.z; ++j, ++q) {
        if ((q & 1) != grp) continue;
        const int sb = q % kSBufs, vs = q % kVStages, pb = q & 1;
        if (!bwait(&s_full[sb], (q / kSBufs) & 1, abort_flag, err) ||
            !bwait(&vl_full[vs], (q / kVStages) & 1, abort_flag, err) ||
            !bwait(&p_empty[pb], ((q >> 1) & 1) ^ 1, abort_flag, err)) {
          ok = false;
          break;
        }
        fence_after();
        // the step's column norms arrived with V_J (the stage stays until this step's second MMA)
        const float4* nj4 = reinterpret_cast<const float4*>(base + kOffV + vs * kVStride + kVBytes);
        // both 32-column halves of the S row in flight at once, one wait
        uint32_t graw[64];
        tmem_ld32_nowait(tmem + (uint32_t)(sb * 64) + lane_off, graw);
        tmem_ld32_nowait(tmem + (uint32_t)(sb * 64 + 32) + lane_off, graw + 32);
        tmem_wait_ld();
#pragma unroll
        for (int ch = 0; ch < 2; ++ch) {
          uint32_t e[32];
#pragma unroll
          for (int c4 = 0; c4 < 8; ++c4) {
            const float4 nn = nj4[ch * 8 + c4];
            const uint32_t* g = graw + ch * 32 + 4 * c4;
            e[4 * c4 + 0] = tf32_rna(ex2_approx(fmaf(2.f, __uint_as_float(g[0]), -(ni + nn.x))));
            e[4 * c4 + 1] = tf32_rna(ex2_approx(fmaf(2.f, __uint_as_float(g[1]), -(ni + nn.y))));
            e[4 * c4 + 2] = tf32_rna(ex2_approx(fmaf(2.f, __uint_as_float(g[2]), -(ni + nn.z))));
            e[4 * c4 + 3] = tf32_rna(ex2_approx(fmaf(2.f, __uint_as_float(g[3]), -(ni + nn.w))));
          }
          if (PT) {
            // P tile in tensor memory, lane = row, columns [32 ch, 32 ch + 32)
            tmem_st32_nowait(tmem + kPCol + (uint32_t)(pb * 64 + ch * 32) + lane_off, e);
          } else {
            // columns [32 ch, 32 ch + 32) are swizzle atom ch of the P tile in shared memory
            unsigned char* prow = base + kOffP + pb * kPBytes + ch * kPAtom + r * 128;
#pragma unroll
            for (int c = 0; c < 8; ++c)
              *reinterpret_cast<uint4*>(prow + ((c ^ (r & 7)) * 16)) =
                  make_uint4(e[4 * c], e[4 * c + 1], e[4 * c + 2], e[4 * c + 3]);
          }
        }
        if (PT) tmem_wait_st();
        fence_before();
        if (!PT) fence_async_smem();
        __syncwarp();
        if (lane == 0) {
          mbar_arrive(&s_empty[sb]);
          mbar_arrive(&p_full[pb]);
        }
      }
      if (!ok) break;
      if ((q_last & 1) != grp) continue;        // the other group reads this item's result
      const int ub = seq & 1;
      if (!bwait(&u_full[ub], (seq >> 1) & 1, abort_flag, err)) break;
      fence_after();
#pragma unroll 1
      for (int ch = 0; ch < 2; ++ch) {
        float u[32];
        tmem_load32(tmem + kUCol + (uint32_t)(ub * 64 + ch * 32) + lane_off, u);
        if (r < I.w) {
          double* o = out + (size_t)(out0[it] + r) * m + ch * 32;
          const int mc = m - ch * 32;
#pragma unroll
          for (int c = 0; c < 32; ++c)
            if (c < mc) o[c] = (double)u[c];
        }
      }
      fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&u_empty[ub]);
    }
  }
  fence_before();
  __syncthreads();
  fence_after();
  if (warp == 1) tmem_dealloc_b(tmem, 512);
}

// Row-major padded TF32 coordinates xt[R][32] and squared norms of the rounded rows.
__global__ void batch_prep_x_kernel(const double* __restrict__ X, const int64_t* __restrict__ off,
                                    const int64_t* __restrict__ roff, const double* __restrict__ mean,
                                    const double* __restrict__ scale, int B, int p, int64_t R,
                                    float* __restrict__ xt, float* __restrict__ nrm) {
  for (int64_t row = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; row < R; row += (int64_t)gridDim.x * blockDim.x) {
    int lo = 0, hi = B;   // last b with roff[b] <= row
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (roff[mid] <= row) lo = mid;
      else hi = mid;
    }
    const int b = lo;
    const int64_t local = row - roff[b];
    const int64_t nb = off[b + 1] - off[b];
    float s = 0.f;
    for (int k = 0; k < 32; ++k) {
      float v = 0.f;
      if (local < nb && k < p) {
        const double x = (X[(size_t)(off[b] + local) * p + k] - mean[(size_t)b * p + k]) * scale[b];
        v = __uint_as_float(tf32_rna((float)x));
      }
      xt[(size_t)row * 32 + k] = v;
      s = fmaf(v, v, s);
    }
    nrm[row] = s;
  }
}

// vt[c][row] = TF32(V[off_b + local][c]) for c < m and local < n_b, else 0 (64 x 64 tiles).
__global__ void batch_prep_v_kernel(const double* __restrict__ V, const int64_t* __restrict__ off,
                                    const int64_t* __restrict__ roff, int B, int m, int64_t R,
                                    float* __restrict__ vt) {
  __shared__ float tile[64][65];
  const int64_t r0 = (int64_t)blockIdx.x * 64;
  if (r0 >= R) return;
  int lo = 0, hi = B;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (roff[mid] <= r0) lo = mid;
    else hi = mid;
  }
  const int b = lo;
  const int64_t nb = off[b + 1] - off[b];
  for (int e = threadIdx.x; e < 64 * 64; e += blockDim.x) {
    const int rr = e >> 6, c = e & 63;
    const int64_t local = r0 + rr - roff[b];
    float v = 0.f;
    if (c < m && local < nb) v = __uint_as_float(tf32_rna((float)V[(size_t)(off[b] + local) * m + c]));
    tile[rr][c] = v;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < 64 * 64; e += blockDim.x) {
    const int c = e >> 6, rr = e & 63;
    vt[(size_t)c * R + r0 + rr] = tile[rr][c];
  }
}

bool make_tmap_2d_f32_sw128(CUtensorMap* tm, void* base, int64_t inner, int64_t outer, int64_t row_bytes,
                            int box_inner, int box_outer);

kqr_status batch_create(Handle* h, const double* X, const int64_t* offsets, int64_t B, int64_t p,
                        const double* gammas, int32_t flags) {
  if (!X || !offsets || !gammas) return fail(h, KQR_INVALID_ARG, "X, offsets and gammas must be non-null");
  if (B < 1 || B > (1 << 24)) return fail(h, KQR_INVALID_ARG, "B must be in [1, 2^24]");
  if (p < 1 || p > 32) return fail(h, KQR_INVALID_ARG, "batched products take p in [1, 32]");
  if (offsets[0] != 0) return fail(h, KQR_INVALID_ARG, "offsets[0] must be 0");
  for (int64_t b = 0; b < B; ++b) {
    if (offsets[b + 1] <= offsets[b]) return fail(h, KQR_INVALID_ARG, "every problem needs at least one row");
    if (!(gammas[b] > 0.0) || !std::isfinite(gammas[b])) return fail(h, KQR_INVALID_ARG, "gammas must be positive");
  }
  const int64_t N = offsets[B];
  if (N > ((int64_t)1 << 30)) return fail(h, KQR_INVALID_ARG, "too many rows in total");
  for (int64_t i = 0; i < N * p; ++i)
    if (!std::isfinite(X[i])) return fail(h, KQR_INVALID_ARG, "X has a non-finite entry");
  if (flags & ~KQR_BATCH_P_IN_SMEM) return fail(h, KQR_INVALID_ARG, "unknown batch flags");
  BatchData* bd = new BatchData();
  h->batch = bd;
  bd->p_in_smem = (flags & KQR_BATCH_P_IN_SMEM) != 0;
  bd->B = B;
  bd->p = p;
  bd->off.assign(offsets, offsets + B + 1);
  bd->roff.resize(B + 1);
  bd->roff[0] = 0;
  std::vector<double> mean((size_t)B * p, 0.0), scale(B);
  for (int64_t b = 0; b < B; ++b) {
    const int64_t nb = offsets[b + 1] - offsets[b];
    bd->roff[b + 1] = bd->roff[b] + (nb + kBM - 1) / kBM * kBM;
    for (int64_t i = offsets[b]; i < offsets[b + 1]; ++i)
      for (int64_t k = 0; k < p; ++k) mean[(size_t)b * p + k] += X[(size_t)i * p + k];
    for (int64_t k = 0; k < p; ++k) mean[(size_t)b * p + k] /= (double)nb;
    scale[b] = std::sqrt(gammas[b] / std::log(2.0));
  }
  const int64_t R = bd->roff[B];
  bd->R = R;
  // Work items, longest first, dealt round-robin to the persistent CTAs.
  struct It {
    int row0, col0, nt, nvalid, out0;
  };
  std::vector<It> its;
  for (int64_t b = 0; b < B; ++b) {
    const int64_t nb = offsets[b + 1] - offsets[b];
    const int nt = (int)((nb + kBN - 1) / kBN);
    for (int64_t i0 = 0; i0 < nb; i0 += kBM)
      its.push_back({(int)(bd->roff[b] + i0), (int)bd->roff[b], nt, (int)std::min<int64_t>(kBM, nb - i0),
                     (int)(offsets[b] + i0)});
  }
  std::stable_sort(its.begin(), its.end(), [](const It& a, const It& b) { return a.nt > b.nt; });
  bd->n_items = (int)its.size();
  std::vector<int> hitems((size_t)bd->n_items * 4), hout0(bd->n_items);
  for (int i = 0; i < bd->n_items; ++i) {
    hitems[4 * i] = its[i].row0;
    hitems[4 * i + 1] = its[i].col0;
    hitems[4 * i + 2] = its[i].nt;
    hitems[4 * i + 3] = its[i].nvalid;
    hout0[i] = its[i].out0;
  }
  double entries = 0.0;
  for (int64_t b = 0; b < B; ++b) {
    const double nb = (double)(offsets[b + 1] - offsets[b]);
    entries += nb * nb;
  }
  bd->entries = entries;
  cudaStream_t st = h->stream;
  bd->xt = (float*)dev_alloc(h, sizeof(float) * R * 32);
  bd->nrm = (float*)dev_alloc(h, sizeof(float) * R);
  bd->vt = (float*)dev_alloc(h, sizeof(float) * R * kBR);
  bd->items = (int*)dev_alloc(h, sizeof(int) * 4 * bd->n_items);
  bd->out0 = (int*)dev_alloc(h, sizeof(int) * bd->n_items);
  bd->d_off = (int64_t*)dev_alloc(h, sizeof(int64_t) * (B + 1));
  bd->d_roff = (int64_t*)dev_alloc(h, sizeof(int64_t) * (B + 1));
  double* Xd = (double*)dev_alloc(h, sizeof(double) * N * p);
  double* md = (double*)dev_alloc(h, sizeof(double) * (B * p + B));
  if (!bd->xt || !bd->nrm || !bd->vt || !bd->items || !bd->out0 || !bd->d_off || !bd->d_roff || !Xd || !md) {
    dev_free(h, Xd);
    dev_free(h, md);
    return fail(h, KQR_OOM, "batch buffers");
  }
  cudaError_t e;
  if ((e = cudaMemcpyAsync(Xd, X, sizeof(double) * N * p, cudaMemcpyHostToDevice, st)) != cudaSuccess ||
      (e = cudaMemcpyAsync(md, mean.data(), sizeof(double) * B * p, cudaMemcpyHostToDevice, st)) != cudaSuccess ||
      (e = cudaMemcpyAsync(md + B * p, scale.data(), sizeof(double) * B, cudaMemcpyHostToDevice, st)) !=
          cudaSuccess ||
      (e = cudaMemcpyAsync(bd->d_off, offsets, sizeof(int64_t) * (B + 1), cudaMemcpyHostToDevice, st)) !=
          cudaSuccess ||
      (e = cudaMemcpyAsync(bd->d_roff, bd->roff.data(), sizeof(int64_t) * (B + 1), cudaMemcpyHostToDevice, st)) !=
          cudaSuccess ||
      (e = cudaMemcpyAsync(bd->items, hitems.data(), sizeof(int) * hitems.size(), cudaMemcpyHostToDevice, st)) !=
          cudaSuccess ||
      (e = cudaMemcpyAsync(bd->out0, hout0.data(), sizeof(int) * hout0.size(), cudaMemcpyHostToDevice, st)) !=
          cudaSuccess) {
    dev_free(h, Xd);
    dev_free(h, md);
    return cuda_fail(h, e, "batch upload");
  }
  batch_prep_x_kernel<<<grid_for(R), 256, 0, st>>>(Xd, bd->d_off, bd->d_roff, md, md + B * p, (int)B, (int)p, R,
                                                   bd->xt, bd->nrm);
  h->launches++;
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  dev_free(h, Xd);
  dev_free(h, md);
  if (e != cudaSuccess) return cuda_fail(h, e, "batch layout");
  if (!make_tmap_2d_f32_sw128(&bd->tm_xi, bd->xt, 32, R, 128, 32, kBM) ||
      !make_tmap_2d_f32_sw128(&bd->tm_xj, bd->xt, 32, R, 128, 32, kBN) ||
      !make_tmap_2d_f32_sw128(&bd->tm_v, bd->vt, R, kBR, R * 4, 32, kBR))
    return fail(h, KQR_CUDA_ERROR, "tensor map encoding failed");
  return KQR_OK;
}

cudaError_t batch_kmatmul(Handle* h, const double* V, double* U, int m, cudaStream_t st) {
  BatchData* bd = h->batch;
  const int64_t R = bd->R;
  batch_prep_v_kernel<<<(unsigned)(R / 64), 256, 0, st>>>(V, bd->d_off, bd->d_roff, (int)bd->B, m, R, bd->vt);
  h->launches++;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  auto kern = bd->p_in_smem ? batch_kv_kernel<false> : batch_kv_kernel<true>;
  e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kBatchSmem);
  if (e != cudaSuccess) return e;
  const int grid = std::min(h->num_sms, bd->n_items);
  const int ksteps = (int)((bd->p + 7) / 8);
  prof_mark(h, 0, true, st);
  kern<<<grid, kBatchThreads, kBatchSmem, st>>>(bd->tm_xi, bd->tm_xj, bd->tm_v, bd->nrm,
                                              reinterpret_cast<const int4*>(bd->items), bd->out0, bd->n_items,
                                              ksteps, U, m, h->err_flag);
  prof_mark(h, 0, false, st);
  h->launches++;
  return cudaGetLastError();
}

void batch_free(Handle* h) {
  BatchData* bd = h->batch;
  if (!bd) return;
  void* bufs[] = {bd->xt, bd->nrm, bd->vt, bd->items, bd->out0, bd->d_off, bd->d_roff};
  for (void* b : bufs) dev_free(h, b);
  delete bd;
  h->batch = nullptr;
}

}  // namespace kqr
