// extern "C" entry points of kqr.h and problem set-up.
#include <cmath>
#include <cstring>
#include <new>

#include "kqr_internal.h"

namespace kqr {

static Allocator g_alloc;

void* dev_alloc(Handle* h, size_t bytes) {
  if (bytes == 0) bytes = 16;
  if (h->alloc.alloc) return h->alloc.alloc(bytes, h->alloc.ctx);
  void* p = nullptr;
  return cudaMalloc(&p, bytes) == cudaSuccess ? p : nullptr;
}

void dev_free(Handle* h, void* p) {
  if (!p) return;
  if (h->alloc.free_fn) h->alloc.free_fn(p, h->alloc.ctx);
  else cudaFree(p);
}

kqr_status fail(Handle* h, kqr_status s, const std::string& msg) {
  if (h) h->err = msg;
  return s;
}

kqr_status cuda_fail(Handle* h, cudaError_t e, const char* what) {
  if (h) h->err = std::string(what) + ": " + cudaGetErrorString(e);
  return e == cudaErrorMemoryAllocation ? KQR_OOM : KQR_CUDA_ERROR;
}

cudaStream_t pick_stream(Handle* h, void* stream) { return stream ? (cudaStream_t)stream : h->stream; }

void prof_mark(Handle* h, int k, bool begin, cudaStream_t st) {
  if (!h->profile) return;
  std::vector<cudaEvent_t>& ev = h->prof_ev[k];
  if (begin && h->prof_used[k] + 2 > ev.size()) {
    for (int i = 0; i < 256; ++i) {
      cudaEvent_t e;
      if (cudaEventCreate(&e) != cudaSuccess) return;
      ev.push_back(e);
    }
  }
  if (h->prof_used[k] >= ev.size()) return;
  cudaEventRecord(ev[h->prof_used[k]], st);
  h->prof_used[k]++;
}

// ---- data layout kernels --------------------------------------------------------
// Per feature k: mean, min and max over the n rows of X (row-major n x p).
__global__ void colstats_kernel(const double* __restrict__ X, int64_t n, int p, double* __restrict__ stats) {
  const int k = blockIdx.x;
  double s = 0.0, lo = INFINITY, hi = -INFINITY;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    const double x = X[i * p + k];
    s += x;
    lo = fmin(lo, x);
    hi = fmax(hi, x);
  }
  __shared__ double ss[256], sl[256], sh[256];
  ss[threadIdx.x] = s;
  sl[threadIdx.x] = lo;
  sh[threadIdx.x] = hi;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) {
      ss[threadIdx.x] += ss[threadIdx.x + o];
      sl[threadIdx.x] = fmin(sl[threadIdx.x], sl[threadIdx.x + o]);
      sh[threadIdx.x] = fmax(sh[threadIdx.x], sh[threadIdx.x + o]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    stats[3 * k + 0] = ss[0] / (double)n;
    stats[3 * k + 1] = sl[0];
    stats[3 * k + 2] = sh[0];
  }
}

// Feature-major layouts of the centred data (padding rows i >= n are zero):
//   xc64 = x - mean; xs32 = float(scale * xc64); Laplacian fixed point hq, hl of scale * xc64.
__global__ void layout_kernel(const double* __restrict__ X, const double* __restrict__ stats, int64_t n, int64_t ldn,
                              int p, double scale, int fixed, int G, double* __restrict__ xc64, float* __restrict__ xs32,
                              int32_t* __restrict__ hq, float* __restrict__ hl) {
  const double twoG = ldexp(1.0, G), twomG = ldexp(1.0, -G);
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < ldn * p; e += (int64_t)gridDim.x * blockDim.x) {
    const int k = (int)(e / ldn);
    const int64_t i = e % ldn;
    const double x = i < n ? X[i * p + k] - stats[3 * k] : 0.0;
    xc64[e] = x;
    const double xs = scale * x;
    xs32[e] = (float)xs;
    if (fixed) {
      const double H = rint(xs * twoG);
      hq[e] = (int32_t)H;
      hl[e] = (float)(xs - H * twomG);
    }
  }
}

__global__ void norms_kernel(const float* __restrict__ xs32, int64_t ldn, int p, float* __restrict__ nrm) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < ldn; i += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int k = 0; k < p; ++k) {
      const double x = (double)xs32[(size_t)k * ldn + i];
      s += x * x;
    }
    nrm[i] = (float)s;
  }
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn get_encode() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiledFn)p;
  }
  return fn;
}

// Tensor map over a feature-major [p][ldn] array of 4-byte elements, box 128 x p.
static bool make_tmap(CUtensorMap* tm, void* base, CUtensorMapDataType dt, int64_t ldn, int64_t p) {
  EncodeTiledFn enc = get_encode();
  if (!enc) return false;
  cuuint64_t dims[2] = {(cuuint64_t)ldn, (cuuint64_t)p};
  cuuint64_t strides[1] = {(cuuint64_t)ldn * 4};
  cuuint32_t box[2] = {(cuuint32_t)kTile, (cuuint32_t)p};
  cuuint32_t estr[2] = {1, 1};
  return enc(tm, dt, 2, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Tensor map over a row-major [ldn][Kp] FP32 array, box 32 x 128 (128 bytes x 128 rows),
// 128-byte swizzle: the canonical K-major operand layout of tcgen05.mma.
bool make_tmap_rowmajor_sw128(CUtensorMap* tm, void* base, int64_t ldn, int Kp) {
  EncodeTiledFn enc = get_encode();
  if (!enc) return false;
  cuuint64_t dims[2] = {(cuuint64_t)Kp, (cuuint64_t)ldn};
  cuuint64_t strides[1] = {(cuuint64_t)Kp * 4};
  cuuint32_t box[2] = {32, 128};
  cuuint32_t estr[2] = {1, 1};
  return enc(tm, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
             CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
         CUDA_SUCCESS;
}

// Tensor map over a 2-D FP32 array (inner extent, outer extent, row pitch in bytes) with
// the 128-byte swizzle; box_inner x 4 must be 128 bytes.
bool make_tmap_2d_f32_sw128(CUtensorMap* tm, void* base, int64_t inner, int64_t outer, int64_t row_bytes,
                            int box_inner, int box_outer) {
  EncodeTiledFn enc = get_encode();
  if (!enc) return false;
  cuuint64_t dims[2] = {(cuuint64_t)inner, (cuuint64_t)outer};
  cuuint64_t strides[1] = {(cuuint64_t)row_bytes};
  cuuint32_t box[2] = {(cuuint32_t)box_inner, (cuuint32_t)box_outer};
  cuuint32_t estr[2] = {1, 1};
  return enc(tm, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
             CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
         CUDA_SUCCESS;
}

// Tensor map over a row-major [ldn][64] bf16 array, box 64 x 128 (128 bytes x 128 rows),
// 128-byte swizzle: the K-major operand layout of tcgen05.mma kind::f16.
bool make_tmap_rowmajor_bf16_sw128(CUtensorMap* tm, void* base, int64_t ldn) {
  EncodeTiledFn enc = get_encode();
  if (!enc) return false;
  cuuint64_t dims[2] = {64, (cuuint64_t)ldn};
  cuuint64_t strides[1] = {128};
  cuuint32_t box[2] = {64, 128};
  cuuint32_t estr[2] = {1, 1};
  return enc(tm, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
             CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
         CUDA_SUCCESS;
}

static void free_all(Handle* h) {
  void* bufs[] = {h->xs32, h->nrm32, h->hq, h->hl, h->exp_table, h->xc64, h->y, h->F32, h->dres, h->core, h->tvec,
                  h->Linv, h->part, h->v32, h->vec_pool, h->scal, h->red_counter, h->red_part, h->err_flag,
                  h->st_alpha, h->st_v, h->st_z, h->sym_units, h->tc_hi, h->tc_lo, h->tc_bf, h->tc_sym_units, h->tc_a16, h->tc_b16};
  for (void* b : bufs) dev_free(h, b);
  kstore_free(h);
  batch_free(h);
  for (auto& g : h->cg_graph)
    if (g.exec) {
      cudaGraphExecDestroy(g.exec);
      g.exec = nullptr;
    }
  if (h->scal_host) cudaFreeHost(h->scal_host);
  for (int k = 0; k < 3; ++k) {
    for (cudaEvent_t e : h->prof_ev[k]) cudaEventDestroy(e);
    h->prof_ev[k].clear();
  }
  if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
}

static kqr_status create(Handle* h, const double* X, const double* y, int64_t n, int64_t p, kqr_kernel kind,
                         double gamma, const kqr_options* opts) {
  if (!X || !y) return fail(h, KQR_INVALID_ARG, "X and y must be non-null");
  if (n < 2) return fail(h, KQR_INVALID_ARG, "n must be >= 2");
  if (p < 1 || p > kMaxP) return fail(h, KQR_INVALID_ARG, "p must be in [1, 64]");
  if (n > (int64_t)1 << 30) return fail(h, KQR_INVALID_ARG, "n too large");
  if (kind != KQR_RBF && kind != KQR_LAPLACIAN) return fail(h, KQR_INVALID_ARG, "unknown kernel");
  if (!(gamma > 0.0) || !std::isfinite(gamma)) return fail(h, KQR_INVALID_ARG, "gamma must be positive and finite");
  for (int64_t i = 0; i < n; ++i)
    if (!std::isfinite(y[i])) return fail(h, KQR_INVALID_ARG, "y has a non-finite entry");
  for (int64_t i = 0; i < n * p; ++i)
    if (!std::isfinite(X[i])) return fail(h, KQR_INVALID_ARG, "X has a non-finite entry");
  if (opts) h->opt = *opts;
  else kqr_default_options(&h->opt);
  const double* uniforms = h->opt.pivot_uniforms;
  h->opt.pivot_uniforms = nullptr;
  h->alloc = g_alloc;
  h->n = n;
  h->p = p;
  h->ldn = (n + kTile - 1) / kTile * kTile;
  h->kind = kind;
  h->gamma = gamma;
  cudaError_t e;
  if ((e = cudaGetDevice(&h->device)) != cudaSuccess) return cuda_fail(h, e, "cudaGetDevice");
  if ((e = cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device)) != cudaSuccess)
    return cuda_fail(h, e, "SM count");
  if ((e = cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking)) != cudaSuccess)
    return cuda_fail(h, e, "stream");
  h->own_stream = true;
  cudaStream_t st = h->stream;
  const int64_t ldn = h->ldn;
  const size_t fe = (size_t)ldn * p;
  h->xs32 = (float*)dev_alloc(h, fe * 4);
  h->nrm32 = (float*)dev_alloc(h, ldn * 4);
  h->xc64 = (double*)dev_alloc(h, fe * 8);
  h->y = (double*)dev_alloc(h, ldn * 8);
  // Fixed-point layout for the FP64-class products: every Laplacian problem, and RBF
  // problems with p <= kRbfEmuMaxP (the emulated RBF product's shared-memory limit).
  const bool fixed_point = kind == KQR_LAPLACIAN || p <= kRbfEmuMaxP;
  if (fixed_point) {
    h->hq = (int32_t*)dev_alloc(h, fe * 4);
    h->hl = (float*)dev_alloc(h, fe * 4);
    h->exp_table = (float2*)dev_alloc(h, sizeof(float2) << kExpTableBits);
  }
  h->vec_pool = (double*)dev_alloc(h, sizeof(double) * V_COUNT * ldn);
  h->scal = (double*)dev_alloc(h, sizeof(double) * S_COUNT);
  h->red_counter = (unsigned int*)dev_alloc(h, 64);
  h->red_part = (double*)dev_alloc(h, sizeof(double) * 304 * 10);
  h->err_flag = (int*)dev_alloc(h, 64);
  h->st_alpha = (double*)dev_alloc(h, ldn * 8);
  h->st_v = (double*)dev_alloc(h, ldn * 8);
  h->st_z = (double*)dev_alloc(h, ldn * 8);
  double* Xd = (double*)dev_alloc(h, (size_t)n * p * 8);
  double* stats = (double*)dev_alloc(h, (size_t)p * 3 * 8);
  if (!h->xs32 || !h->nrm32 || !h->xc64 || !h->y || (fixed_point && (!h->hq || !h->hl || !h->exp_table)) ||
      !h->vec_pool || !h->scal || !h->red_counter || !h->red_part || !h->err_flag || !h->st_alpha || !h->st_v ||
      !h->st_z || !Xd || !stats) {
    dev_free(h, Xd);
    dev_free(h, stats);
    return fail(h, KQR_OOM, "device buffers");
  }
  if ((e = cudaMallocHost(&h->scal_host, sizeof(double) * S_COUNT)) != cudaSuccess) {
    dev_free(h, Xd);
    dev_free(h, stats);
    return cuda_fail(h, e, "pinned scalars");
  }
  cudaMemsetAsync(h->red_counter, 0, 64, st);
  cudaMemsetAsync(h->err_flag, 0, 64, st);
  cudaMemsetAsync(h->scal, 0, sizeof(double) * S_COUNT, st);
  cudaMemsetAsync(h->vec_pool, 0, sizeof(double) * V_COUNT * ldn, st);
  cudaMemsetAsync(h->y, 0, ldn * 8, st);
  cudaMemcpyAsync(Xd, X, (size_t)n * p * 8, cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(h->y, y, (size_t)n * 8, cudaMemcpyHostToDevice, st);
  colstats_kernel<<<(unsigned)p, 256, 0, st>>>(Xd, n, (int)p, stats);
  h->launches++;
  std::vector<double> hs((size_t)p * 3);
  e = cudaMemcpyAsync(hs.data(), stats, hs.size() * 8, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    dev_free(h, Xd);
    dev_free(h, stats);
    return cuda_fail(h, e, "column statistics");
  }
  // K_ij = exp2(-(log2 e) gamma dist): fold log2(e) gamma into the stored coordinates.
  const double g2 = gamma / std::log(2.0);
  const double scale = kind == KQR_LAPLACIAN ? g2 : std::sqrt(g2);
  int G = 0;
  if (fixed_point) {
    double R = 0.0;
    for (int64_t k = 0; k < p; ++k) R = std::fmax(R, (hs[3 * k + 2] - hs[3 * k + 1]) * scale);
    if (kind == KQR_LAPLACIAN) {
      // sum_k |hq_ik - hq_jk| <= p R 2^G must stay below 2^30 (int32 with a spare bit)
      G = R > 0 ? (int)std::floor(std::log2(((double)(1 << 30) - 1.0) / ((double)p * R))) : 33;
      if (G > 33) G = 33;
    } else {
      // sum_k (hq_ik - hq_jk)^2 <= p (R 2^G)^2 must stay below 2^62 (int64 with a spare bit);
      // G <= 28 keeps the sub-table remainder (< 2^(2G - 10)) within two 23-bit floats
      G = R > 0 ? (int)std::floor(std::log2(2147483000.0 / (R * std::sqrt((double)p)))) : 28;
      if (G > 28) G = 28;
    }
    const int Gmin = kind == KQR_LAPLACIAN ? kExpTableBits + 1 : 17;
    if (G < Gmin) {
      dev_free(h, Xd);
      dev_free(h, stats);
      return fail(h, KQR_INVALID_ARG, "gamma * data range too large for the high-precision fixed-point layout");
    }
    h->grid_G = G;
    std::vector<float2> tab(1 << kExpTableBits);
    for (int k2 = 0; k2 < (1 << kExpTableBits); ++k2) {
      const double t = std::exp2(-(double)k2 / (double)(1 << kExpTableBits));
      const float hi = (float)t;
      tab[k2] = make_float2(hi, (float)(t - (double)hi));
    }
    cudaMemcpyAsync(h->exp_table, tab.data(), tab.size() * sizeof(float2), cudaMemcpyHostToDevice, st);
  }
  layout_kernel<<<grid_for(ldn * p), 256, 0, st>>>(Xd, stats, n, ldn, (int)p, scale, fixed_point ? 1 : 0, G, h->xc64,
                                                    h->xs32, h->hq, h->hl);
  norms_kernel<<<grid_for(ldn), 256, 0, st>>>(h->xs32, ldn, (int)p, h->nrm32);
  h->launches += 2;
  e = cudaStreamSynchronize(st);
  dev_free(h, Xd);
  dev_free(h, stats);
  if (e != cudaSuccess) return cuda_fail(h, e, "layout");
  if (!make_tmap(&h->tm_xs32, h->xs32, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, ldn, p))
    return fail(h, KQR_CUDA_ERROR, "cuTensorMapEncodeTiled failed for the FP32 layout");
  if (fixed_point) {
    if (!make_tmap(&h->tm_hq, h->hq, CU_TENSOR_MAP_DATA_TYPE_INT32, ldn, p) ||
        !make_tmap(&h->tm_hl, h->hl, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, ldn, p))
      return fail(h, KQR_CUDA_ERROR, "cuTensorMapEncodeTiled failed for the fixed-point layout");
  }
  kqr_status ks = kstore_setup(h);
  if (ks != KQR_OK) return ks;
  return rpcholesky_setup(h, uniforms);
}

}  // namespace kqr

using namespace kqr;

extern "C" {

void kqr_default_options(kqr_options* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->rank0 = 0;
  o->adaptive_rank = 1;
  o->xi = 1e-10;
  o->seed = 12345;
  o->pivot_uniforms = nullptr;
  o->precond = KQR_PRECOND_NYSTROM_DIAG;
  o->sigma0 = 1.0;
  o->gamma_admm = 1.618;
  o->admm_tol = 1e-3;
  o->admm_cg_rtol = 3e-4;
  o->admm_maxit = 100;
  o->balance_every = 5;
  o->balance_ratio = 5.0;
  o->balance_factor = 1.5;
  o->alm_maxit = 1000;
  o->sigma_alm_scale = 1.0;
  o->sigma_factor = 10.0;
  o->sigma_max = 1e8;
  o->eta_bar = 0.5;
  o->iota = 0.5;
  o->mu = 1e-4;
  o->r_ls = 0.5;
  o->tau1 = 1e-2;
  o->tau2 = 1e-1;
  o->ssn_maxit = 50;
  o->ls_maxit = 40;
  o->pcg_maxit = 1000;
  o->core_reuse_rtol = 1e-2;
  o->time_limit_s = 0.0;
  o->phase1_only = 0;
  o->symmetric_gram = 1;
  o->rbf_tensor_cores = 1;
  o->verbose = 0;
  o->cg_high = 2;
  o->gram_store = 2;
}

void kqr_set_allocator(void* (*alloc)(size_t, void*), void (*free_fn)(void*, void*), void* ctx) {
  g_alloc.alloc = alloc;
  g_alloc.free_fn = free_fn;
  g_alloc.ctx = ctx;
}

kqr_status kqr_create(const double* X, const double* y, int64_t n, int64_t p, kqr_kernel kind, double gamma,
                      const kqr_options* opts, kqr_handle** out) {
  if (!out) return KQR_INVALID_ARG;
  *out = nullptr;
  kqr_handle* kh = new (std::nothrow) kqr_handle();
  if (!kh) return KQR_OOM;
  kqr_status s = create(&kh->h, X, y, n, p, kind, gamma, opts);
  if (s != KQR_OK) {
    free_all(&kh->h);
    *out = kh;  // keep the handle so kqr_last_error can report; caller destroys it
    return s;
  }
  *out = kh;
  return KQR_OK;
}

void kqr_destroy(kqr_handle* kh) {
  if (!kh) return;
  Handle* h = &kh->h;
  if (h->stream) cudaStreamSynchronize(h->stream);
  free_all(h);
  delete kh;
}

const char* kqr_last_error(const kqr_handle* kh) { return kh ? kh->h.err.c_str() : "null handle"; }

const char* kqr_status_string(kqr_status s) {
  switch (s) {
    case KQR_OK: return "ok";
    case KQR_INVALID_ARG: return "invalid argument";
    case KQR_OOM: return "out of device memory";
    case KQR_CUDA_ERROR: return "CUDA error";
    case KQR_NOT_CONVERGED: return "not converged";
    case KQR_BREAKDOWN: return "breakdown";
    case KQR_TIMEOUT: return "time limit";
    case KQR_DEVICE_WAIT_TIMEOUT: return "device wait timeout";
  }
  return "unknown status";
}

int64_t kqr_n(const kqr_handle* kh) { return kh ? kh->h.n : 0; }
int64_t kqr_p(const kqr_handle* kh) { return kh ? kh->h.p : 0; }
int64_t kqr_launch_count(const kqr_handle* kh) { return kh ? kh->h.launches : 0; }

kqr_status kqr_set_stream(kqr_handle* kh, void* stream) {
  if (!kh) return KQR_INVALID_ARG;
  Handle* h = &kh->h;
  if (stream) {
    // The caller keeps ownership of its stream; release ours.
    if (h->own_stream && h->stream) {
      cudaStreamSynchronize(h->stream);
      cudaStreamDestroy(h->stream);
    }
    h->stream = (cudaStream_t)stream;
    h->own_stream = false;
  } else {
    cudaStream_t s;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return KQR_CUDA_ERROR;
    if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
    h->stream = s;
    h->own_stream = true;
    return KQR_OK;
  }
  return KQR_OK;
}

kqr_status kqr_solve(kqr_handle* kh, double tau, double lambda, double tol, double* alpha, double* beta, double* kkt_out,
                     kqr_info* info) {
  if (!kh) return KQR_INVALID_ARG;
  Handle* h = &kh->h;
  KQR_SINGLE(h);
  if (!(tau > 0.0 && tau < 1.0)) return fail(h, KQR_INVALID_ARG, "tau must be in (0, 1)");
  if (!(lambda > 0.0) || !std::isfinite(lambda)) return fail(h, KQR_INVALID_ARG, "lambda must be positive");
  if (!(tol > 0.0)) return fail(h, KQR_INVALID_ARG, "tol must be positive");
  kqr_info inf{};
  kqr_status s = kqr::solve(h, tau, lambda, tol, &inf);
  if (info) *info = inf;
  if (h->has_state && (s == KQR_OK || s == KQR_NOT_CONVERGED || s == KQR_TIMEOUT)) {
    if (alpha) {
      cudaError_t e = cudaMemcpy(alpha, h->st_alpha, sizeof(double) * h->n, cudaMemcpyDeviceToHost);
      if (e != cudaSuccess) return cuda_fail(h, e, "copy alpha");
    }
    if (beta) *beta = h->st_beta;
    if (kkt_out) *kkt_out = inf.eta_kkt;
  }
  return s;
}

kqr_status kqr_get_state(kqr_handle* kh, double* v, double* z) {
  if (!kh) return KQR_INVALID_ARG;
  Handle* h = &kh->h;
  KQR_SINGLE(h);
  if (!h->has_state) return fail(h, KQR_INVALID_ARG, "no solve has run on this handle");
  if (v && cudaMemcpy(v, h->st_v, sizeof(double) * h->n, cudaMemcpyDeviceToHost) != cudaSuccess)
    return fail(h, KQR_CUDA_ERROR, "copy v");
  if (z && cudaMemcpy(z, h->st_z, sizeof(double) * h->n, cudaMemcpyDeviceToHost) != cudaSuccess)
    return fail(h, KQR_CUDA_ERROR, "copy z");
  return KQR_OK;
}

kqr_status kqr_kmatvec_dev(kqr_handle* kh, const double* V, double* U, int64_t m, kqr_precision prec, void* stream) {
  if (!kh) return KQR_INVALID_ARG;
  Handle* h = &kh->h;
  KQR_SINGLE(h);
  if (!V || !U) return fail(h, KQR_INVALID_ARG, "V and U must be non-null");
  if (m < 1 || m > kMaxRhs) return fail(h, KQR_INVALID_ARG, "m must be in [1, 8]");
  cudaStream_t st = pick_stream(h, stream);
  cudaError_t e;
  if (prec == KQR_PREC_FP32) e = gram_f32(h, V, U, (int)m, nullptr, st);
  else if (prec == KQR_PREC_HIGH) e = gram_high(h, V, U, (int)m, st);
  else if (prec == KQR_PREC_TF32) {
    if (h->kind != KQR_RBF) return fail(h, KQR_INVALID_ARG, "KQR_PREC_TF32 applies to the RBF kernel only");
    e = gram_rbf_tc(h, V, U, (int)m, false, nullptr, st);
  } else if (prec == KQR_PREC_BF16) {
    if (h->kind != KQR_RBF) return fail(h, KQR_INVALID_ARG, "KQR_PREC_BF16 applies to the RBF kernel only");
    e = gram_rbf_tc_bf16(h, V, U, (int)m, st);
  } else return fail(h, KQR_INVALID_ARG, "unknown precision");
  if (e != cudaSuccess) return cuda_fail(h, e, "Gram product");
  return KQR_OK;
}

kqr_status kqr_kmatvec(kqr_handle* kh, const double* V, double* U, int64_t m, kqr_precision prec) {
  if (!kh) return KQR_INVALID_ARG;
  Handle* h = &kh->h;
  KQR_SINGLE(h);
  if (!V || !U) return fail(h, KQR_INVALID_ARG, "V and U must be non-null");
  if (m < 1 || m > kMaxRhs) return fail(h, KQR_INVALID_ARG, "m must be in [1, 8]");
  const size_t bytes = sizeof(double) * (size_t)h->n * m;
  double* dV = (double*)dev_alloc(h, bytes);
  double* dU = (double*)dev_alloc(h, bytes);
  if (!dV || !dU) {
    dev_free(h, dV);
    dev_free(h, dU);
    return fail(h, KQR_OOM, "kmatvec buffers");
  }
  cudaStream_t st = h->stream;
  cudaError_t e = cudaMemcpyAsync(dV, V, bytes, cudaMemcpyHostToDevice, st);
  kqr_status s = KQR_OK;
  if (e == cudaSuccess) {
    s = kqr_kmatvec_dev(kh, dV, dU, m, prec, st);
    if (s == KQR_OK) {
      e = cudaMemcpyAsync(U, dU, bytes, cudaMemcpyDeviceToHost, st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    }
  }
  if (s == KQR_OK && e == cudaSuccess) {
    int flag = 0;
    cudaMemcpy(&flag, h->err_flag, sizeof(int), cudaMemcpyDeviceToHost);
    if (flag) s = fail(h, KQR_DEVICE_WAIT_TIMEOUT, "a Gram kernel gave up waiting for a tile copy");
  }
  dev_free(h, dV);
  dev_free(h, dU);
  if (s != KQR_OK) return s;
  if (e != cudaSuccess) return cuda_fail(h, e, "kmatvec copy");
  return KQR_OK;
}

kqr_status kqr_box_grad_dev(kqr_handle* kh, const double* alpha, const double* z, const double* Kalpha, double beta,
                            double sigma, double tau, double lambda, double eps, double* v, double* S, double* grad,
                            double* Ldiag, double* grad_norm2, void* stream) {
  if (!kh) return KQR_INVALID_ARG;
  Handle* h = &kh->h;
  KQR_SINGLE(h);
  if (!alpha || !z || !Kalpha) return fail(h, KQR_INVALID_ARG, "alpha, z and Kalpha must be non-null");
  if (!(sigma > 0) || !(lambda > 0) || !(tau > 0 && tau < 1)) return fail(h, KQR_INVALID_ARG, "bad sigma/lambda/tau");
  cudaStream_t st = pick_stream(h, stream);
  cudaError_t e = box_grad(h, alpha, z, Kalpha, h->y, beta, sigma, tau, lambda, eps, nullptr, v, S, grad, Ldiag,
                           nullptr, h->n, st);
  if (e != cudaSuccess) return cuda_fail(h, e, "box_grad");
  if (grad_norm2) {
    e = cudaMemcpyAsync(h->scal_host + S_RED0 + 13, h->scal + S_RED0 + 13, sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(h, e, "grad norm");
    *grad_norm2 = h->scal_host[S_RED0 + 13];
  }
  return KQR_OK;
}

kqr_status kqr_precond_apply_dev(kqr_handle* kh, const double* Ldiag, double gam, const double* r, double* out,
                                 void* stream) {
  if (!kh) return KQR_INVALID_ARG;
  Handle* h = &kh->h;
  KQR_SINGLE(h);
  if (!Ldiag || !r || !out) return fail(h, KQR_INVALID_ARG, "null vector");
  if (!(gam > 0)) return fail(h, KQR_INVALID_ARG, "gam must be positive");
  cudaStream_t st = pick_stream(h, stream);
  const kqr_precond saved = h->opt.precond;
  h->opt.precond = KQR_PRECOND_PAPER;
  kqr_status s = precond_build(h, Ldiag, gam, st);
  if (s == KQR_OK) {
    cudaError_t e = precond_apply(h, Ldiag, r, out, nullptr, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) s = cuda_fail(h, e, "precond apply");
  }
  h->opt.precond = saved;
  return s;
}

kqr_status kqr_pcg_dev(kqr_handle* kh, const double* Ldiag, double gam, const double* b, double* x, double tol,
                       int32_t maxit, int32_t* iters, void* stream) {
  if (!kh) return KQR_INVALID_ARG;
  Handle* h = &kh->h;
  KQR_SINGLE(h);
  h->cg_high_on = false;   // the parity entry point always runs FP32 products
  if (!Ldiag || !b || !x) return fail(h, KQR_INVALID_ARG, "null vector");
  if (!(gam >= 0) || !(tol > 0) || maxit < 1) return fail(h, KQR_INVALID_ARG, "bad gam/tol/maxit");
  cudaStream_t st = pick_stream(h, stream);
  double* Lpre = vec(h, V_LPRE);
  double* L = vec(h, V_L);
  cudaError_t e = vec_copy(h, L, Ldiag, h->n, st);
  if (e == cudaSuccess) e = vec_copy(h, Lpre, Ldiag, h->n, st);
  if (e == cudaSuccess && h->opt.precond == KQR_PRECOND_NYSTROM_DIAG) e = axpy_vec(h, Lpre, h->dres, 1.0, h->n, st);
  if (e != cudaSuccess) return cuda_fail(h, e, "pcg set-up");
  kqr_status s = precond_build(h, Lpre, gam > 0 ? gam : 1e-300, st);
  if (s != KQR_OK) return s;
  int it = 0;
  s = pcg(h, L, Lpre, gam, b, x, nullptr, false, tol, maxit, &it, st);
  if (iters) *iters = it;
  if (s == KQR_OK && cudaStreamSynchronize(st) != cudaSuccess) return fail(h, KQR_CUDA_ERROR, "pcg sync");
  if (s == KQR_OK && !h->cg_met)
    return fail(h, KQR_NOT_CONVERGED, h->cg_truncated ? "CG stopped at a non-positive curvature p^T A p <= 0"
                                                      : "CG reached maxit before the tolerance");
  return s;
}

kqr_status kqr_kkt(kqr_handle* kh, const double* alpha, const double* v, double beta, const double* z, double tau,
                   double lambda, double* out7) {
  if (!kh) return KQR_INVALID_ARG;
  Handle* h = &kh->h;
  KQR_SINGLE(h);
  if (!alpha || !v || !z || !out7) return fail(h, KQR_INVALID_ARG, "null pointer");
  const size_t bytes = sizeof(double) * h->n;
  double* buf = (double*)dev_alloc(h, bytes * 4);
  if (!buf) return fail(h, KQR_OOM, "kkt buffers");
  double *da = buf, *dv = buf + h->n, *dz = buf + 2 * h->n, *dK = buf + 3 * h->n;
  cudaStream_t st = h->stream;
  cudaMemcpyAsync(da, alpha, bytes, cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(dv, v, bytes, cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(dz, z, bytes, cudaMemcpyHostToDevice, st);
  cudaError_t e = gram_high(h, da, dK, 1, st);
  kqr_status s = KQR_OK;
  if (e != cudaSuccess) s = cuda_fail(h, e, "kkt Gram product");
  else s = kqr::kkt(h, da, dv, beta, dz, dK, tau, lambda, out7, st);
  cudaStreamSynchronize(st);
  dev_free(h, buf);
  return s;
}

kqr_status kqr_check_device(kqr_handle* kh) {
  if (!kh) return KQR_INVALID_ARG;
  Handle* h = &kh->h;
  if (!h->err_flag) return fail(h, KQR_INVALID_ARG, "handle has no device state");
  int flag = 0;
  cudaError_t e = cudaMemcpy(&flag, h->err_flag, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(h, e, "read device error word");
  if (!flag) return KQR_OK;
  if ((e = cudaMemset(h->err_flag, 0, sizeof(int))) != cudaSuccess) return cuda_fail(h, e, "clear device error word");
  return fail(h, KQR_DEVICE_WAIT_TIMEOUT, "a kernel gave up a bounded wait; its results are incomplete");
}

kqr_status kqr_test_bounded_wait(kqr_handle* kh, uint32_t max_polls) {
  if (!kh) return KQR_INVALID_ARG;
  Handle* h = &kh->h;
  if (!h->err_flag) return fail(h, KQR_INVALID_ARG, "handle has no device state");
  if (max_polls < 1 || max_polls > (1u << 20)) return fail(h, KQR_INVALID_ARG, "max_polls must be in [1, 2^20]");
  cudaError_t e = launch_wait_probe(h, max_polls, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "bounded-wait probe");
  return KQR_OK;
}

kqr_status kqr_refactor(kqr_handle* kh, const double* pivot_uniforms) {
  if (!kh) return KQR_INVALID_ARG;
  Handle* h = &kh->h;
  KQR_SINGLE(h);
  h->has_state = false;
  return rpcholesky_setup(h, pivot_uniforms);
}

kqr_status kqr_batch_create(const double* X, const int64_t* offsets, int64_t B, int64_t p, const double* gammas,
                            int32_t flags, kqr_handle** out) {
  if (!out) return KQR_INVALID_ARG;
  *out = nullptr;
  kqr_handle* kh = new (std::nothrow) kqr_handle();
  if (!kh) return KQR_OOM;
  *out = kh;
  Handle* h = &kh->h;
  h->alloc = g_alloc;
  cudaError_t e;
  if ((e = cudaGetDevice(&h->device)) != cudaSuccess) return cuda_fail(h, e, "cudaGetDevice");
  if ((e = cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device)) != cudaSuccess)
    return cuda_fail(h, e, "SM count");
  if ((e = cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking)) != cudaSuccess)
    return cuda_fail(h, e, "stream");
  h->own_stream = true;
  h->err_flag = (int*)dev_alloc(h, 64);
  if (!h->err_flag) return fail(h, KQR_OOM, "error flag");
  if ((e = cudaMemsetAsync(h->err_flag, 0, 64, h->stream)) != cudaSuccess) return cuda_fail(h, e, "error flag");
  kqr_status s = batch_create(h, X, offsets, B, p, gammas, flags);
  if (s != KQR_OK) return s;
  h->n = offsets[B];
  h->p = p;
  h->kind = KQR_RBF;
  return KQR_OK;
}

kqr_status kqr_batch_kmatmul_dev(kqr_handle* kh, const double* V, double* U, int64_t m) {
  if (!kh) return KQR_INVALID_ARG;
  Handle* h = &kh->h;
  if (!h->batch) return fail(h, KQR_INVALID_ARG, "not a batch handle (kqr_batch_create)");
  if (!V || !U) return fail(h, KQR_INVALID_ARG, "V and U must be non-null");
  if (m < 1 || m > 64) return fail(h, KQR_INVALID_ARG, "m must be in [1, 64]");
  cudaError_t e = batch_kmatmul(h, V, U, (int)m, h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "batched Gram product");
  return KQR_OK;
}

kqr_status kqr_batch_kmatmul(kqr_handle* kh, const double* V, double* U, int64_t m) {
  if (!kh) return KQR_INVALID_ARG;
  Handle* h = &kh->h;
  if (!h->batch) return fail(h, KQR_INVALID_ARG, "not a batch handle (kqr_batch_create)");
  if (!V || !U) return fail(h, KQR_INVALID_ARG, "V and U must be non-null");
  if (m < 1 || m > 64) return fail(h, KQR_INVALID_ARG, "m must be in [1, 64]");
  const size_t bytes = sizeof(double) * (size_t)h->n * m;
  double* dV = (double*)dev_alloc(h, bytes);
  double* dU = (double*)dev_alloc(h, bytes);
  kqr_status s = KQR_OK;
  cudaError_t e = cudaSuccess;
  if (!dV || !dU) {
    s = fail(h, KQR_OOM, "batched product buffers");
  } else {
    e = cudaMemcpyAsync(dV, V, bytes, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) {
      s = kqr_batch_kmatmul_dev(kh, dV, dU, m);
      if (s == KQR_OK) {
        e = cudaMemcpyAsync(U, dU, bytes, cudaMemcpyDeviceToHost, h->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
      }
    }
    if (s == KQR_OK && e != cudaSuccess) s = cuda_fail(h, e, "batched product copies");
  }
  if (s == KQR_OK) {
    int flag = 0;
    if (cudaMemcpy(&flag, h->err_flag, sizeof(int), cudaMemcpyDeviceToHost) == cudaSuccess && flag)
      s = fail(h, KQR_DEVICE_WAIT_TIMEOUT, "the batched Gram kernel gave up waiting");
  }
  dev_free(h, dV);
  dev_free(h, dU);
  return s;
}

kqr_status kqr_profile(kqr_handle* kh, int32_t enable) {
  if (!kh) return KQR_INVALID_ARG;
  Handle* h = &kh->h;
  h->prof_used[0] = h->prof_used[1] = h->prof_used[2] = 0;
  h->profile = enable != 0;
  return KQR_OK;
}

kqr_status kqr_profile_read(kqr_handle* kh, int32_t kernel_id, int64_t* launches, double* total_ms) {
  if (!kh) return KQR_INVALID_ARG;
  Handle* h = &kh->h;
  if (kernel_id < 0 || kernel_id > 2) return fail(h, KQR_INVALID_ARG, "kernel_id must be 0, 1 or 2");
  if (cudaStreamSynchronize(h->stream) != cudaSuccess) return fail(h, KQR_CUDA_ERROR, "profile sync");
  double tot = 0.0;
  const size_t pairs = h->prof_used[kernel_id] / 2;
  for (size_t i = 0; i < pairs; ++i) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, h->prof_ev[kernel_id][2 * i], h->prof_ev[kernel_id][2 * i + 1]) == cudaSuccess)
      tot += ms;
  }
  if (launches) *launches = (int64_t)pairs;
  if (total_ms) *total_ms = tot;
  return KQR_OK;
}

kqr_status kqr_get_factor(kqr_handle* kh, float* F, int64_t* pivots, int32_t* rank, int32_t* rank0) {
  if (!kh) return KQR_INVALID_ARG;
  Handle* h = &kh->h;
  KQR_SINGLE(h);
  if (rank) *rank = h->r;
  if (rank0) *rank0 = h->r0;
  if (pivots)
    for (size_t i = 0; i < h->pivots.size(); ++i) pivots[i] = h->pivots[i];
  if (F && h->r > 0) {
    if (cudaMemcpy(F, h->F32, sizeof(float) * (size_t)h->r * h->n, cudaMemcpyDeviceToHost) != cudaSuccess)
      return fail(h, KQR_CUDA_ERROR, "copy factor");
  }
  return KQR_OK;
}

}  // extern "C"
