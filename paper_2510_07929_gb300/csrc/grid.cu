// Solves over a grid of (tau, lambda) pairs: many columns of the dual (1.3) on
// one kernel matrix, and many problems at once.
//
// Every pair needs the same products with K (the ADMM systems of Alg. 1, the
// Newton systems (3.1) of Alg. 3, the gradient (2.3) and the Sec. 4 residuals),
// so the columns run in lockstep on their products.  Each column runs the
// single-pair solver (solver.cu) unchanged, on a clone of the problem's handle
// that shares the read-only state (the layouts of X, y, the RPCholesky factor
// F, a stored K) and owns its mutable state (solver vectors, device scalars,
// Woodbury core, stream).  Its Gram products go through a rendezvous: each
// active column posts its vector and waits; the leader gathers the posted
// vectors into n x m blocks of up to 8 columns, runs one multi-right-
// hand-side product per block on the base handle (FP32 and FP64-class requests
// separately) and scatters the results, after which every column continues on
// its own stream.  The first column to post leads: it waits a short window for
// the others (all active columns, or whoever posted within 200 us) and runs the
// batch, so a column that is busy elsewhere does not hold the rest back.  A
// column that has converged (or stopped) leaves the group, so later products
// carry only the active columns.  A column's CG (the bulk of the products)
// runs in a shared engine instead: the column queues its CG set-up on its own
// stream and posts the solve; a leader runs blocks of iterations for every
// posted column (the products of all their directions on the base stream,
// then each column's iteration chain on its own stream, forked and joined by
// events) with one status read per block for all of them, and releases the
// columns whose CG stopped.
#include <chrono>
#include <condition_variable>
#include <mutex>
#include <thread>
#include <vector>

#include "kqr_internal.h"

namespace kqr {

struct GridRdv {
  Handle* base = nullptr;
  cudaStream_t st = nullptr;
  std::mutex mu;
  std::condition_variable cv;
  int active = 0;                 // columns still solving
  bool leading = false;           // a column is gathering the next batch
  struct Req {
    const double* p;
    double* out;
    bool high;
    cudaEvent_t ready;
    bool done;
  };
  std::vector<Req*> reqs;         // posted, not yet taken into a batch
  cudaEvent_t done = nullptr;     // recorded after each batch (the product stream runs batches in order)
  cudaError_t err = cudaSuccess;
  double* V = nullptr;            // gathered vectors, ldn x 8
  double* U = nullptr;            // products, ldn x 8
  int64_t rounds = 0, columns = 0;
  // shared CG engine: columns waiting to join, columns iterating, the thread running blocks
  struct CgJob {
    Handle* h;
    CgArgs a;
    bool done;
  };
  std::vector<CgJob*> cg_new, cg_active;
  bool cg_leading = false;
  cudaEvent_t ev_scatter = nullptr, ev_block = nullptr;
  double* status_host = nullptr;  // pinned, 2 per column (status, iterations)
  int64_t cg_blocks = 0, cg_iterations = 0;
};

// CG iterations the engine runs between two status reads of its columns.
constexpr int kGridCgBlock = 2;

// How long the first column to post a product waits for the others before it runs
// the batch with whatever has been posted: long enough for columns that are between
// two products of the same CG iteration, short enough that a column busy elsewhere
// (a host read, a core build) does not hold the others back.
constexpr auto kGridWindow = std::chrono::microseconds(200);

struct Ptr8 {
  const double* p[8];
};
struct OutPtr8 {
  double* p[8];
};

__global__ void grid_gather_kernel(Ptr8 src, int cnt, int64_t n, double* __restrict__ V) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * cnt; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / cnt;
    const int k = (int)(e % cnt);
    V[e] = src.p[k][i];
  }
}

__global__ void grid_scatter_kernel(const double* __restrict__ U, int cnt, int64_t n, OutPtr8 dst) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * cnt; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / cnt;
    const int k = (int)(e % cnt);
    dst.p[k][i] = U[e];
  }
}

// K p for each (p, out, high) on the base handle's stream, up to 8 columns per launch,
// FP32 and FP64-class requests separately (caller holds the lock).
struct ProdReq {
  const double* p;
  double* out;
  bool high;
};

static cudaError_t run_products(GridRdv* g, const std::vector<ProdReq>& reqs) {
  Handle* b = g->base;
  cudaError_t e = cudaSuccess;
  for (int pass = 0; pass < 2 && e == cudaSuccess; ++pass) {
    const bool high = pass == 1;
    std::vector<const ProdReq*> sel;
    for (auto& r : reqs)
      if (r.high == high) sel.push_back(&r);
    for (size_t k0 = 0; k0 < sel.size() && e == cudaSuccess; k0 += 8) {
      const int cnt = (int)std::min<size_t>(8, sel.size() - k0);
      Ptr8 src{};
      OutPtr8 dst{};
      for (int k = 0; k < cnt; ++k) {
        src.p[k] = sel[k0 + k]->p;
        dst.p[k] = sel[k0 + k]->out;
      }
      const double* V = src.p[0];
      double* U = dst.p[0];
      if (cnt > 1) {
        grid_gather_kernel<<<grid_for(b->n * cnt), 256, 0, g->st>>>(src, cnt, b->n, g->V);
        b->launches++;
        if ((e = cudaGetLastError()) != cudaSuccess) break;
        V = g->V;
        U = g->U;
      }
      e = high ? gram_high(b, V, U, cnt, g->st) : gram_f32(b, V, U, cnt, nullptr, g->st);
      if (e != cudaSuccess) break;
      if (cnt > 1) {
        grid_scatter_kernel<<<grid_for(b->n * cnt), 256, 0, g->st>>>(g->U, cnt, b->n, dst);
        b->launches++;
        e = cudaGetLastError();
      }
      g->columns += cnt;
    }
  }
  return e;
}

// Runs a batch of posted products (caller holds the lock).
static void run_batch(GridRdv* g, std::vector<GridRdv::Req*>& batch) {
  cudaError_t e = cudaSuccess;
  for (auto* r : batch)
    if (e == cudaSuccess) e = cudaStreamWaitEvent(g->st, r->ready, 0);
  std::vector<ProdReq> reqs;
  for (auto* r : batch) reqs.push_back({r->p, r->out, r->high});
  if (e == cudaSuccess) e = run_products(g, reqs);
  if (e == cudaSuccess) e = cudaEventRecord(g->done, g->st);
  if (e != cudaSuccess && g->err == cudaSuccess) g->err = e;
  g->rounds++;
  for (auto* r : batch) r->done = true;
}

// One block of the shared CG engine (caller holds the lock; it is released while the
// block runs on the GPU).  New columns join; every active column gets kGridCgBlock
// iterations: per iteration, the products of all columns' search directions on the base
// stream, then each column's chain (cg_after_product) on its own stream, the streams
// forked and joined by events so the chains run side by side; then one status read for
// all columns, after which the ones that stopped are released.
static void run_cg_block(GridRdv* g, std::unique_lock<std::mutex>& lk) {
  cudaError_t e = cudaSuccess;
  for (auto* j : g->cg_new) {
    if (e == cudaSuccess) e = cudaStreamWaitEvent(g->st, j->h->rdv_ev, 0);
    g->cg_active.push_back(j);
  }
  g->cg_new.clear();
  std::vector<GridRdv::CgJob*> act = g->cg_active;
  if (act.empty()) return;
  for (int it = 0; it < kGridCgBlock && e == cudaSuccess; ++it) {
    std::vector<ProdReq> reqs;
    for (auto* j : act) reqs.push_back({vec(j->h, V_P), vec(j->h, V_KP), j->h->cg_high_on});
    if ((e = run_products(g, reqs)) != cudaSuccess) break;
    if ((e = cudaEventRecord(g->ev_scatter, g->st)) != cudaSuccess) break;
    for (auto* j : act) {
      cudaStream_t js = j->h->stream;
      if ((e = cudaStreamWaitEvent(js, g->ev_scatter, 0)) != cudaSuccess) break;
      if ((e = cg_after_product(j->h, j->a, js)) != cudaSuccess) break;
      if ((e = cudaEventRecord(j->h->rdv_ev, js)) != cudaSuccess) break;
      if ((e = cudaStreamWaitEvent(g->st, j->h->rdv_ev, 0)) != cudaSuccess) break;
    }
  }
  for (size_t k = 0; k < act.size() && e == cudaSuccess; ++k)
    e = cudaMemcpyAsync(g->status_host + 2 * k, act[k]->h->scal + S_CGST, 2 * sizeof(double), cudaMemcpyDeviceToHost,
                        g->st);
  if (e == cudaSuccess) e = cudaEventRecord(g->ev_block, g->st);
  lk.unlock();
  if (e == cudaSuccess) e = cudaEventSynchronize(g->ev_block);
  lk.lock();
  g->cg_blocks++;
  g->cg_iterations += (int64_t)kGridCgBlock * (int64_t)act.size();
  if (e != cudaSuccess) {
    if (g->err == cudaSuccess) g->err = e;
    for (auto* j : act) j->done = true;   // the columns read the error and stop
    g->cg_active.clear();
    return;
  }
  std::vector<GridRdv::CgJob*> keep;
  for (size_t k = 0; k < act.size(); ++k) {
    if ((int)g->status_host[2 * k] != 0) act[k]->done = true;   // status left "running"
    else keep.push_back(act[k]);
  }
  g->cg_active.swap(keep);
}

cudaError_t grid_cg(Handle* h, const CgArgs& a) {
  GridRdv* g = h->rdv;
  cudaError_t e = cudaEventRecord(h->rdv_ev, h->stream);   // the column's CG set-up is queued before this
  if (e != cudaSuccess) return e;
  GridRdv::CgJob me{h, a, false};
  std::unique_lock<std::mutex> lk(g->mu);
  g->cg_new.push_back(&me);
  g->cv.notify_all();
  while (!me.done) {
    if (!g->cg_leading) {
      g->cg_leading = true;
      run_cg_block(g, lk);
      g->cg_leading = false;
      g->cv.notify_all();
    } else {
      g->cv.wait(lk);
    }
  }
  return g->err;
}

cudaError_t grid_product(Handle* h, const double* p, double* out, bool high, cudaStream_t st) {
  GridRdv* g = h->rdv;
  cudaError_t e = cudaEventRecord(h->rdv_ev, st);
  if (e != cudaSuccess) return e;
  GridRdv::Req me{p, out, high, h->rdv_ev, false};
  std::unique_lock<std::mutex> lk(g->mu);
  g->reqs.push_back(&me);
  g->cv.notify_all();
  while (!me.done) {
    if (!g->leading) {
      // lead: gather posts for up to kGridWindow (or until every active column posted)
      g->leading = true;
      g->cv.wait_for(lk, kGridWindow, [&] { return (int)g->reqs.size() >= g->active; });
      std::vector<GridRdv::Req*> batch;
      batch.swap(g->reqs);
      run_batch(g, batch);
      g->leading = false;
      g->cv.notify_all();
    } else {
      g->cv.wait(lk);
    }
  }
  e = g->err;
  lk.unlock();
  if (e != cudaSuccess) return e;
  // g->done holds this batch's record or a later one; the product stream runs batches
  // in order, so either covers this column's product.
  return cudaStreamWaitEvent(st, g->done, 0);
}

static void grid_leave(GridRdv* g) {
  std::lock_guard<std::mutex> lk(g->mu);
  g->active--;
  g->cv.notify_all();
}

// A column of the grid: the base handle's read-only state, its own mutable state.
static Handle* column_clone(Handle* base, GridRdv* g, kqr_status* st) {
  Handle* c = new (std::nothrow) Handle(*base);
  if (!c) {
    *st = KQR_OOM;
    return nullptr;
  }
  c->err.clear();
  for (int k = 0; k < 3; ++k) {
    c->prof_ev[k].clear();
    c->prof_used[k] = 0;
  }
  c->profile = false;
  for (auto& gr : c->cg_graph) gr = Handle::CgGraph();
  c->cg_graphs_off = true;
  c->batch = nullptr;
  c->rdv = g;
  c->part = nullptr;
  c->part_cap = 0;
  c->v32 = nullptr;
  c->v32_cap = 0;
  c->stream = nullptr;
  c->scal_host = nullptr;
  c->opt.cg_tf32 = 0;       // the grid runs FP32 or FP64-class CG products only
  c->opt.verbose = 0;
  const int N = c->r + 1;
  c->vec_pool = (double*)dev_alloc(base, sizeof(double) * V_COUNT * c->ldn);
  c->scal = (double*)dev_alloc(base, sizeof(double) * S_COUNT);
  c->red_counter = (unsigned int*)dev_alloc(base, 64);
  c->red_part = (double*)dev_alloc(base, sizeof(double) * 304 * 10);
  c->err_flag = (int*)dev_alloc(base, 64);
  c->core = (double*)dev_alloc(base, sizeof(double) * 3 * (size_t)N * N);
  c->tvec = (double*)dev_alloc(base, sizeof(double) * 2 * N);
  c->Linv = (double*)dev_alloc(base, sizeof(double) * c->n);
  c->st_alpha = (double*)dev_alloc(base, sizeof(double) * c->ldn);
  c->st_v = (double*)dev_alloc(base, sizeof(double) * c->ldn);
  c->st_z = (double*)dev_alloc(base, sizeof(double) * c->ldn);
  c->core_valid = false;
  c->has_state = false;
  *st = KQR_OK;
  if (!c->vec_pool || !c->scal || !c->red_counter || !c->red_part || !c->err_flag || !c->core || !c->tvec ||
      !c->Linv || !c->st_alpha || !c->st_v || !c->st_z) {
    *st = KQR_OOM;
    return c;
  }
  if (cudaMallocHost(&c->scal_host, sizeof(double) * S_COUNT) != cudaSuccess ||
      cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->rdv_ev, cudaEventDisableTiming) != cudaSuccess) {
    *st = KQR_CUDA_ERROR;
    return c;
  }
  c->own_stream = true;
  cudaStream_t s = c->stream;
  if (cudaMemsetAsync(c->red_counter, 0, 64, s) != cudaSuccess || cudaMemsetAsync(c->err_flag, 0, 64, s) != cudaSuccess ||
      cudaMemsetAsync(c->scal, 0, sizeof(double) * S_COUNT, s) != cudaSuccess ||
      cudaMemsetAsync(c->vec_pool, 0, sizeof(double) * V_COUNT * c->ldn, s) != cudaSuccess)
    *st = KQR_CUDA_ERROR;
  return c;
}

static void column_free(Handle* base, Handle* c) {
  if (!c) return;
  if (c->stream) cudaStreamSynchronize(c->stream);
  void* bufs[] = {c->vec_pool, c->scal, c->red_counter, c->red_part, c->err_flag, c->core,
                  c->tvec, c->Linv, c->st_alpha, c->st_v, c->st_z};
  for (void* b : bufs) dev_free(base, b);
  if (c->scal_host) cudaFreeHost(c->scal_host);
  if (c->rdv_ev) cudaEventDestroy(c->rdv_ev);
  if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
  delete c;
}

// Solves the m pairs of one problem; alpha is host n x m column-major.
static kqr_status solve_grid(Handle* h, int64_t m, const double* taus, const double* lambdas, double tol,
                             double* alpha, double* beta, double* kkt, int32_t* status, kqr_info* info) {
  GridRdv g;
  g.base = h;
  g.st = h->stream;
  cudaError_t e = cudaEventCreateWithFlags(&g.done, cudaEventDisableTiming);
  if (e != cudaSuccess) return cuda_fail(h, e, "grid event");
  g.V = (double*)dev_alloc(h, sizeof(double) * h->ldn * 8);
  g.U = (double*)dev_alloc(h, sizeof(double) * h->ldn * 8);
  std::vector<Handle*> cols(m, nullptr);
  kqr_status result = KQR_OK;
  if (!g.V || !g.U) result = fail(h, KQR_OOM, "grid product buffers");
  if (result == KQR_OK && ((e = cudaEventCreateWithFlags(&g.ev_scatter, cudaEventDisableTiming)) != cudaSuccess ||
                           (e = cudaEventCreateWithFlags(&g.ev_block, cudaEventDisableTiming)) != cudaSuccess ||
                           (e = cudaMallocHost(&g.status_host, sizeof(double) * 2 * m)) != cudaSuccess))
    result = cuda_fail(h, e, "grid CG engine");
  for (int64_t c = 0; c < m && result == KQR_OK; ++c) {
    kqr_status s = KQR_OK;
    cols[c] = column_clone(h, &g, &s);
    if (s != KQR_OK) result = fail(h, s, "grid column state");
  }
  if (result == KQR_OK && (e = cudaDeviceSynchronize()) != cudaSuccess) result = cuda_fail(h, e, "grid set-up");
  if (result == KQR_OK) {
    g.active = (int)m;
    std::vector<std::thread> threads;
    std::vector<kqr_status> st(m, KQR_OK);
    std::vector<kqr_info> inf(m);
    const int dev = h->device;
    for (int64_t c = 0; c < m; ++c) {
      threads.emplace_back([&, c]() {
        cudaSetDevice(dev);
        st[c] = solve(cols[c], taus[c], lambdas[c], tol, &inf[c]);
        grid_leave(&g);
      });
    }
    for (auto& t : threads) t.join();
    for (int64_t c = 0; c < m; ++c) {
      Handle* col = cols[c];
      if (status) status[c] = st[c];
      if (info) info[c] = inf[c];
      if (col->has_state) {
        if (alpha &&
            (e = cudaMemcpy(alpha + c * h->n, col->st_alpha, sizeof(double) * h->n, cudaMemcpyDeviceToHost)) !=
                cudaSuccess)
          result = cuda_fail(h, e, "grid alpha");
        if (beta) beta[c] = col->st_beta;
      }
      if (kkt) kkt[c] = inf[c].eta_kkt;
      if (st[c] != KQR_OK && st[c] != KQR_NOT_CONVERGED && st[c] != KQR_TIMEOUT && result == KQR_OK)
        result = fail(h, st[c], "grid column " + std::to_string(c) + ": " + col->err);
    }
    if (g.err != cudaSuccess && result == KQR_OK) result = cuda_fail(h, g.err, "grid product");
    int flag = 0;
    if (cudaMemcpy(&flag, h->err_flag, sizeof(int), cudaMemcpyDeviceToHost) == cudaSuccess && flag &&
        result == KQR_OK)
      result = fail(h, KQR_DEVICE_WAIT_TIMEOUT, "a Gram kernel gave up waiting for a tile copy");
  }
  for (Handle* c : cols) column_free(h, c);
  dev_free(h, g.V);
  dev_free(h, g.U);
  cudaEventDestroy(g.done);
  if (g.ev_scatter) cudaEventDestroy(g.ev_scatter);
  if (g.ev_block) cudaEventDestroy(g.ev_block);
  if (g.status_host) cudaFreeHost(g.status_host);
  h->grid_rounds += g.rounds;
  h->grid_columns += g.columns;
  return result;
}

static kqr_status check_grid_args(Handle* h, int64_t m, const double* taus, const double* lambdas, double tol) {
  if (m < 1 || m > 4096) return fail(h, KQR_INVALID_ARG, "m must be in [1, 4096]");
  if (!taus || !lambdas) return fail(h, KQR_INVALID_ARG, "taus and lambdas must be non-null");
  if (!(tol > 0.0)) return fail(h, KQR_INVALID_ARG, "tol must be positive");
  for (int64_t c = 0; c < m; ++c) {
    if (!(taus[c] > 0.0 && taus[c] < 1.0)) return fail(h, KQR_INVALID_ARG, "every tau must be in (0, 1)");
    if (!(lambdas[c] > 0.0) || !std::isfinite(lambdas[c])) return fail(h, KQR_INVALID_ARG, "every lambda must be positive");
  }
  return KQR_OK;
}

}  // namespace kqr

using namespace kqr;

extern "C" kqr_status kqr_solve_grid(kqr_handle* kh, int64_t m, const double* taus, const double* lambdas, double tol,
                                     double* alpha, double* beta, double* kkt, int32_t* status, kqr_info* info) {
  if (!kh) return KQR_INVALID_ARG;
  Handle* h = &kh->h;
  KQR_SINGLE(h);
  kqr_status s = check_grid_args(h, m, taus, lambdas, tol);
  if (s != KQR_OK) return s;
  return solve_grid(h, m, taus, lambdas, tol, alpha, beta, kkt, status, info);
}

extern "C" kqr_status kqr_solve_grid_batch(kqr_handle* const* hs, int64_t B, int64_t m, const double* taus,
                                           const double* lambdas, double tol, int32_t workers, double* alpha,
                                           double* beta, double* kkt, int32_t* status) {
  if (!hs || B < 1) return KQR_INVALID_ARG;
  for (int64_t b = 0; b < B; ++b) {
    if (!hs[b]) return KQR_INVALID_ARG;
    Handle* h = &hs[b]->h;
    if (h->batch) return fail(h, KQR_INVALID_ARG, "this call takes single-problem handles");
    kqr_status s = check_grid_args(h, m, taus, lambdas, tol);
    if (s != KQR_OK) return s;
  }
  std::vector<int64_t> off(B + 1, 0);
  for (int64_t b = 0; b < B; ++b) off[b + 1] = off[b] + hs[b]->h.n;
  const int nw = (int)std::max<int64_t>(1, std::min<int64_t>(workers > 0 ? workers : 4, B));
  std::vector<kqr_status> res(B, KQR_OK);
  std::mutex mu;
  int64_t next = 0;
  int dev = 0;
  cudaGetDevice(&dev);
  std::vector<std::thread> pool;
  for (int w = 0; w < nw; ++w) {
    pool.emplace_back([&]() {
      cudaSetDevice(dev);
      for (;;) {
        int64_t b;
        {
          std::lock_guard<std::mutex> lk(mu);
          if (next >= B) return;
          b = next++;
        }
        Handle* h = &hs[b]->h;
        res[b] = solve_grid(h, m, taus, lambdas, tol, alpha ? alpha + off[b] * m : nullptr, beta ? beta + b * m : nullptr,
                            kkt ? kkt + b * m : nullptr, status ? status + b * m : nullptr, nullptr);
      }
    });
  }
  for (auto& t : pool) t.join();
  for (int64_t b = 0; b < B; ++b)
    if (res[b] != KQR_OK) return res[b];
  return KQR_OK;
}
