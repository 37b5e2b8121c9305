// gp_server: a device-resident request loop with continuous batching.
//
// Serving side of the exact-GP path (Eq. pred: predictive mean
// K(X',X) K-hat^{-1} y with the trained alpha = K-hat^{-1} y resident on the
// device; Sec. 3.1-3.2 for the solves that produce alpha).
//
// * Each resident model owns a context (stream + workspace) and a batching
//   thread.  The thread takes every predict request queued for its model (up
//   to a row budget), packs their feature rows into one pinned block, and
//   runs ONE fused K(X',X) alpha launch for all of them; requests that arrive
//   while a batch is on the GPU join the next batch.  Models run on separate
//   streams, so batches of different models overlap on the device.
// * Solve requests (a new model's alpha) run on their own context and stream
//   and overlap with the predict batches.  A solve is admitted when the
//   device's free memory covers its estimated footprint plus the configured
//   reserve; otherwise it waits (bounded) for memory to free up.
// * A molecule request (Sec. 2.1: E_corr is the sum of the pair energies)
//   is split into one part per model (its diagonal and off-diagonal pair
//   rows); the parts join their models' batches like predict requests, and
//   each batch computes, besides the means, the parts' sums: 1^T K(X',X') 1
//   over the part's rows and R^T K(X, X') 1 from the model's variance cache,
//   so that the variance of the part's sum is the first minus |the second|^2.
//   The molecule completes with its last part: E_corr = the two sums of
//   means, its variance = the two variances (independent GPs).
// * Every request records submit and completion times (steady clock); the
//   caller reads its latency from gp_server_wait.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "gp_internal.cuh"

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
  uint64_t ticket = 0;
  int kind = 0;               // 0 predict, 1 solve, 2 molecule part, 3 molecule
  int model = -1;
  // predict (kind 0) and one model's part of a molecule (kind 2)
  const float* xp = nullptr;  // host, M x d
  int64_t m = 0;
  float* mean = nullptr;      // host, M (kind 0)
  float* var = nullptr;       // host, M, nullable (kind 0; needs the model's cache)
  double sum_mean = 0.0;      // kind 2: sum of the means over the rows
  double sum_var = 0.0;       // kind 2: variance of that sum (cache)
  Request* parent = nullptr;  // kind 2: the molecule request (kind 3)
  // molecule (kind 3): completes when both parts are done
  int pending = 0;
  double* energy = nullptr;   // host, 2: E_corr mean and variance
  std::unique_ptr<Request> part[2];
  // solve
  const float* x = nullptr;   // host, N x d
  const float* y = nullptr;   // host, N
  int64_t n = 0;
  int d = 0;
  std::vector<double> ell;
  double s = 1.0, sigma2 = 1e-4, tol = 1e-4;
  int k = 0, max_iter = 1000;
  float* alpha = nullptr;     // host, N
  // completion
  int status = GP_OK;
  bool done = false;
  Clock::time_point t_submit, t_done;
};

struct Slot {
  gp_ctx* ctx = nullptr;
  gp_model* model = nullptr;
  int d = 0;
  std::deque<Request*> queue;
  std::thread worker;
  // packed batch buffers (grown on demand): features, means, variances
  float* h_x = nullptr;
  float* h_mean = nullptr;
  float* h_var = nullptr;
  float* d_x = nullptr;
  float* d_mean = nullptr;
  float* d_var = nullptr;
  int64_t cap_rows = 0;
  // molecule parts of a batch: row offsets (device and pinned host) and the
  // per-part sums (FP64): [0] 1^T K(X',X') 1, [1..kc] R^T K(X, X') 1
  int64_t* d_seg = nullptr;
  int64_t* h_seg = nullptr;
  double* d_sums = nullptr;
  double* h_sums = nullptr;
  int cap_segs = 0;
};

}  // namespace

struct gp_server {
  int device = 0;
  int64_t max_rows = 1 << 16;
  double reserve = 0.0;
  std::mutex mu;
  std::condition_variable cv;       // new work or shutdown
  std::condition_variable cv_done;  // a request completed
  bool stop = false;
  uint64_t next_ticket = 1;
  std::unordered_map<uint64_t, std::unique_ptr<Request>> reqs;
  std::vector<std::unique_ptr<Slot>> slots;
  std::deque<Request*> solves;
  std::thread solver;
  gp_ctx* solve_ctx = nullptr;
  int64_t batches = 0, predicted = 0;
  std::string err;
};

namespace {

void finish(gp_server* srv, Request* r, int status) {
  std::lock_guard<std::mutex> lk(srv->mu);
  r->status = status;
  r->t_done = Clock::now();
  r->done = true;
  if (Request* mol = r->parent) {
    // a molecule completes with its last part: E_corr and its variance are
    // the sums over the diagonal and off-diagonal models (independent GPs)
    if (status != GP_OK) mol->status = status;
    if (--mol->pending == 0) {
      if (mol->status == GP_OK) {
        mol->energy[0] = mol->part[0]->sum_mean + mol->part[1]->sum_mean;
        mol->energy[1] = mol->part[0]->sum_var + mol->part[1]->sum_var;
      }
      mol->t_done = r->t_done;
      mol->done = true;
    }
  }
  srv->cv_done.notify_all();
}

int grow(Slot* sl, int64_t rows, int segs) {
  if (rows > sl->cap_rows) {
    int64_t cap = std::max<int64_t>(rows, 2 * sl->cap_rows);
    cudaFreeHost(sl->h_x);
    cudaFreeHost(sl->h_mean);
    cudaFreeHost(sl->h_var);
    cudaFree(sl->d_x);
    cudaFree(sl->d_mean);
    cudaFree(sl->d_var);
    sl->h_x = sl->h_mean = sl->h_var = sl->d_x = sl->d_mean = sl->d_var = nullptr;
    sl->cap_rows = 0;
    if (cudaMallocHost(&sl->h_x, sizeof(float) * cap * sl->d) != cudaSuccess ||
        cudaMallocHost(&sl->h_mean, sizeof(float) * cap) != cudaSuccess ||
        cudaMallocHost(&sl->h_var, sizeof(float) * cap) != cudaSuccess ||
        cudaMalloc(&sl->d_x, sizeof(float) * cap * sl->d) != cudaSuccess ||
        cudaMalloc(&sl->d_mean, sizeof(float) * cap) != cudaSuccess ||
        cudaMalloc(&sl->d_var, sizeof(float) * cap) != cudaSuccess) {
      cudaGetLastError();
      return GP_ENOMEM;
    }
    sl->cap_rows = cap;
  }
  if (segs > sl->cap_segs) {
    const int cap = std::max(segs, 2 * sl->cap_segs);
    const int kc = std::max(sl->model->love_m, 0);
    cudaFreeHost(sl->h_seg);
    cudaFreeHost(sl->h_sums);
    cudaFree(sl->d_seg);
    cudaFree(sl->d_sums);
    sl->h_seg = sl->d_seg = nullptr;
    sl->h_sums = sl->d_sums = nullptr;
    sl->cap_segs = 0;
    if (cudaMallocHost(&sl->h_seg, sizeof(int64_t) * 2 * cap) != cudaSuccess ||
        cudaMallocHost(&sl->h_sums, sizeof(double) * (size_t)cap * (1 + kc)) != cudaSuccess ||
        cudaMalloc(&sl->d_seg, sizeof(int64_t) * 2 * cap) != cudaSuccess ||
        cudaMalloc(&sl->d_sums, sizeof(double) * (size_t)cap * (1 + kc)) != cudaSuccess) {
      cudaGetLastError();
      return GP_ENOMEM;
    }
    sl->cap_segs = cap;
  }
  return GP_OK;
}

// One batching thread per resident model.
void predict_loop(gp_server* srv, Slot* sl) {
  cudaSetDevice(srv->device);
  const int kc = sl->model->love_m;
  for (;;) {
    std::vector<Request*> batch;
    int64_t rows = 0, max_part = 0;
    int nseg = 0;
    bool want_var = false;
    {
      std::unique_lock<std::mutex> lk(srv->mu);
      srv->cv.wait(lk, [&] { return srv->stop || !sl->queue.empty(); });
      if (srv->stop && sl->queue.empty()) return;
      // continuous batching: everything queued now, up to the row budget
      while (!sl->queue.empty()) {
        Request* r = sl->queue.front();
        if (!batch.empty() && rows + r->m > srv->max_rows) break;
        batch.push_back(r);
        rows += r->m;
        if (r->kind == 2) {
          ++nseg;
          max_part = std::max(max_part, r->m);
        } else if (r->var) {
          want_var = true;
        }
        sl->queue.pop_front();
      }
    }
    int rc = grow(sl, rows, nseg);
    if (rc == GP_OK) {
      int64_t off = 0;
      int si = 0;
      for (Request* r : batch) {
        std::memcpy(sl->h_x + off * sl->d, r->xp, sizeof(float) * r->m * sl->d);
        if (r->kind == 2) {
          sl->h_seg[2 * si] = off;
          sl->h_seg[2 * si + 1] = off + r->m;
          ++si;
        }
        off += r->m;
      }
      cudaStream_t st = sl->ctx->stream;
      if (cudaMemcpyAsync(sl->d_x, sl->h_x, sizeof(float) * rows * sl->d, cudaMemcpyHostToDevice, st) !=
              cudaSuccess ||
          (nseg > 0 && cudaMemcpyAsync(sl->d_seg, sl->h_seg, sizeof(int64_t) * 2 * nseg, cudaMemcpyHostToDevice,
                                       st) != cudaSuccess))
        rc = GP_ECUDA;
      if (rc == GP_OK)
        rc = gp::serve_batch(sl->ctx, sl->model, sl->d_x, rows, sl->d_mean, want_var ? sl->d_var : nullptr, nseg,
                             sl->d_seg, sl->d_sums, max_part);
      if (rc == GP_OK &&
          (cudaMemcpyAsync(sl->h_mean, sl->d_mean, sizeof(float) * rows, cudaMemcpyDeviceToHost, st) !=
               cudaSuccess ||
           (want_var &&
            cudaMemcpyAsync(sl->h_var, sl->d_var, sizeof(float) * rows, cudaMemcpyDeviceToHost, st) != cudaSuccess) ||
           (nseg > 0 && cudaMemcpyAsync(sl->h_sums, sl->d_sums, sizeof(double) * (size_t)nseg * (1 + kc),
                                        cudaMemcpyDeviceToHost, st) != cudaSuccess)))
        rc = GP_ECUDA;
      if (rc == GP_OK && cudaStreamSynchronize(st) != cudaSuccess) rc = GP_ECUDA;
      if (rc == GP_OK) rc = gp::check_status(sl->ctx);
      if (rc == GP_OK) {
        off = 0;
        si = 0;
        for (Request* r : batch) {
          if (r->kind == 2) {
            double ms = 0.0;
            for (int64_t i = 0; i < r->m; ++i) ms += (double)sl->h_mean[off + i];
            const double* sm = sl->h_sums + (size_t)si * (1 + kc);
            double quad = 0.0;
            for (int j = 0; j < kc; ++j) quad += sm[1 + j] * sm[1 + j];
            r->sum_mean = ms;
            r->sum_var = sm[0] - quad;
            ++si;
          } else {
            std::memcpy(r->mean, sl->h_mean + off, sizeof(float) * r->m);
            if (r->var) std::memcpy(r->var, sl->h_var + off, sizeof(float) * r->m);
          }
          off += r->m;
        }
      }
    }
    {
      std::lock_guard<std::mutex> lk(srv->mu);
      srv->batches++;
      srv->predicted += (int64_t)batch.size();
    }
    for (Request* r : batch) finish(srv, r, rc);
  }
}

// Device bytes a solve of N rows needs (features, preconditioner, CG state).
double solve_bytes(int64_t n, int d, int k) {
  const double np = (double)((n + 255) / 256 * 256);
  const double dp = (double)((d + 31) / 32 * 32);
  return np * dp * 4.0 * 4.0           // X copy, X~, hi, lo
         + np * (double)k * 12.0       // L (FP64) + FP32 copy
         + np * 4.0 * 12.0             // y, alpha, CG vectors, Woodbury scratch
         + 64.0 * 1024 * 1024;         // small buffers and slack
}

void solve_loop(gp_server* srv) {
  cudaSetDevice(srv->device);
  for (;;) {
    Request* r = nullptr;
    {
      std::unique_lock<std::mutex> lk(srv->mu);
      srv->cv.wait(lk, [&] { return srv->stop || !srv->solves.empty(); });
      if (srv->stop && srv->solves.empty()) return;
      r = srv->solves.front();
      srv->solves.pop_front();
    }
    // admission by free device memory (bounded wait: ~60 s)
    const double need = solve_bytes(r->n, r->d, r->k) + srv->reserve;
    int rc = GP_ENOMEM;
    for (int tries = 0; tries < 60000; ++tries) {
      size_t fr = 0, tot = 0;
      if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
        cudaGetLastError();
        rc = GP_ECUDA;
        break;
      }
      if ((double)fr >= need) {
        rc = GP_OK;
        break;
      }
      std::this_thread::sleep_for(std::chrono::milliseconds(1));
    }
    float *dx = nullptr, *dy = nullptr;
    gp_model* m = nullptr;
    if (rc == GP_OK) {
      if (cudaMalloc(&dx, sizeof(float) * r->n * r->d) != cudaSuccess ||
          cudaMalloc(&dy, sizeof(float) * r->n) != cudaSuccess) {
        cudaGetLastError();
        rc = GP_ENOMEM;
      }
    }
    cudaStream_t st = srv->solve_ctx->stream;
    if (rc == GP_OK &&
        (cudaMemcpyAsync(dx, r->x, sizeof(float) * r->n * r->d, cudaMemcpyHostToDevice, st) != cudaSuccess ||
         cudaMemcpyAsync(dy, r->y, sizeof(float) * r->n, cudaMemcpyHostToDevice, st) != cudaSuccess))
      rc = GP_ECUDA;
    if (rc == GP_OK) {
      gp_theta th{r->ell.data(), r->s, r->sigma2};
      rc = gp_model_fit(srv->solve_ctx, dx, r->n, r->d, &th, dy, r->k, GP_PC_RESID, 1, r->tol, r->max_iter,
                        GP_STOP_RECURRENCE,
                        GP_FP32_SPLIT_TF32, &m, nullptr);
    }
    if (rc == GP_OK) {
      if (cudaMemcpyAsync(r->alpha, m->alpha, sizeof(float) * r->n, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
          cudaStreamSynchronize(st) != cudaSuccess)
        rc = GP_ECUDA;
    }
    if (m) gp_model_free(m);
    cudaFree(dx);
    cudaFree(dy);
    finish(srv, r, rc);
  }
}

int srv_err(gp_server* srv, int code, const char* msg) {
  if (srv) {
    std::lock_guard<std::mutex> lk(srv->mu);
    srv->err = msg;
  }
  return code;
}

}  // namespace

extern "C" {

int gp_server_create(gp_server** out, int device, int64_t max_batch_rows, double reserve_bytes) {
  if (!out || max_batch_rows < 1 || !(reserve_bytes >= 0.0)) return GP_EINVAL;
  *out = nullptr;
  auto* srv = new gp_server();
  srv->device = device;
  srv->max_rows = max_batch_rows;
  srv->reserve = reserve_bytes;
  cudaStream_t st = nullptr;
  if (cudaSetDevice(device) != cudaSuccess ||
      cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    delete srv;
    return GP_ECUDA;
  }
  if (gp_create(&srv->solve_ctx, device, st) != GP_OK) {
    cudaStreamDestroy(st);
    delete srv;
    return GP_ECUDA;
  }
  srv->solver = std::thread(solve_loop, srv);
  *out = srv;
  return GP_OK;
}

int gp_server_add_model(gp_server* srv, const float* X, int64_t N, int d, const gp_theta* theta,
                        const float* y, int k, int precond, double tol, int max_iter, int precision,
                        int var_rank, int* model_id) {
  if (!srv || !model_id || var_rank < 0 || var_rank > GP_VAR_CACHE_MAX_RANK) return GP_EINVAL;
  auto sl = std::make_unique<Slot>();
  sl->d = d;
  cudaStream_t st = nullptr;
  if (cudaSetDevice(srv->device) != cudaSuccess ||
      cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    return srv_err(srv, GP_ECUDA, "stream creation failed");
  }
  if (gp_create(&sl->ctx, srv->device, st) != GP_OK) {
    cudaStreamDestroy(st);
    return srv_err(srv, GP_ECUDA, "context creation failed");
  }
  int rc = gp_model_fit(sl->ctx, X, N, d, theta, y, k, precond, 1, tol, max_iter, GP_STOP_RECURRENCE, precision,
                        &sl->model,
                        nullptr);
  if (rc == GP_OK && var_rank > 0) {
    // the variance cache, started at K-hat a (= y up to the fit's tolerance)
    int got = 0;
    rc = gp_model_variance_cache(sl->ctx, sl->model, nullptr, std::min<int64_t>(var_rank, N), &got);
  }
  if (rc != GP_OK) {
    std::string msg = gp_last_error(sl->ctx);
    if (sl->model) gp_model_free(sl->model);
    gp_destroy(sl->ctx);
    cudaStreamDestroy(st);
    return srv_err(srv, rc, msg.c_str());
  }
  std::lock_guard<std::mutex> lk(srv->mu);
  *model_id = (int)srv->slots.size();
  Slot* raw = sl.get();
  srv->slots.push_back(std::move(sl));
  raw->worker = std::thread(predict_loop, srv, raw);
  return GP_OK;
}

int gp_server_predict(gp_server* srv, int model_id, const float* Xp, int64_t M, float* mean, float* var,
                      uint64_t* ticket) {
  if (!srv || !Xp || M < 1 || !mean || !ticket) return GP_EINVAL;
  std::lock_guard<std::mutex> lk(srv->mu);
  if (model_id < 0 || model_id >= (int)srv->slots.size() || srv->stop) return GP_EINVAL;
  if (M > srv->max_rows) return GP_EINVAL;
  if (var && !srv->slots[model_id]->model->love_R) return GP_EINVAL;
  auto r = std::make_unique<Request>();
  r->ticket = srv->next_ticket++;
  r->kind = 0;
  r->model = model_id;
  r->xp = Xp;
  r->m = M;
  r->mean = mean;
  r->var = var;
  r->t_submit = Clock::now();
  srv->slots[model_id]->queue.push_back(r.get());
  *ticket = r->ticket;
  srv->reqs.emplace(r->ticket, std::move(r));
  srv->cv.notify_all();
  return GP_OK;
}

int gp_server_molecule(gp_server* srv, int diag_model, const float* Xd, int64_t Md, int off_model,
                       const float* Xo, int64_t Mo, double* energy, uint64_t* ticket) {
  if (!srv || !Xd || Md < 1 || Mo < 0 || (Mo > 0 && !Xo) || !energy || !ticket) return GP_EINVAL;
  std::lock_guard<std::mutex> lk(srv->mu);
  const int ns = (int)srv->slots.size();
  if (srv->stop || diag_model < 0 || diag_model >= ns || off_model < 0 || off_model >= ns) return GP_EINVAL;
  if (Md > srv->max_rows || Mo > srv->max_rows) return GP_EINVAL;
  if (!srv->slots[diag_model]->model->love_R || (Mo > 0 && !srv->slots[off_model]->model->love_R))
    return GP_EINVAL;
  auto mol = std::make_unique<Request>();
  mol->kind = 3;
  mol->energy = energy;
  mol->ticket = srv->next_ticket++;
  mol->t_submit = Clock::now();
  const int models[2] = {diag_model, off_model};
  const float* xs[2] = {Xd, Xo};
  const int64_t ms[2] = {Md, Mo};
  for (int i = 0; i < 2; ++i) {
    auto part = std::make_unique<Request>();
    part->kind = 2;
    part->model = models[i];
    part->xp = xs[i];
    part->m = ms[i];
    part->parent = mol.get();
    part->t_submit = mol->t_submit;
    if (ms[i] > 0) {
      mol->pending++;
      srv->slots[models[i]]->queue.push_back(part.get());
    }
    mol->part[i] = std::move(part);
  }
  *ticket = mol->ticket;
  srv->reqs.emplace(mol->ticket, std::move(mol));
  srv->cv.notify_all();
  return GP_OK;
}

int gp_server_solve(gp_server* srv, const float* X, int64_t N, int d, const gp_theta* theta,
                    const float* y, int k, double tol, int max_iter, float* alpha, uint64_t* ticket) {
  if (!srv || !X || N < 1 || d < 1 || !theta || !theta->lengthscale || !y || k < 0 || k > N ||
      !(tol > 0.0) || max_iter < 1 || !alpha || !ticket)
    return GP_EINVAL;
  auto r = std::make_unique<Request>();
  r->kind = 1;
  r->x = X;
  r->y = y;
  r->n = N;
  r->d = d;
  r->ell.assign(theta->lengthscale, theta->lengthscale + d);
  r->s = theta->outputscale;
  r->sigma2 = theta->sigma2;
  r->k = k;
  r->tol = tol;
  r->max_iter = max_iter;
  r->alpha = alpha;
  std::lock_guard<std::mutex> lk(srv->mu);
  if (srv->stop) return GP_EINVAL;
  r->ticket = srv->next_ticket++;
  r->t_submit = Clock::now();
  srv->solves.push_back(r.get());
  *ticket = r->ticket;
  srv->reqs.emplace(r->ticket, std::move(r));
  srv->cv.notify_all();
  return GP_OK;
}

int gp_server_wait(gp_server* srv, uint64_t ticket, double timeout_s, double* latency_ms) {
  if (!srv || !(timeout_s >= 0.0)) return GP_EINVAL;
  std::unique_lock<std::mutex> lk(srv->mu);
  auto it = srv->reqs.find(ticket);
  if (it == srv->reqs.end()) return GP_EINVAL;
  Request* r = it->second.get();
  const bool ok = srv->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), [&] { return r->done; });
  if (!ok) return GP_ETIMEOUT;
  const int status = r->status;
  if (latency_ms) latency_ms[0] = std::chrono::duration<double, std::milli>(r->t_done - r->t_submit).count();
  srv->reqs.erase(it);
  return status;
}

int gp_server_stats(gp_server* srv, int64_t* batches, int64_t* predicted) {
  if (!srv) return GP_EINVAL;
  std::lock_guard<std::mutex> lk(srv->mu);
  if (batches) *batches = srv->batches;
  if (predicted) *predicted = srv->predicted;
  return GP_OK;
}

const char* gp_server_last_error(gp_server* srv) { return srv ? srv->err.c_str() : "null server"; }

void gp_server_destroy(gp_server* srv) {
  if (!srv) return;
  {
    std::lock_guard<std::mutex> lk(srv->mu);
    srv->stop = true;
    srv->cv.notify_all();
  }
  for (auto& sl : srv->slots)
    if (sl->worker.joinable()) sl->worker.join();
  if (srv->solver.joinable()) srv->solver.join();
  cudaSetDevice(srv->device);
  for (auto& sl : srv->slots) {
    cudaStream_t st = sl->ctx ? sl->ctx->stream : nullptr;
    if (sl->model) gp_model_free(sl->model);
    if (sl->ctx) gp_destroy(sl->ctx);
    if (st) cudaStreamDestroy(st);
    cudaFreeHost(sl->h_x);
    cudaFreeHost(sl->h_mean);
    cudaFreeHost(sl->h_var);
    cudaFreeHost(sl->h_seg);
    cudaFreeHost(sl->h_sums);
    cudaFree(sl->d_x);
    cudaFree(sl->d_mean);
    cudaFree(sl->d_var);
    cudaFree(sl->d_seg);
    cudaFree(sl->d_sums);
  }
  cudaStream_t sst = srv->solve_ctx ? srv->solve_ctx->stream : nullptr;
  if (srv->solve_ctx) gp_destroy(srv->solve_ctx);
  if (sst) cudaStreamDestroy(sst);
  delete srv;
}

}  // extern "C"
