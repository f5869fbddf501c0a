// batch.cu -- continuous-batching server for many independent lattices (the
// lbm_batch_* calls of include/ctulbm.h).  Host code only: it is a client of
// the single-lattice C ABI (lbm_create, lbm_init_rho_u, lbm_step_many,
// lbm_diagnostics, lbm_moments, lbm_destroy) driven by one worker thread; it
// asks the library's internals only how many batched CTAs fit on an SM.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include <cuda_runtime.h>

#include "ctulbm.h"
#include "lbm_internal.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Job {
  int64_t id = 0;
  lbm_params p{};
  std::vector<double> init;  // rho, ux, uy until admitted
  std::vector<double> out;   // final rho, ux, uy once done (until fetched)
  int64_t nsteps = 0, diag_every = 0;
  double threshold = 0.0;
  size_t bytes = 0;
  lbm_handle* h = nullptr;
  lbm_job_result r{};
};

size_t footprint(const lbm_params& p) {
  const size_t n = (size_t)p.Lx * (size_t)p.Ly;
  const size_t elem = p.precision == LBM_FP64 ? 8 : (p.precision == LBM_FP16_SHIFTED ? 2 : 4);
  return 32 * elem * n + 24 * n + 4096;  // two buffers of 16 planes, FP64 work planes, small state
}

}  // namespace

struct lbm_batch {
  size_t max_bytes = 0;
  int chunk = 1;
  long long fill_nodes = 0;  // lattice nodes per launch that keep every SM busy
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  Clock::time_point t0;

  std::mutex mu;
  std::condition_variable cv;       // worker: new work or stop; waiters: job state changes
  bool stop = false;
  int64_t next_id = 0;
  std::deque<Job*> pending;         // submission order
  std::vector<Job*> active;         // owned by the worker between scheduling decisions
  std::map<int64_t, std::unique_ptr<Job>> jobs;
  size_t used = 0;
  int64_t node_updates = 0, launches = 0, done = 0, failed = 0;
  std::thread worker;

  double now() const { return std::chrono::duration<double>(Clock::now() - t0).count(); }
  void run();
  void finish(Job* j, int error);   // called with mu held
};

// Called with mu held: release the job's device memory and record its end.
void lbm_batch::finish(Job* j, int error) {
  if (j->h) lbm_destroy(j->h);
  j->h = nullptr;
  used -= j->bytes;
  j->r.error = error;
  j->r.status = error == LBM_OK ? LBM_JOB_DONE : LBM_JOB_FAILED;
  j->r.t_finish = now();
  if (error == LBM_OK)
    ++done;
  else
    ++failed;
}

void lbm_batch::run() {
  cudaSetDevice(device);
  for (;;) {
    std::vector<Job*> admitted;
    {
      std::unique_lock<std::mutex> lk(mu);
      // admit in submission order while the head of the queue fits
      for (;;) {
        while (!stop && pending.empty() && active.empty()) cv.wait(lk);
        if (stop) return;
        while (!pending.empty() && used + pending.front()->bytes <= max_bytes) {
          Job* j = pending.front();
          pending.pop_front();
          used += j->bytes;
          j->r.status = LBM_JOB_ACTIVE;
          j->r.t_start = now();
          admitted.push_back(j);
        }
        if (!admitted.empty() || !active.empty()) break;
        cv.wait(lk);  // the head does not fit yet and nothing runs: wait (cannot happen, see submit)
      }
    }
    // device work without the lock: create and initialise the admitted jobs
    for (Job* j : admitted) {
      int e = lbm_create(&j->p, stream, &j->h);
      const size_t n = (size_t)j->p.Lx * j->p.Ly;
      if (e == LBM_OK) e = lbm_init_rho_u(j->h, j->init.data(), j->init.data() + n,
                                          j->init.data() + 2 * n);
      std::lock_guard<std::mutex> lk(mu);
      std::vector<double>().swap(j->init);
      if (e != LBM_OK)
        finish(j, e);
      else
        active.push_back(j);
      cv.notify_all();
    }
    if (active.empty()) continue;
    // shortest remaining work first: advance the resident jobs with the fewest
    // node-steps left, just enough of them to fill the GPU; the others stay
    // resident and wait (short jobs finish early instead of crawling at the
    // pace of the largest lattice in the batch)
    std::vector<Job*> order(active), run, idle;
    auto left_work = [](const Job* j) {
      return (double)(j->nsteps - j->r.steps_done) * j->p.Lx * j->p.Ly;
    };
    std::stable_sort(order.begin(), order.end(),
                     [&](const Job* a, const Job* b) { return left_work(a) < left_work(b); });
    long long nodes = 0;
    for (Job* j : order) {
      if (!run.empty() && nodes >= fill_nodes)
        idle.push_back(j);
      else {
        run.push_back(j);
        nodes += (long long)j->p.Lx * j->p.Ly;
      }
    }
    // steps until the next event (a diagnostics record or a job's end)
    int64_t k = chunk;
    for (Job* j : run) {
      const int64_t left = j->nsteps - j->r.steps_done;
      k = left < k ? left : k;
      if (j->diag_every > 0) {
        const int64_t to_diag = j->diag_every - j->r.steps_done % j->diag_every;
        k = to_diag < k ? to_diag : k;
      }
    }
    std::vector<lbm_handle*> hs;
    for (Job* j : run) hs.push_back(j->h);
    const int e = lbm_step_many(hs.data(), (int32_t)hs.size(), k);
    std::vector<Job*> keep(idle);
    std::vector<std::pair<Job*, int>> ended;
    for (Job* j : run) {
      if (e != LBM_OK) {
        ended.emplace_back(j, e);
        continue;
      }
      const int64_t s = j->r.steps_done + k;
      const bool end = s >= j->nsteps;
      const bool rec = end || (j->diag_every > 0 && s % j->diag_every == 0);
      lbm_diag d{};
      int ej = LBM_OK;
      if (rec) ej = lbm_diagnostics(j->h, j->threshold, 0.0, &d);
      if (ej == LBM_OK) ej = lbm_sync(j->h);
      std::vector<double> out;
      if (ej == LBM_OK && end) {
        const size_t n = (size_t)j->p.Lx * j->p.Ly;
        out.resize(3 * n);
        ej = lbm_moments(j->h, out.data(), out.data() + n, out.data() + 2 * n);
      }
      std::lock_guard<std::mutex> lk(mu);
      j->r.steps_done = s;
      node_updates += (int64_t)j->p.Lx * j->p.Ly * k;
      if (rec && ej == LBM_OK) {
        j->r.diag = d;
        j->r.diag_step = s;
      }
      if (ej != LBM_OK) {
        ended.emplace_back(j, ej);
      } else if (end) {
        j->out.swap(out);
        ended.emplace_back(j, LBM_OK);
      } else {
        keep.push_back(j);
      }
    }
    std::lock_guard<std::mutex> lk(mu);
    ++launches;
    for (auto& je : ended) finish(je.first, je.second);
    active.swap(keep);
    cv.notify_all();
  }
}

extern "C" {

int lbm_batch_create(size_t max_bytes, int32_t chunk_steps, void* cuda_stream, lbm_batch** out) {
  if (!out || max_bytes == 0 || chunk_steps < 1) return LBM_ERR_INVALID_ARG;
  *out = nullptr;
  std::unique_ptr<lbm_batch> b(new (std::nothrow) lbm_batch());
  if (!b) return LBM_ERR_OOM;
  b->max_bytes = max_bytes;
  b->chunk = chunk_steps;
  b->t0 = Clock::now();
  if (cudaGetDevice(&b->device) != cudaSuccess) return LBM_ERR_CUDA;
  int nsm = 0;
  if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, b->device) != cudaSuccess)
    return LBM_ERR_CUDA;
  // the batched kernel's resident CTAs per SM (CTU2 + MC, FP32 storage), two
  // work items of 96 rows x 56 columns each
  int occ = ctulbm::step_batch_occupancy_f32(2, 0, false, ctulbm::step_smem_bytes(4, 4));
  if (occ < 1) occ = 2;
  b->fill_nodes = (long long)nsm * occ * 2 * 96 * 56;
  b->stream = static_cast<cudaStream_t>(cuda_stream);
  if (!b->stream) {
    if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess)
      return LBM_ERR_CUDA;
    b->own_stream = true;
  }
  try {
    b->worker = std::thread([p = b.get()] { p->run(); });
  } catch (...) {
    if (b->own_stream) cudaStreamDestroy(b->stream);
    return LBM_ERR_OOM;
  }
  *out = b.release();
  return LBM_OK;
}

void lbm_batch_destroy(lbm_batch* b) {
  if (!b) return;
  {
    std::lock_guard<std::mutex> lk(b->mu);
    b->stop = true;
  }
  b->cv.notify_all();
  if (b->worker.joinable()) b->worker.join();
  for (auto& kv : b->jobs)
    if (kv.second->h) lbm_destroy(kv.second->h);
  if (b->own_stream) cudaStreamDestroy(b->stream);
  delete b;
}

int64_t lbm_batch_submit(lbm_batch* b, const lbm_params* p, const double* rho, const double* ux,
                         const double* uy, int64_t nsteps, int64_t diag_every, double threshold) {
  if (!b || !p || !rho || !ux || !uy || nsteps < 1 || diag_every < 0) return LBM_ERR_INVALID_ARG;
  if (p->Lx < 1 || p->Ly < 1 || (long long)p->Lx * p->Ly > (1LL << 31) - 1)
    return LBM_ERR_INVALID_ARG;
  const size_t bytes = footprint(*p);
  if (bytes > b->max_bytes) return LBM_ERR_OOM;
  std::unique_ptr<Job> j(new (std::nothrow) Job());
  if (!j) return LBM_ERR_OOM;
  const size_t n = (size_t)p->Lx * p->Ly;
  try {
    j->init.resize(3 * n);
  } catch (...) {
    return LBM_ERR_OOM;
  }
  std::memcpy(j->init.data(), rho, n * sizeof(double));
  std::memcpy(j->init.data() + n, ux, n * sizeof(double));
  std::memcpy(j->init.data() + 2 * n, uy, n * sizeof(double));
  j->p = *p;
  j->nsteps = nsteps;
  j->diag_every = diag_every;
  j->threshold = threshold;
  j->bytes = bytes;
  j->r.status = LBM_JOB_PENDING;
  j->r.error = LBM_OK;
  j->r.nsteps = nsteps;
  j->r.diag_step = -1;
  j->r.t_start = j->r.t_finish = -1.0;
  std::lock_guard<std::mutex> lk(b->mu);
  j->id = b->next_id++;
  j->r.t_submit = b->now();
  Job* raw = j.get();
  b->jobs.emplace(raw->id, std::move(j));
  b->pending.push_back(raw);
  b->cv.notify_all();
  return raw->id;
}

int lbm_batch_poll(lbm_batch* b, int64_t job, lbm_job_result* out) {
  if (!b || !out) return LBM_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(b->mu);
  auto it = b->jobs.find(job);
  if (it == b->jobs.end()) return LBM_ERR_INVALID_ARG;
  *out = it->second->r;
  return LBM_OK;
}

int lbm_batch_wait(lbm_batch* b, int64_t job, double timeout_s, lbm_job_result* out) {
  if (!b) return LBM_ERR_INVALID_ARG;
  std::unique_lock<std::mutex> lk(b->mu);
  auto finished = [&]() -> int {  // 1 done, 0 not yet, -1 unknown job
    if (job < 0) {
      for (auto& kv : b->jobs)
        if (kv.second->r.status < LBM_JOB_DONE) return 0;
      return 1;
    }
    auto it = b->jobs.find(job);
    if (it == b->jobs.end()) return -1;
    return it->second->r.status >= LBM_JOB_DONE ? 1 : 0;
  };
  int f = finished();
  if (f < 0) return LBM_ERR_INVALID_ARG;
  if (timeout_s < 0) {
    b->cv.wait(lk, [&] { return finished() != 0; });
  } else if (!b->cv.wait_for(lk, std::chrono::duration<double>(timeout_s),
                             [&] { return finished() != 0; })) {
    return LBM_ERR_TIMEOUT;
  }
  if (out && job >= 0) *out = b->jobs[job]->r;
  return LBM_OK;
}

int lbm_batch_fetch(lbm_batch* b, int64_t job, double* rho, double* ux, double* uy) {
  if (!b) return LBM_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(b->mu);
  auto it = b->jobs.find(job);
  if (it == b->jobs.end()) return LBM_ERR_INVALID_ARG;
  Job* j = it->second.get();
  if (j->r.status != LBM_JOB_DONE || j->out.empty()) return LBM_ERR_INVALID_ARG;
  const size_t n = (size_t)j->p.Lx * j->p.Ly;
  if (rho) std::memcpy(rho, j->out.data(), n * sizeof(double));
  if (ux) std::memcpy(ux, j->out.data() + n, n * sizeof(double));
  if (uy) std::memcpy(uy, j->out.data() + 2 * n, n * sizeof(double));
  std::vector<double>().swap(j->out);
  return LBM_OK;
}

int lbm_batch_get_info(lbm_batch* b, lbm_batch_info* out) {
  if (!b || !out) return LBM_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(b->mu);
  out->pending = (int64_t)b->pending.size();
  out->active = (int64_t)b->active.size();
  out->done = b->done;
  out->failed = b->failed;
  out->used_bytes = (int64_t)b->used;
  out->node_updates = b->node_updates;
  out->launches = b->launches;
  return LBM_OK;
}

}  // extern "C"
