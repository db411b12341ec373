// mprk_server.cu — a request loop that batches coupled solves continuously.
//
// Requests (a configuration, an initial state and a number of slow steps)
// queue on submit. A server thread repeats:
//   1. admit queued requests in arrival order while a slot is free and the
//      HBM ledger has room: the instance is created stream-ordered on the
//      copy stream (cudaMallocAsync, upload, reference set-up);
//   2. advance every resident instance by one slow step: the instances below
//      the solo size with one persistent batched launch per precision on
//      the compute stream, the larger ones by their own stage launches on
//      side streams forked from it and joined back (a large instance fills
//      the GPU by itself, and the single-instance kernels run its tiles
//      faster than the batch kernel, which reads its arguments from shared
//      memory);
//   3. retire instances that reached their step count: the state is copied
//      to pinned host memory on the copy stream after the step's event, and
//      the buffers return to the pool with cudaFreeAsync.
// Requests therefore join and leave between slow steps while the others keep
// running (continuous batching). At most two iterations are in flight, so
// a newly admitted request starts within two slow steps. All timing uses one
// steady clock that starts when the server is created.
#include <cuda_runtime.h>

#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "mprk.h"
#include "mprk_internal.h"

using namespace mprk;

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
  uint64_t ticket = 0;
  mprk_config cfg{};
  std::vector<double> q0;      // host copy made at submit
  int n_steps = 0;
  int state = MPRK_REQ_PENDING;
  int error = 0;
  double t_submit = 0, t_admit = 0, t_finish = 0;
  long long bytes = 0;         // ledger estimate (bytes the instance allocates)
  long long cell_stages = 0;
  int steps_done = 0;
  mprk_instance* inst = nullptr;
  double* pinned = nullptr;    // result staging
  cudaEvent_t copied = nullptr;
  std::vector<double> result;
};

int sfail(int code, const std::string& msg) {
  set_last_error(msg);
  return code;
}

// Pinned host buffers for results, reused by size class (powers of two), so
// that retiring a request does not pin fresh memory each time.
struct PinnedPool {
  std::unordered_map<size_t, std::vector<void*>> free_;
  static size_t cls(size_t n) {
    size_t c = 4096;
    while (c < n) c <<= 1;
    return c;
  }
  void* get(size_t n) {
    const size_t c = cls(n);
    auto& v = free_[c];
    if (!v.empty()) {
      void* p = v.back();
      v.pop_back();
      return p;
    }
    void* p = nullptr;
    if (cudaMallocHost(&p, c) != cudaSuccess) return nullptr;
    return p;
  }
  void put(void* p, size_t n) { free_[cls(n)].push_back(p); }
  void clear() {
    for (auto& kv : free_)
      for (void* p : kv.second) cudaFreeHost(p);
    free_.clear();
  }
};

}  // namespace

struct mprk_server {
  mprk_server_config cfg{};
  Clock::time_point t0;
  std::thread th;
  std::mutex mu;
  std::condition_variable cv;
  bool stop = false;
  int thread_error = 0;
  std::string thread_msg;
  std::deque<Request*> queue;
  std::unordered_map<uint64_t, Request*> all;
  uint64_t next_ticket = 1;
  long long ledger = 0;        // bytes of admitted, not yet freed requests
  // owned by the server thread
  std::vector<Request*> resident;
  std::vector<Request*> retiring;
  cudaStream_t compute = nullptr, copy = nullptr;
  // side streams of the instances stepped alone, with the events that fork
  // them from the compute stream and join them back
  static constexpr int NSIDE = 4;
  cudaStream_t side[NSIDE] = {nullptr, nullptr, nullptr, nullptr};
  cudaEvent_t ev_fork = nullptr, ev_join[NSIDE] = {nullptr, nullptr, nullptr, nullptr};
  long long solo_cells = 0;  // instances of at least this many cells step alone (0: none)
  bool solo_fp64_only = false;  // the default threshold: FP32-flux instances all batched
  BatchRunner* runner[2] = {nullptr, nullptr};
  PinnedPool pool;
  // counters (read under mu)
  long long n_done = 0, n_failed = 0, cells_done = 0, batched_steps = 0;
  int n_resident = 0;
  // time accounting of the loop (written by the server thread under mu):
  // iterations, host seconds in admission, step launch, retirement and the
  // in-flight wait, GPU seconds of the steps, first step start and last
  // step end (server clock), admissions
  double prof[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  double first_step = -1.0;

  double now() const { return std::chrono::duration<double>(Clock::now() - t0).count(); }
};

namespace {

void finish(mprk_server* S, Request* r, int error) {
  std::lock_guard<std::mutex> lk(S->mu);
  r->error = error;
  r->state = MPRK_REQ_DONE;
  r->t_finish = S->now();
  S->ledger -= r->bytes;
  if (error) S->n_failed++;
  else S->n_done++;
}

void server_loop(mprk_server* S) {
  bool ok = cudaSetDevice(S->cfg.device) == cudaSuccess &&
            cudaStreamCreateWithFlags(&S->compute, cudaStreamNonBlocking) == cudaSuccess &&
            cudaStreamCreateWithFlags(&S->copy, cudaStreamNonBlocking) == cudaSuccess &&
            cudaEventCreateWithFlags(&S->ev_fork, cudaEventDisableTiming) == cudaSuccess;
  for (int k = 0; k < mprk_server::NSIDE && ok; k++)
    ok = cudaStreamCreateWithFlags(&S->side[k], cudaStreamNonBlocking) == cudaSuccess &&
         cudaEventCreateWithFlags(&S->ev_join[k], cudaEventDisableTiming) == cudaSuccess;
  if (!ok) {
    std::lock_guard<std::mutex> lk(S->mu);
    S->thread_error = MPRK_ECUDA;
    S->thread_msg = "server: device or stream set-up failed";
    return;
  }
  // step_ev[slot] ends iteration slot's launches; beg_ev[slot] starts them
  // (both timed, for the GPU-seconds account)
  cudaEvent_t step_ev[2] = {nullptr, nullptr}, beg_ev[2] = {nullptr, nullptr};
  if (cudaEventCreate(&step_ev[0]) != cudaSuccess || cudaEventCreate(&step_ev[1]) != cudaSuccess ||
      cudaEventCreate(&beg_ev[0]) != cudaSuccess || cudaEventCreate(&beg_ev[1]) != cudaSuccess) {
    for (cudaEvent_t e : {step_ev[0], step_ev[1], beg_ev[0], beg_ev[1]})
      if (e) cudaEventDestroy(e);
    std::lock_guard<std::mutex> lk(S->mu);
    S->thread_error = MPRK_ECUDA;
    S->thread_msg = "server: event set-up failed";
    return;
  }
  bool step_ev_used[2] = {false, false};
  int it = 0;
  // adds the GPU time of the iteration in slot (its events have completed)
  auto account = [&](int slot) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, beg_ev[slot], step_ev[slot]) == cudaSuccess) {
      std::lock_guard<std::mutex> lk(S->mu);
      S->prof[5] += ms * 1e-3;
      S->prof[6] = S->now();
    }
  };
  for (;;) {
    // ---- 1. admission --------------------------------------------------
    std::vector<Request*> admit;
    {
      std::unique_lock<std::mutex> lk(S->mu);
      if (S->stop) break;
      if (S->resident.empty() && S->retiring.empty() && S->queue.empty())
        S->cv.wait_for(lk, std::chrono::milliseconds(2));
      if (S->stop) break;
      while (!S->queue.empty() && (int)(S->resident.size() + admit.size()) < S->cfg.max_slots &&
             S->ledger + S->queue.front()->bytes <= S->cfg.hbm_budget_bytes) {
        Request* r = S->queue.front();
        S->queue.pop_front();
        S->ledger += r->bytes;
        admit.push_back(r);
      }
    }
    const double t_admit0 = S->now();
    for (Request* r : admit) {
      mprk_instance* inst = nullptr;
      const int rc = create_instance(&r->cfg, r->q0.data(), MPRK_HOST, S->copy, true, &inst);
      if (rc) {
        finish(S, r, rc);
        continue;
      }
      std::vector<double>().swap(r->q0);
      r->inst = inst;
      {
        std::lock_guard<std::mutex> lk(S->mu);
        r->state = MPRK_REQ_RUNNING;
        r->t_admit = S->now();
      }
      S->resident.push_back(r);
    }
    // instances admitted on the copy stream must be ready before the step
    if (!admit.empty()) {
      runner_invalidate(S->runner[0]);
      runner_invalidate(S->runner[1]);
      cudaEvent_t ev = nullptr;
      if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess ||
          cudaEventRecord(ev, S->copy) != cudaSuccess || cudaStreamWaitEvent(S->compute, ev, 0) != cudaSuccess)
        cudaStreamSynchronize(S->copy);  // the uploads land before the step either way
      if (ev) cudaEventDestroy(ev);
    }

    if (!admit.empty()) {
      std::lock_guard<std::mutex> lk(S->mu);
      S->prof[1] += S->now() - t_admit0;
      S->prof[7] += (double)admit.size();
    }

    // ---- 2. one batched slow step for every resident instance ------------
    if (!S->resident.empty()) {
      // keep at most two iterations in flight
      const int slot = it & 1;
      const double t_wait0 = S->now();
      if (step_ev_used[slot]) {
        cudaEventSynchronize(step_ev[slot]);
        account(slot);
      }
      const double t_step0 = S->now();
      cudaEventRecord(beg_ev[slot], S->compute);
      std::vector<mprk_instance*> group[2], alone;
      for (Request* r : S->resident) {
        if (S->solo_cells > 0 && instance_cells(r->inst) >= S->solo_cells &&
            !(S->solo_fp64_only && r->cfg.precision != MPRK_FP64))
          alone.push_back(r->inst);
        else group[r->cfg.precision == MPRK_FP64 ? 0 : 1].push_back(r->inst);
      }
      int err = 0;
      long long cells = 0;
      if (!alone.empty()) {
        // fork: each side stream starts after everything queued on the
        // compute stream so far (uploads of new instances, the previous
        // iteration's work and joins), so an instance's steps stay ordered
        // whichever side stream takes it
        const int nside = std::min((int)alone.size(), (int)mprk_server::NSIDE);
        if (cudaEventRecord(S->ev_fork, S->compute) != cudaSuccess) err = MPRK_ECUDA;
        for (int k = 0; k < nside && !err; k++)
          if (cudaStreamWaitEvent(S->side[k], S->ev_fork, 0) != cudaSuccess) err = MPRK_ECUDA;
        for (size_t j = 0; j < alone.size() && !err; j++) {
          long long cs = 0;
          const int rc = instance_step_alone(alone[j], S->side[j % nside], &cs);
          if (rc) err = rc;
          cells += cs;
        }
        // join: the compute stream (and the step event after it) waits for
        // every side stream used
        for (int k = 0; k < nside; k++)
          if (cudaEventRecord(S->ev_join[k], S->side[k]) != cudaSuccess ||
              cudaStreamWaitEvent(S->compute, S->ev_join[k], 0) != cudaSuccess)
            err = MPRK_ECUDA;
      }
      for (int p = 0; p < 2; p++) {
        if (group[p].empty()) continue;
        if (!S->runner[p]) S->runner[p] = runner_create(p, S->compute);
        long long cs = 0;
        const int rc = runner_step(S->runner[p], group[p].data(), (int)group[p].size(), &cs);
        if (rc) err = rc;
        cells += cs;
      }
      cudaEventRecord(step_ev[slot], S->compute);
      step_ev_used[slot] = true;
      it++;
      const double t_ret0 = S->now();
      {
        std::lock_guard<std::mutex> lk(S->mu);
        S->batched_steps++;
        S->cells_done += cells;
        S->prof[0] += 1.0;
        S->prof[2] += t_ret0 - t_step0;
        S->prof[4] += t_step0 - t_wait0;
        if (S->first_step < 0) S->first_step = t_step0;
      }
      // ---- 3. retire instances that reached their step count -------------
      std::vector<Request*> keep;
      for (Request* r : S->resident) {
        r->steps_done = (int)instance_steps(r->inst);
        if (err) {
          r->steps_done = 0;
        }
        if (err || r->steps_done >= r->n_steps) {
          Geom g;
          Bufs b;
          int prec;
          cudaStream_t st;
          unsigned* status;
          instance_view(r->inst, &g, &b, &prec, &st, &status);
          const size_t nbytes = (size_t)4 * g.nz * g.nx * 8;
          r->pinned = static_cast<double*>(S->pool.get(nbytes + 16));
          cudaStreamWaitEvent(S->copy, step_ev[slot], 0);
          if (r->pinned) {
            cudaMemcpy2DAsync(r->pinned, (size_t)g.nx * 8, b.qA, (size_t)g.pitch * 8, (size_t)g.nx * 8,
                              (size_t)4 * g.nz, cudaMemcpyDeviceToHost, S->copy);
            // the status word rides along behind the state
            cudaMemcpyAsync(reinterpret_cast<char*>(r->pinned) + nbytes, status, sizeof(unsigned),
                            cudaMemcpyDeviceToHost, S->copy);
          }
          r->copied = nullptr;
          if (cudaEventCreateWithFlags(&r->copied, cudaEventDisableTiming) != cudaSuccess ||
              cudaEventRecord(r->copied, S->copy) != cudaSuccess) {
            // no event to poll: wait for the copy here
            if (r->copied) cudaEventDestroy(r->copied);
            r->copied = nullptr;
            cudaStreamSynchronize(S->copy);
          }
          r->error = err;
          S->retiring.push_back(r);
        } else {
          keep.push_back(r);
        }
      }
      if (keep.size() != S->resident.size()) {
        runner_invalidate(S->runner[0]);
        runner_invalidate(S->runner[1]);
      }
      S->resident.swap(keep);
      std::lock_guard<std::mutex> lk(S->mu);
      S->n_resident = (int)S->resident.size();
      S->prof[3] += S->now() - t_ret0;
    }

    // ---- 4. complete retirements whose copies are done --------------------
    std::vector<Request*> still;
    for (Request* r : S->retiring) {
      const cudaError_t q = r->copied ? cudaEventQuery(r->copied) : cudaSuccess;
      if (q == cudaErrorNotReady) {
        still.push_back(r);
        continue;
      }
      if (r->copied) cudaEventDestroy(r->copied);
      r->copied = nullptr;
      Geom g;
      Bufs b;
      int prec;
      cudaStream_t st;
      unsigned* status;
      instance_view(r->inst, &g, &b, &prec, &st, &status);
      const size_t n = (size_t)4 * g.nz * g.nx;
      int error = r->error;
      if (!error && q != cudaSuccess) error = MPRK_ECUDA;  // the copy did not complete
      if (r->pinned) {
        r->result.assign(r->pinned, r->pinned + n);
        unsigned sw;
        memcpy(&sw, reinterpret_cast<char*>(r->pinned) + n * 8, sizeof sw);
        if (!error && (sw & ST_NONFINITE)) error = MPRK_ENONFINITE;
        if (!error && (sw & ST_TIMEOUT)) error = MPRK_ETIMEOUT;
        S->pool.put(r->pinned, n * 8 + 16);
        r->pinned = nullptr;
      } else if (!error) {
        error = MPRK_ENOMEM;
      }
      long long cs_per_step = 0;
      const mprk_config& c = r->cfg;
      const long long s = c.base == MPRK_BASE_RK4 ? 4 : (c.base == MPRK_BASE_RK3 ? 3 : 2);  // base stages
      cs_per_step = (long long)c.nx * (s * c.nz_S + s * c.m * (c.nz_B + c.nz_F));
      r->cell_stages = cs_per_step * r->steps_done;
      destroy_instance(r->inst);  // stream-ordered frees on the copy stream
      r->inst = nullptr;
      finish(S, r, error);
    }
    S->retiring.swap(still);
  }
  // shutdown: drop everything the thread still owns
  cudaStreamSynchronize(S->compute);
  for (int slot = 0; slot < 2; slot++)
    if (step_ev_used[slot]) account(slot);
  cudaStreamSynchronize(S->copy);
  for (Request* r : S->resident)
    if (r->inst) destroy_instance(r->inst), r->inst = nullptr;
  for (Request* r : S->retiring) {
    if (r->copied) cudaEventDestroy(r->copied);
    if (r->pinned) cudaFreeHost(r->pinned);
    if (r->inst) destroy_instance(r->inst), r->inst = nullptr;
  }
  S->pool.clear();
  cudaStreamSynchronize(S->copy);
  for (int p = 0; p < 2; p++) runner_destroy(S->runner[p]);
  cudaStreamSynchronize(S->compute);
  for (cudaEvent_t e : {step_ev[0], step_ev[1], beg_ev[0], beg_ev[1]}) cudaEventDestroy(e);
  for (int k = 0; k < mprk_server::NSIDE; k++) {
    if (S->side[k]) cudaStreamDestroy(S->side[k]);
    if (S->ev_join[k]) cudaEventDestroy(S->ev_join[k]);
  }
  if (S->ev_fork) cudaEventDestroy(S->ev_fork);
  cudaStreamDestroy(S->compute);
  cudaStreamDestroy(S->copy);
}

}  // namespace

extern "C" {

int mprk_server_create(const mprk_server_config* cfg, mprk_server** out) {
  if (!cfg || !out) return sfail(MPRK_EINVAL, "NULL argument");
  *out = nullptr;
  if (cfg->hbm_budget_bytes <= 0 || cfg->max_slots <= 0 || cfg->max_queue <= 0 || cfg->solo_cells < -1)
    return sfail(MPRK_EINVAL, "budget, slots and queue length must be positive, solo_cells >= -1");
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || cfg->device < 0 || cfg->device >= ndev)
    return sfail(MPRK_ECUDA, "no such CUDA device");
  mprk_server* S = new mprk_server();
  S->cfg = *cfg;
  S->solo_cells = cfg->solo_cells == 0 ? MPRK_SOLO_CELLS_DEFAULT : (cfg->solo_cells < 0 ? 0 : cfg->solo_cells);
  S->solo_fp64_only = cfg->solo_cells == 0;
  S->t0 = Clock::now();
  S->th = std::thread(server_loop, S);
  *out = S;
  return MPRK_OK;
}

int mprk_submit(mprk_server* S, const mprk_config* cfg, const double* q0_host, int n_slow_steps,
                uint64_t* ticket) {
  if (!S || !cfg || !q0_host || !ticket) return sfail(MPRK_EINVAL, "NULL argument");
  if (n_slow_steps < 1) return sfail(MPRK_EINVAL, "need at least one slow step");
  int rc = validate_config(cfg);
  if (rc) return rc;
  if (cfg->ny > 1) return sfail(MPRK_EINVAL, "the server takes 2-D requests only");
  const long long bytes = instance_bytes(*cfg);
  if (bytes > S->cfg.hbm_budget_bytes)
    return sfail(MPRK_EBUDGET, "request needs " + std::to_string(bytes) + " device bytes, budget is " +
                                   std::to_string(S->cfg.hbm_budget_bytes));
  Request* r = new Request();
  r->cfg = *cfg;
  r->cfg.diag_every = 0;
  r->n_steps = n_slow_steps;
  r->bytes = bytes;
  const size_t n = (size_t)4 * (cfg->nz_S + cfg->nz_B + cfg->nz_F) * cfg->nx;
  r->q0.assign(q0_host, q0_host + n);
  {
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->thread_error) {
      delete r;
      return sfail(S->thread_error, S->thread_msg);
    }
    if ((int)S->queue.size() >= S->cfg.max_queue) {
      delete r;
      return sfail(MPRK_EBUSY, "server queue is full");
    }
    r->ticket = S->next_ticket++;
    r->t_submit = S->now();
    S->queue.push_back(r);
    S->all[r->ticket] = r;
    *ticket = r->ticket;
  }
  S->cv.notify_one();
  return MPRK_OK;
}

int mprk_poll(mprk_server* S, uint64_t ticket, int* status, double* q_out_host, mprk_stats* stats) {
  if (!S || !status) return sfail(MPRK_EINVAL, "NULL argument");
  std::lock_guard<std::mutex> lk(S->mu);
  auto itr = S->all.find(ticket);
  if (itr == S->all.end()) return sfail(MPRK_ENOTFOUND, "unknown ticket");
  Request* r = itr->second;
  *status = r->state;
  if (stats) {
    stats->t_submit = r->t_submit;
    stats->t_admit = r->t_admit;
    stats->t_finish = r->t_finish;
    stats->cell_stages = r->cell_stages;
    stats->device_bytes = r->bytes;
    stats->steps_done = r->steps_done;
    stats->error = r->error;
  }
  const int err = r->error;
  if (r->state == MPRK_REQ_DONE && q_out_host) {
    if (!r->result.empty()) memcpy(q_out_host, r->result.data(), r->result.size() * sizeof(double));
    S->all.erase(itr);
    delete r;
  }
  return err;
}

int mprk_server_stats(mprk_server* S, double out[8]) {
  if (!S || !out) return sfail(MPRK_EINVAL, "NULL argument");
  std::lock_guard<std::mutex> lk(S->mu);
  out[0] = (double)S->n_done;
  out[1] = (double)S->cells_done;
  out[2] = (double)S->batched_steps;
  out[3] = (double)S->n_resident;
  out[4] = (double)S->queue.size();
  out[5] = (double)S->ledger;
  out[6] = S->now();
  out[7] = (double)S->n_failed;
  return MPRK_OK;
}

int mprk_server_profile(mprk_server* S, double out[8]) {
  if (!S || !out) return sfail(MPRK_EINVAL, "NULL argument");
  std::lock_guard<std::mutex> lk(S->mu);
  for (int j = 0; j < 8; j++) out[j] = S->prof[j];
  out[6] = S->first_step >= 0 ? S->prof[6] - S->first_step : 0.0;
  return MPRK_OK;
}

int mprk_server_destroy(mprk_server* S) {
  if (!S) return sfail(MPRK_EINVAL, "NULL server");
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
  }
  S->cv.notify_one();
  if (S->th.joinable()) S->th.join();
  for (auto& kv : S->all) delete kv.second;
  delete S;
  return MPRK_OK;
}

}  // extern "C"
