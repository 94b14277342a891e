// Request server: continuous admission of subjects into a fixed number of slots under a
// device-memory budget. Each slot owns a host worker thread and a CUDA stream; a request
// runs create -> statistics -> Gibbs sweeps -> copy of W -> destroy on its slot's stream, so
// requests that are admitted while others run overlap on the device. Admission is FIFO: the
// oldest pending request starts as soon as a slot is free and its device-memory estimate
// fits in what the running requests leave of the budget. Each slot's solver grids are
// limited to sm_budget SMs, so the cooperative solves of all slots fit on the GPU together.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/bfmri.h"

namespace bfmri {
void set_global_error(const std::string& msg);                                        // bfmri_api.cu
size_t handle_device_bytes(int N, int T, int K, int P, size_t y_esz, bool mixed);      // bfmri_api.cu
size_t mg_request_bytes(const bfmri_lattice& lat, const uint8_t* mask, int D);         // bfmri_api.cu
}

namespace {

using Clock = std::chrono::steady_clock;

struct Job {
  long long ticket = 0;
  bfmri_request req{};
  size_t bytes = 0;
  int N = 0;
  bfmri_result res{};
  bool done = false;
};

// Stream-ordered allocation from the server's pool: neither allocation nor release
// synchronises the device, so one slot's set-up does not stall the other slots' kernels.
struct SlotAlloc {
  cudaStream_t stream = nullptr;
  cudaMemPool_t pool = nullptr;
};

void* pool_alloc(size_t bytes, void* ctx) {
  SlotAlloc* c = static_cast<SlotAlloc*>(ctx);
  void* p = nullptr;
  if (cudaMallocFromPoolAsync(&p, bytes, c->pool, c->stream) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return p;
}

void pool_free(void* p, void* ctx) {
  SlotAlloc* c = static_cast<SlotAlloc*>(ctx);
  cudaFreeAsync(p, c->stream);
}

}  // namespace

struct bfmri_server {
  size_t budget = 0;
  int slots = 1;
  int sm_budget = 0;
  int device = 0;
  Clock::time_point t0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Job*> pending;
  std::map<long long, Job*> jobs;
  std::vector<Job*> slot_job;
  std::vector<std::thread> workers;
  std::vector<cudaStream_t> streams;
  std::vector<SlotAlloc> alloc;
  cudaMemPool_t pool = nullptr;
  size_t in_use = 0, peak_in_use = 0;
  long long next_ticket = 1;
  bool stop = false;
  int running = 0, peak_running = 0;

  double now() const { return std::chrono::duration<double>(Clock::now() - t0).count(); }

  // admit from the head of the queue while a slot is free and the budget allows
  void admit_locked() {
    while (!pending.empty()) {
      Job* j = pending.front();
      if (in_use + j->bytes > budget) break;
      int free_slot = -1;
      for (int s = 0; s < slots; ++s)
        if (!slot_job[s]) { free_slot = s; break; }
      if (free_slot < 0) break;
      pending.pop_front();
      slot_job[free_slot] = j;
      in_use += j->bytes;
      peak_in_use = std::max(peak_in_use, in_use);
      running += 1;
      peak_running = std::max(peak_running, running);
      cv_work.notify_all();
    }
  }

  void run(int slot) {
    cudaSetDevice(device);
    for (;;) {
      Job* j = nullptr;
      {
        std::unique_lock<std::mutex> lk(mu);
        cv_work.wait(lk, [&] { return stop || slot_job[slot] != nullptr; });
        if (!slot_job[slot]) return;
        j = slot_job[slot];
      }
      j->res.start_s = now();
      bfmri_options o = j->req.opt;
      o.cuda_stream = streams[slot];
      o.sm_budget = sm_budget;
      o.dev_alloc = pool_alloc;
      o.dev_free = pool_free;
      o.alloc_ctx = &alloc[slot];
      bfmri_handle* h = nullptr;
      bfmri_status st = bfmri_create(&j->req.lat, j->req.mask, j->req.X, j->req.Y, j->req.y_dtype,
                                     j->req.T, j->req.K, j->req.P, &o, &h);
      bfmri_sweep_info info{};
      if (st == BFMRI_OK) st = bfmri_precompute_stats(h);
      if (st == BFMRI_OK) st = bfmri_gibbs_sweep(h, j->req.n_sweeps, j->req.first_counter, &info);
      if (st == BFMRI_OK && j->req.W_out) st = bfmri_get_state(h, j->req.W_out, nullptr, nullptr, nullptr, nullptr);
      if (st == BFMRI_OK && j->req.alpha_out)
        st = bfmri_get_state(h, nullptr, nullptr, nullptr, j->req.alpha_out, nullptr);
      if (h) bfmri_destroy(h);
      {
        std::lock_guard<std::mutex> lk(mu);
        j->res.status = st;
        j->res.end_s = now();
        j->res.pcg_iterations = info.pcg_iterations_W + info.pcg_iterations_A;
        j->done = true;
        slot_job[slot] = nullptr;
        in_use -= j->bytes;
        running -= 1;
        admit_locked();
      }
      cv_done.notify_all();
    }
  }
};

extern "C" {

size_t bfmri_request_device_bytes(int N, int T, int K, int P, int y_dtype, int precision) {
  if (N < 1 || T < 1 || K < 1 || P < 0) return 0;
  // every allocation of the request's handle, Y included (released after the statistics),
  // plus a margin for the pool's own rounding
  const size_t b = bfmri::handle_device_bytes(N, T, K, P, y_dtype == BFMRI_F64 ? 8 : 4,
                                               precision == BFMRI_PREC_MIXED);
  return b + b / 32 + ((size_t)2 << 20);
}

bfmri_status bfmri_server_pool_usage(bfmri_server* s, size_t* used_high, int reset) {
  if (!s || !s->pool) return BFMRI_ERR_INVALID_ARG;
  uint64_t v = 0;
  if (cudaMemPoolGetAttribute(s->pool, cudaMemPoolAttrUsedMemHigh, &v) != cudaSuccess) return BFMRI_ERR_CUDA;
  if (used_high) *used_high = (size_t)v;
  if (reset) {
    uint64_t zero = 0;
    if (cudaMemPoolSetAttribute(s->pool, cudaMemPoolAttrUsedMemHigh, &zero) != cudaSuccess) return BFMRI_ERR_CUDA;
  }
  return BFMRI_OK;
}

bfmri_status bfmri_server_create(size_t budget_bytes, int max_slots, int sm_budget, bfmri_server** out) {
  if (!out || max_slots < 1 || max_slots > 64 || budget_bytes == 0 || sm_budget < 0) {
    bfmri::set_global_error("bfmri_server_create: bad arguments");
    return BFMRI_ERR_INVALID_ARG;
  }
  bfmri_server* s = new bfmri_server();
  s->budget = budget_bytes;
  s->slots = max_slots;
  s->sm_budget = sm_budget;
  s->t0 = Clock::now();
  if (cudaGetDevice(&s->device) != cudaSuccess) {
    delete s;
    bfmri::set_global_error("bfmri_server_create: no CUDA device");
    return BFMRI_ERR_CUDA;
  }
  s->slot_job.assign(max_slots, nullptr);
  s->streams.resize(max_slots);
  for (int i = 0; i < max_slots; ++i) {
    if (cudaStreamCreateWithFlags(&s->streams[i], cudaStreamNonBlocking) != cudaSuccess) {
      for (int k = 0; k < i; ++k) cudaStreamDestroy(s->streams[k]);
      delete s;
      bfmri::set_global_error("bfmri_server_create: stream creation failed");
      return BFMRI_ERR_CUDA;
    }
  }
  cudaMemPoolProps props;
  memset(&props, 0, sizeof(props));
  props.allocType = cudaMemAllocationTypePinned;
  props.location.type = cudaMemLocationTypeDevice;
  props.location.id = s->device;
  if (cudaMemPoolCreate(&s->pool, &props) != cudaSuccess) {
    for (int k = 0; k < max_slots; ++k) cudaStreamDestroy(s->streams[k]);
    delete s;
    bfmri::set_global_error("bfmri_server_create: memory pool creation failed");
    return BFMRI_ERR_CUDA;
  }
  uint64_t keep = budget_bytes;   // keep released memory cached up to the budget
  cudaMemPoolSetAttribute(s->pool, cudaMemPoolAttrReleaseThreshold, &keep);
  s->alloc.resize(max_slots);
  for (int i = 0; i < max_slots; ++i) {
    s->alloc[i].stream = s->streams[i];
    s->alloc[i].pool = s->pool;
  }
  for (int i = 0; i < max_slots; ++i) s->workers.emplace_back([s, i] { s->run(i); });
  *out = s;
  return BFMRI_OK;
}

bfmri_status bfmri_server_submit(bfmri_server* s, const bfmri_request* req, long long* ticket) {
  if (!s || !req || !ticket || !req->mask) return BFMRI_ERR_INVALID_ARG;
  const long long nsite = (long long)req->lat.nx * req->lat.ny * req->lat.nz;
  if (nsite < 1) return BFMRI_ERR_INVALID_ARG;
  int N = 0;
  for (long long l = 0; l < nsite; ++l) N += req->mask[l] ? 1 : 0;
  Job* j = new Job();
  j->req = *req;
  j->N = N;
  j->bytes = bfmri_request_device_bytes(N, req->T, req->K, req->P, req->y_dtype, req->opt.precision);
  if (req->opt.w_prior == BFMRI_PRIOR_LTL && N > 0) {
    // the L'L prior's plane for L v ([K][ld] doubles), with the same margin
    const size_t lt = (((size_t)req->K * (((size_t)N + 31) & ~size_t(31)) * 8 + 255) & ~size_t(255));
    j->bytes += lt + lt / 32;
  }
  if (req->opt.w_prior == BFMRI_PRIOR_ANISO && N > 0) {
    // the exchange step's auxiliary field ([K][ld] doubles), its small per-k arrays and the
    // direction edge sums' partials (three per component), with the same margin
    const size_t ldr = ((size_t)N + 31) & ~size_t(31);
    auto r256 = [](size_t b) { return (b + 255) & ~size_t(255); };
    const size_t hp = (size_t)1024 * std::max(req->K, req->P) * 8;   // at most 1024 partial rows
    const size_t an = r256((size_t)req->K * ldr * 8) + 6 * r256(6 * (size_t)req->K * 8) + r256(3 * hp);
    j->bytes += an + an / 32;
  }
  if (req->opt.precond == BFMRI_PRECOND_MULTIGRID && N > 0) {
    // the hierarchy a multigrid request builds on its first solve, with the same margin
    const size_t mg = bfmri::mg_request_bytes(req->lat, req->mask, std::max(req->K, req->P));
    j->bytes += mg + mg / 32;
  }
  std::lock_guard<std::mutex> lk(s->mu);
  if (j->bytes > s->budget) {
    delete j;
    bfmri::set_global_error("bfmri_server_submit: request exceeds the whole device-memory budget");
    return BFMRI_ERR_OOM;
  }
  j->ticket = s->next_ticket++;
  j->res.submit_s = s->now();
  j->res.N = N;
  j->res.device_bytes = j->bytes;
  j->res.status = BFMRI_PENDING;
  s->jobs[j->ticket] = j;
  s->pending.push_back(j);
  s->admit_locked();
  *ticket = j->ticket;
  return BFMRI_OK;
}

bfmri_status bfmri_server_poll(bfmri_server* s, long long ticket, int wait, bfmri_result* res) {
  if (!s) return BFMRI_ERR_INVALID_ARG;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->jobs.find(ticket);
  if (it == s->jobs.end()) return BFMRI_ERR_INVALID_ARG;
  Job* j = it->second;
  if (wait) s->cv_done.wait(lk, [&] { return j->done; });
  if (!j->done) {
    if (res) *res = j->res;
    return BFMRI_PENDING;
  }
  if (res) *res = j->res;
  s->jobs.erase(it);
  delete j;
  return BFMRI_OK;
}

bfmri_status bfmri_server_stats(bfmri_server* s, size_t* peak_bytes, int* peak_running, size_t* in_use) {
  if (!s) return BFMRI_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  if (peak_bytes) *peak_bytes = s->peak_in_use;
  if (peak_running) *peak_running = s->peak_running;
  if (in_use) *in_use = s->in_use;
  return BFMRI_OK;
}

bfmri_status bfmri_server_destroy(bfmri_server* s) {
  if (!s) return BFMRI_OK;
  {
    std::unique_lock<std::mutex> lk(s->mu);
    s->cv_done.wait(lk, [&] { return s->pending.empty() && s->running == 0; });
    s->stop = true;
  }
  s->cv_work.notify_all();
  for (auto& t : s->workers) t.join();
  for (cudaStream_t st : s->streams) {
    cudaStreamSynchronize(st);
    cudaStreamDestroy(st);
  }
  if (s->pool) cudaMemPoolDestroy(s->pool);
  for (auto& kv : s->jobs) delete kv.second;
  delete s;
  return BFMRI_OK;
}

}  // extern "C"
