// Serving: many characterization jobs streaming trace chunks at once.
//
// A server owns a pool of slots; each slot is a handle with its own CUDA
// stream, so the ingest of one job's chunks and the reduction of another run
// side by side on the device. A job is admitted when a slot is free and its
// memory reservation fits the server's HBM budget (memory held by idle slots
// is released first when needed); otherwise aiwc_job_open answers
// AIWC_EAGAIN and the caller retries later. aiwc_job_finish hands the job to
// a worker thread that runs the end-of-kernel reduction; aiwc_job_poll /
// aiwc_job_wait return the metrics and release the slot. Results are those
// of aiwc_compute on the same events: jobs share no device state.
#include <atomic>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_set>
#include <vector>

#include "aiwc_internal.cuh"

struct aiwc_job;

struct aiwc_server {
  aiwc_server_config cfg;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  struct Slot {
    aiwc_handle* h = nullptr;
    cudaStream_t stream = nullptr;
    bool busy = false;
    uint64_t reserved = 0;
  };
  std::vector<Slot> slots;
  uint64_t reserved_total = 0;
  std::deque<aiwc_job*> queue;
  std::unordered_set<aiwc_job*> jobs;  // opened and not yet collected
  std::vector<std::thread> workers;
  bool stopping = false;
  uint64_t admitted = 0, rejected = 0, completed = 0;
};

struct aiwc_job {
  aiwc_server* srv = nullptr;
  size_t slot = 0;
  aiwc_handle* h = nullptr;
  // the caller's thread reads the state without the server lock (push guards,
  // aiwc_job_wait) while a worker sets kDone under it
  enum State { kOpen, kQueued, kDone };
  std::atomic<State> state{kOpen};
  aiwc_status status = AIWC_OK;
  aiwc_metrics result;
  std::vector<uint64_t> hist;
  std::string err;
};

namespace {

aiwc_status srv_fail(aiwc_status s, const std::string& msg) {
  aiwc::set_last_error(msg);
  return s;
}

uint64_t held_bytes(aiwc_server* s) {
  uint64_t b = 0;
  for (auto& sl : s->slots)
    if (sl.h) b += aiwc_device_bytes(sl.h);
  return b;
}

void worker_loop(aiwc_server* s) {
  for (;;) {
    aiwc_job* j = nullptr;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      s->cv_work.wait(lk, [&] { return s->stopping || !s->queue.empty(); });
      if (s->queue.empty()) return;
      j = s->queue.front();
      s->queue.pop_front();
    }
    aiwc_metrics m;
    memset(&m, 0, sizeof(m));
    m.opcode_hist = j->hist.data();
    const aiwc_status st = aiwc_compute(j->h, &m);
    {
      std::lock_guard<std::mutex> lk(s->mu);
      j->result = m;
      j->status = st;
      if (st != AIWC_OK) j->err = aiwc_last_error(j->h);
      j->state = aiwc_job::kDone;
      ++s->completed;
    }
    s->cv_done.notify_all();
  }
}

}  // namespace

extern "C" {

void aiwc_server_config_default(aiwc_server_config* c) {
  if (!c) return;
  memset(c, 0, sizeof(*c));
  c->device = 0;
  c->hbm_budget = 120ull << 30;
  c->max_jobs = 32;
  c->workers = 4;
}

aiwc_status aiwc_server_create(const aiwc_server_config* cfg, aiwc_server** out) {
  if (!cfg || !out) return srv_fail(AIWC_EINVAL, "null server config or output");
  if (cfg->max_jobs == 0 || cfg->max_jobs > 4096 || cfg->workers == 0 || cfg->workers > 64 || cfg->hbm_budget == 0)
    return srv_fail(AIWC_EINVAL, "server config out of range");
  aiwc_server* s = new aiwc_server();
  s->cfg = *cfg;
  s->slots.resize(cfg->max_jobs);
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(cfg->device);
  for (auto& sl : s->slots) {
    if (cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      cudaSetDevice(prev);
      aiwc_server_destroy(s);
      return srv_fail(AIWC_ECUDA, "could not create slot streams");
    }
  }
  cudaSetDevice(prev);
  for (uint32_t i = 0; i < cfg->workers; ++i) s->workers.emplace_back(worker_loop, s);
  *out = s;
  return AIWC_OK;
}

aiwc_status aiwc_job_open(aiwc_server* s, const aiwc_config* job_cfg, uint64_t reserve_bytes, aiwc_job** out) {
  if (!s || !job_cfg || !out) return srv_fail(AIWC_EINVAL, "null server, config or output");
  *out = nullptr;
  std::lock_guard<std::mutex> lk(s->mu);
  if (job_cfg->partitions > 1) return srv_fail(AIWC_EINVAL, "server jobs are not partitioned");
  if (reserve_bytes > s->cfg.hbm_budget) {
    ++s->rejected;
    return srv_fail(AIWC_ENOMEM, "job reservation exceeds the server's HBM budget");
  }
  aiwc_config c = *job_cfg;
  c.device = s->cfg.device;
  c.hbm_budget = reserve_bytes;
  // a free slot, preferring one whose handle already has this metric configuration
  size_t k = s->slots.size();
  for (size_t i = 0; i < s->slots.size(); ++i) {
    if (s->slots[i].busy) continue;
    if (k == s->slots.size()) k = i;
    if (s->slots[i].h && aiwc::handle_config_matches(s->slots[i].h, &c)) {
      k = i;
      break;
    }
  }
  if (k == s->slots.size()) {
    ++s->rejected;
    return AIWC_EAGAIN;
  }
  auto& sl = s->slots[k];
  c.cuda_stream = sl.stream;
  // device memory in use: busy slots count their reservation (or what they
  // hold, if more); idle slots what they hold; idle memory is released first
  auto in_use = [&]() {
    uint64_t b = 0;
    for (size_t i = 0; i < s->slots.size(); ++i) {
      const auto& x = s->slots[i];
      const uint64_t held = x.h ? aiwc_device_bytes(x.h) : 0;
      if (i == k) continue;
      b += x.busy ? (held > x.reserved ? held : x.reserved) : held;
    }
    return b;
  };
  if (in_use() + reserve_bytes > s->cfg.hbm_budget) {
    for (size_t i = 0; i < s->slots.size() && in_use() + reserve_bytes > s->cfg.hbm_budget; ++i) {
      if (i != k && !s->slots[i].busy && s->slots[i].h) {
        aiwc_destroy(s->slots[i].h);
        s->slots[i].h = nullptr;
      }
    }
    if (in_use() + reserve_bytes > s->cfg.hbm_budget) {
      ++s->rejected;
      return AIWC_EAGAIN;
    }
  }
  if (sl.h && (!aiwc::handle_config_matches(sl.h, &c) || aiwc_device_bytes(sl.h) > reserve_bytes)) {
    aiwc_destroy(sl.h);
    sl.h = nullptr;
  }
  if (sl.h) {
    aiwc::handle_set_budget(sl.h, reserve_bytes);
  } else {
    aiwc_status st = aiwc_create(&c, &sl.h);
    if (st != AIWC_OK) {
      sl.h = nullptr;
      return st;
    }
  }
  sl.busy = true;
  sl.reserved = reserve_bytes;
  s->reserved_total += reserve_bytes;
  ++s->admitted;
  aiwc_job* j = new aiwc_job();
  j->srv = s;
  j->slot = k;
  j->h = sl.h;
  j->hist.assign(c.n_opcodes, 0);
  s->jobs.insert(j);
  *out = j;
  return AIWC_OK;
}

aiwc_status aiwc_job_push_mem(aiwc_job* j, const aiwc_mem_event* ev, size_t n, int on_device) {
  if (!j || j->state != aiwc_job::kOpen) return srv_fail(AIWC_EINVAL, "job is not open");
  return aiwc_push_mem(j->h, ev, n, on_device);
}

aiwc_status aiwc_job_push_branch(aiwc_job* j, const aiwc_branch_event* ev, size_t n, int on_device) {
  if (!j || j->state != aiwc_job::kOpen) return srv_fail(AIWC_EINVAL, "job is not open");
  return aiwc_push_branch(j->h, ev, n, on_device);
}

aiwc_status aiwc_job_push_widths(aiwc_job* j, const uint16_t* widths, size_t n, int on_device) {
  if (!j || j->state != aiwc_job::kOpen) return srv_fail(AIWC_EINVAL, "job is not open");
  return aiwc_push_widths(j->h, widths, n, on_device);
}

aiwc_status aiwc_job_push_instr_runs(aiwc_job* j, const uint32_t* run_wi, const uint64_t* run_off,
                                     const uint64_t* run_len, size_t n_runs, const uint16_t* ops, size_t n_ops,
                                     int on_device) {
  if (!j || j->state != aiwc_job::kOpen) return srv_fail(AIWC_EINVAL, "job is not open");
  return aiwc_push_instr_runs(j->h, run_wi, run_off, run_len, n_runs, ops, n_ops, on_device);
}

aiwc_status aiwc_job_finish(aiwc_job* j) {
  if (!j || j->state != aiwc_job::kOpen) return srv_fail(AIWC_EINVAL, "job is not open");
  aiwc_server* s = j->srv;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    j->state = aiwc_job::kQueued;
    s->queue.push_back(j);
  }
  s->cv_work.notify_one();
  return AIWC_OK;
}

static aiwc_status collect(aiwc_job* j, aiwc_metrics* out) {
  // caller holds s->mu and the job is done
  aiwc_server* s = j->srv;
  uint64_t* user_hist = out->opcode_hist;
  *out = j->result;
  out->opcode_hist = user_hist;
  if (user_hist) memcpy(user_hist, j->hist.data(), j->hist.size() * 8);
  const aiwc_status st = j->status;
  if (st != AIWC_OK) aiwc::set_last_error(j->err);
  auto& sl = s->slots[j->slot];
  sl.busy = false;
  s->reserved_total -= sl.reserved;
  sl.reserved = 0;
  s->jobs.erase(j);
  delete j;
  return st;
}

aiwc_status aiwc_job_poll(aiwc_job* j, aiwc_metrics* out) {
  if (!j || !out) return srv_fail(AIWC_EINVAL, "null job or output");
  std::lock_guard<std::mutex> lk(j->srv->mu);
  if (j->state != aiwc_job::kDone) return AIWC_EAGAIN;
  return collect(j, out);
}

aiwc_status aiwc_job_wait(aiwc_job* j, aiwc_metrics* out) {
  if (!j || !out) return srv_fail(AIWC_EINVAL, "null job or output");
  aiwc_server* s = j->srv;
  if (j->state == aiwc_job::kOpen) {
    aiwc_status st = aiwc_job_finish(j);
    if (st != AIWC_OK) return st;
  }
  std::unique_lock<std::mutex> lk(s->mu);
  s->cv_done.wait(lk, [&] { return j->state == aiwc_job::kDone; });
  return collect(j, out);
}

aiwc_status aiwc_server_stats(const aiwc_server* s, uint64_t* admitted, uint64_t* rejected, uint64_t* completed,
                              uint64_t* device_bytes) {
  if (!s) return srv_fail(AIWC_EINVAL, "null server");
  aiwc_server* m = const_cast<aiwc_server*>(s);
  std::lock_guard<std::mutex> lk(m->mu);
  if (admitted) *admitted = m->admitted;
  if (rejected) *rejected = m->rejected;
  if (completed) *completed = m->completed;
  if (device_bytes) *device_bytes = held_bytes(m);
  return AIWC_OK;
}

aiwc_status aiwc_server_destroy(aiwc_server* s) {
  if (!s) return AIWC_OK;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stopping = true;
  }
  s->cv_work.notify_all();
  for (auto& t : s->workers) t.join();
  for (aiwc_job* j : s->jobs) delete j;
  for (auto& sl : s->slots) {
    if (sl.h) aiwc_destroy(sl.h);
    if (sl.stream) cudaStreamDestroy(sl.stream);
  }
  delete s;
  return AIWC_OK;
}

}  // extern "C"
