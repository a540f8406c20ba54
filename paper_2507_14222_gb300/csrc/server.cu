// Continuous-batching scoring server over a device-resident model (Eq. 4,
// Regulations 1-3 per flow, through ig_score).
//
// Requests (host arrays of packed flows) join a queue.  A scheduler thread
// forms a batch from the requests waiting at the front of the queue -- as
// many as fit the per-batch flow cap and the device-memory budget, without
// waiting for more to arrive -- and hands it to a free slot.  Each slot owns a
// stream, pinned staging buffers sized for the cap, and a thread that copies
// the batch in, scores it, copies the results out and completes the
// requests.  With several slots, batches admitted while others run overlap
// on the device.  A request's latency runs from its submission to the moment
// its results are in its own host arrays.
//
// Scoring is a pure function of each flow and the model, so a flow's A, N
// and label do not depend on which other flows share its batch.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/ig.h"
#include "internal.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
  uint64_t ticket = 0;
  const uint64_t* rows = nullptr;
  int64_t m = 0;
  int64_t* A = nullptr;
  int64_t* N = nullptr;
  uint8_t* labels = nullptr;
  Clock::time_point submitted, completed;
  bool done = false;
  int rc = IG_OK;
  std::string error;
};

struct Slot {
  cudaStream_t stream = nullptr;
  uint64_t* d_rows = nullptr;
  int64_t* d_A = nullptr;
  int64_t* d_N = nullptr;
  uint8_t* d_lab = nullptr;
  uint64_t* h_rows = nullptr;  // pinned
  int64_t* h_A = nullptr;      // pinned
  int64_t* h_N = nullptr;      // pinned
  uint8_t* h_lab = nullptr;    // pinned
  std::vector<Request*> batch;
  int64_t batch_bytes = 0;
  bool busy = false;
  bool has_work = false;
  std::thread thread;
};

int set_error(const char* msg) { return igk::report_error(IG_E_INVAL, msg); }

}  // namespace

struct ig_server {
  const ig_model* model = nullptr;
  int K = 0;
  int device = 0;
  ig_server_config cfg{};
  int64_t bytes_per_flow = 0;
  std::mutex mu;
  std::condition_variable cv;       // scheduler: queue or slot changes
  std::condition_variable done_cv;  // waiters: a request completed
  std::deque<Request*> queue;
  std::unordered_map<uint64_t, Request*> live;
  std::vector<Slot> slots;
  std::thread scheduler;
  bool stop = false;
  int64_t inflight_bytes = 0;
  uint64_t next_ticket = 1;
  int64_t batches = 0, flows = 0;
};

namespace {

void slot_loop(ig_server* sv, Slot* sl) {
  cudaSetDevice(sv->device);
  for (;;) {
    {
      std::unique_lock<std::mutex> lk(sv->mu);
      sv->cv.wait(lk, [&] { return sl->has_work || sv->stop; });
      if (!sl->has_work && sv->stop) return;
    }
    // Gather the batch's flows into the pinned buffer, score, scatter back.
    int64_t total = 0;
    for (Request* r : sl->batch) {
      std::memcpy(sl->h_rows + total * sv->K, r->rows, sizeof(uint64_t) * r->m * sv->K);
      total += r->m;
    }
    int rc = IG_OK;
    std::string err;
    cudaError_t e = cudaMemcpyAsync(sl->d_rows, sl->h_rows, sizeof(uint64_t) * total * sv->K,
                                    cudaMemcpyHostToDevice, sl->stream);
    if (e != cudaSuccess) {
      rc = IG_E_CUDA;
      err = cudaGetErrorString(e);
    }
    if (rc == IG_OK) {
      rc = ig_score(sv->model, sl->d_rows, total, sl->d_A, sl->d_N, sl->d_lab,
                    reinterpret_cast<ig_stream_t>(sl->stream));
      if (rc != IG_OK) err = ig_last_error();
    }
    if (rc == IG_OK) {
      cudaMemcpyAsync(sl->h_A, sl->d_A, sizeof(int64_t) * total, cudaMemcpyDeviceToHost, sl->stream);
      cudaMemcpyAsync(sl->h_N, sl->d_N, sizeof(int64_t) * total, cudaMemcpyDeviceToHost, sl->stream);
      cudaMemcpyAsync(sl->h_lab, sl->d_lab, total, cudaMemcpyDeviceToHost, sl->stream);
      e = cudaStreamSynchronize(sl->stream);
      if (e != cudaSuccess) {
        rc = IG_E_CUDA;
        err = cudaGetErrorString(e);
      }
    }
    int64_t off = 0;
    for (Request* r : sl->batch) {
      if (rc == IG_OK) {
        if (r->A) std::memcpy(r->A, sl->h_A + off, sizeof(int64_t) * r->m);
        if (r->N) std::memcpy(r->N, sl->h_N + off, sizeof(int64_t) * r->m);
        if (r->labels) std::memcpy(r->labels, sl->h_lab + off, r->m);
      }
      off += r->m;
    }
    const Clock::time_point now = Clock::now();
    {
      std::lock_guard<std::mutex> lk(sv->mu);
      for (Request* r : sl->batch) {
        r->rc = rc;
        r->error = err;
        r->completed = now;
        r->done = true;
      }
      sv->inflight_bytes -= sl->batch_bytes;
      sv->batches += 1;
      sv->flows += total;
      sl->batch.clear();
      sl->batch_bytes = 0;
      sl->has_work = false;
      sl->busy = false;
    }
    sv->done_cv.notify_all();
    sv->cv.notify_all();
  }
}

void scheduler_loop(ig_server* sv) {
  std::unique_lock<std::mutex> lk(sv->mu);
  for (;;) {
    sv->cv.wait(lk, [&] {
      if (sv->stop) return true;
      if (sv->queue.empty()) return false;
      for (const Slot& s : sv->slots)
        if (!s.busy) return true;
      return false;
    });
    if (sv->stop) return;
    Slot* free_slot = nullptr;
    for (Slot& s : sv->slots)
      if (!s.busy) {
        free_slot = &s;
        break;
      }
    // Continuous batching: take what has arrived, in order, while the batch
    // stays within the flow cap and the in-flight memory within the budget.
    int64_t flows = 0, bytes = 0;
    while (!sv->queue.empty()) {
      Request* r = sv->queue.front();
      const int64_t b = r->m * sv->bytes_per_flow;
      if (flows + r->m > sv->cfg.max_batch_flows) break;
      if (flows > 0 && sv->inflight_bytes + bytes + b > sv->cfg.memory_budget_bytes) break;
      if (flows == 0 && sv->inflight_bytes > 0 &&
          sv->inflight_bytes + b > sv->cfg.memory_budget_bytes)
        break;  // wait for memory to free up
      sv->queue.pop_front();
      free_slot->batch.push_back(r);
      flows += r->m;
      bytes += b;
    }
    if (free_slot->batch.empty()) {
      // Nothing admitted (memory): wait for a batch to finish.
      sv->cv.wait(lk, [&] {
        return sv->stop || sv->inflight_bytes == 0 ||
               (!sv->queue.empty() &&
                sv->inflight_bytes + sv->queue.front()->m * sv->bytes_per_flow <=
                    sv->cfg.memory_budget_bytes);
      });
      continue;
    }
    free_slot->busy = true;
    free_slot->has_work = true;
    free_slot->batch_bytes = bytes;
    sv->inflight_bytes += bytes;
    sv->cv.notify_all();
  }
}

}  // namespace

extern "C" {

int ig_server_create(const ig_model* model, const ig_server_config* cfg, ig_server** out) {
  return igk::guarded("ig_server_create", [&]() -> int {
    if (!model || !out) return set_error("ig_server_create: NULL argument");
    *out = nullptr;
    ig_model_info_t info;
    if (ig_model_info(model, &info) != IG_OK) return IG_E_INVAL;
    ig_server* sv = new ig_server;
    sv->model = model;
    sv->K = info.K;
    cudaGetDevice(&sv->device);
    ig_server_config c{};
    if (cfg) c = *cfg;
    if (c.slots <= 0) c.slots = 3;
    if (c.max_batch_flows <= 0) c.max_batch_flows = 65536;
    // Device bytes per flow in flight: the packed row, A, N and label, plus
    // the item index of a scoring call (at most a quarter of all item slots
    // filled, each copy a padded row).
    const int KT = igk::padded_words(sv->K);
    sv->bytes_per_flow = int64_t(KT) * 8 * (1 + 64 * sv->K / 4) + 32;
    if (c.memory_budget_bytes <= 0) {
      size_t free_b = 0, total_b = 0;
      cudaMemGetInfo(&free_b, &total_b);
      c.memory_budget_bytes = int64_t(free_b / 4);
    }
    c.memory_budget_bytes = std::max<int64_t>(c.memory_budget_bytes, sv->bytes_per_flow);
    sv->cfg = c;
    sv->slots.resize(c.slots);
    const int64_t cap = c.max_batch_flows;
    for (Slot& s : sv->slots) {
      bool ok = cudaStreamCreateWithFlags(&s.stream, cudaStreamNonBlocking) == cudaSuccess &&
                cudaMalloc(&s.d_rows, sizeof(uint64_t) * cap * sv->K) == cudaSuccess &&
                cudaMalloc(&s.d_A, sizeof(int64_t) * cap) == cudaSuccess &&
                cudaMalloc(&s.d_N, sizeof(int64_t) * cap) == cudaSuccess &&
                cudaMalloc(&s.d_lab, cap) == cudaSuccess &&
                cudaMallocHost(&s.h_rows, sizeof(uint64_t) * cap * sv->K) == cudaSuccess &&
                cudaMallocHost(&s.h_A, sizeof(int64_t) * cap) == cudaSuccess &&
                cudaMallocHost(&s.h_N, sizeof(int64_t) * cap) == cudaSuccess &&
                cudaMallocHost(&s.h_lab, cap) == cudaSuccess;
      if (!ok) {
        ig_server_destroy(sv);
        return igk::report_error(IG_E_NOMEM, "ig_server_create: device or pinned allocation failed");
      }
    }
    for (Slot& s : sv->slots) s.thread = std::thread(slot_loop, sv, &s);
    sv->scheduler = std::thread(scheduler_loop, sv);
    *out = sv;
    return IG_OK;
  });
}

int ig_server_submit(ig_server* sv, const uint64_t* rows, int64_t m, int64_t* A_out,
                     int64_t* N_out, uint8_t* label_out, uint64_t* ticket) {
  return igk::guarded("ig_server_submit", [&]() -> int {
    if (!sv || !ticket || m <= 0 || !rows) return set_error("ig_server_submit: bad arguments");
    if (m > sv->cfg.max_batch_flows)
      return set_error("ig_server_submit: request larger than the batch cap");
    Request* r = new Request;
    r->rows = rows;
    r->m = m;
    r->A = A_out;
    r->N = N_out;
    r->labels = label_out;
    r->submitted = Clock::now();
    {
      std::lock_guard<std::mutex> lk(sv->mu);
      r->ticket = sv->next_ticket++;
      sv->live[r->ticket] = r;
      sv->queue.push_back(r);
    }
    sv->cv.notify_all();
    *ticket = r->ticket;
    return IG_OK;
  });
}

int ig_server_wait(ig_server* sv, uint64_t ticket, double* latency_ms) {
  return igk::guarded("ig_server_wait", [&]() -> int {
    if (!sv) return set_error("ig_server_wait: NULL server");
    std::unique_lock<std::mutex> lk(sv->mu);
    auto it = sv->live.find(ticket);
    if (it == sv->live.end()) return set_error("ig_server_wait: unknown ticket");
    Request* r = it->second;
    sv->done_cv.wait(lk, [&] { return r->done; });
    sv->live.erase(it);
    const int rc = r->rc;
    if (latency_ms)
      *latency_ms = std::chrono::duration<double, std::milli>(r->completed - r->submitted).count();
    std::string err = r->error;
    delete r;
    if (rc != IG_OK) return igk::report_error(rc, err.c_str());
    return rc;
  });
}

int ig_server_stats(ig_server* sv, int64_t* batches, int64_t* flows) {
  if (!sv) return set_error("ig_server_stats: NULL server");
  std::lock_guard<std::mutex> lk(sv->mu);
  if (batches) *batches = sv->batches;
  if (flows) *flows = sv->flows;
  return IG_OK;
}

void ig_server_destroy(ig_server* sv) {
  if (!sv) return;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->stop = true;
  }
  sv->cv.notify_all();
  if (sv->scheduler.joinable()) sv->scheduler.join();
  for (Slot& s : sv->slots) {
    if (s.thread.joinable()) s.thread.join();
    if (s.stream) cudaStreamSynchronize(s.stream);
    cudaFree(s.d_rows);
    cudaFree(s.d_A);
    cudaFree(s.d_N);
    cudaFree(s.d_lab);
    cudaFreeHost(s.h_rows);
    cudaFreeHost(s.h_A);
    cudaFreeHost(s.h_N);
    cudaFreeHost(s.h_lab);
    if (s.stream) cudaStreamDestroy(s.stream);
  }
  for (auto& kv : sv->live) delete kv.second;
  delete sv;
}

}  // extern "C"
