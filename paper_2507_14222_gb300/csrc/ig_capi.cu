// C ABI of the IG library (declared in include/ig.h): argument checks,
// staging of host buffers, the orchestration of IG training (Section 3.1:
// Eq. 1 -> Eq. 3 -> Eq. 2 per class, then the Regulation 3 statistics) and
// inference (Eq. 4, Regulations 1-3), model persistence and stage timing.
// Every step of the computation runs in the kernels of encode.cu, dedup.cu,
// subset.cu and sort.cu; this file only sizes buffers and launches them.
#include <cuda_runtime.h>
#include <sys/types.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <condition_variable>
#include <functional>
#include <memory>
#include <thread>
#include <mutex>
#include <string>
#include <utility>
#include <vector>

#include "../../include/ig.h"
#include "common.cuh"
#include "internal.h"

namespace {

thread_local std::string g_last_error;

int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return code;
}

int fail_cuda(cudaError_t e, const char* where) {
  if (e == cudaErrorMemoryAllocation)
    return fail(IG_E_NOMEM, "%s: device allocation failed (%s)", where,
                cudaGetErrorString(e));
  return fail(IG_E_CUDA, "%s: %s", where, cudaGetErrorString(e));
}

#define IG_CUDA(expr, where)                          \
  do {                                                \
    cudaError_t e_ = (expr);                          \
    if (e_ != cudaSuccess) return fail_cuda(e_, where); \
  } while (0)

#define IG_CHECK(expr)           \
  do {                           \
    int rc_ = (expr);            \
    if (rc_ != IG_OK) return rc_; \
  } while (0)

// ---- per-stage timing -------------------------------------------------------
const char* kStageNames[IG_PROF_STAGES] = {
    "encode",         "split",          "pair_insert",  "rehash",
    "compact",        "coherence",      "select",       "canonical_sort",
    "support",        "pattern_score",  "evidence",     "labels",
    "coherence_tc",   "support_tc",     "evidence_tc",  "expand",
    "coherence_idx",  "support_idx",    "evidence_idx", "index_build"};
enum Stage {
  S_ENCODE, S_SPLIT, S_PAIR, S_REHASH, S_COMPACT, S_COHERENCE,
  S_SELECT, S_SORT, S_SUPPORT, S_PSCORE, S_EVIDENCE, S_LABELS,
  S_COHERENCE_TC, S_SUPPORT_TC, S_EVIDENCE_TC, S_EXPAND,
  S_COHERENCE_IDX, S_SUPPORT_IDX, S_EVIDENCE_IDX, S_INDEX_BUILD
};

struct Prof {
  std::mutex mu;
  bool on = false;
  uint32_t mask = 0xffffffffu;  // stages whose launches are timed while on
  double ms[IG_PROF_STAGES] = {};
  int64_t launches[IG_PROF_STAGES] = {};
  int64_t work[IG_PROF_STAGES] = {};
  struct Pending {
    int stage;
    cudaStream_t s;
    cudaEvent_t a, b;
  };
  std::vector<Pending> pending;
  std::vector<cudaEvent_t> pool;
  // Timeline since the last reset: begin and end of every recorded stage,
  // in ms after the reference event recorded by the reset.
  cudaEvent_t ref = nullptr;
  struct Span {
    int stage;
    cudaStream_t s;
    double t0, t1;
  };
  std::vector<Span> spans;
};
Prof g_prof;

cudaEvent_t prof_event() {
  if (!g_prof.pool.empty()) {
    cudaEvent_t e = g_prof.pool.back();
    g_prof.pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// Brackets the launches of one stage with CUDA events on their stream.
struct ProfScope {
  void* token;
  ProfScope(int st, cudaStream_t stream) : token(igk::prof_begin(st, stream)) {}
  ~ProfScope() { igk::prof_end(token); }
};

struct ProfToken {
  int stage;
  cudaStream_t s;
  cudaEvent_t a;
};

void prof_drain_locked() {
  for (auto& p : g_prof.pending) {
    cudaEventSynchronize(p.b);
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
      g_prof.ms[p.stage] += ms;
      g_prof.launches[p.stage] += 1;
      float t0 = 0.f;
      if (g_prof.ref && cudaEventElapsedTime(&t0, g_prof.ref, p.a) == cudaSuccess)
        g_prof.spans.push_back({p.stage, p.s, double(t0), double(t0) + double(ms)});
    }
    cudaGetLastError();
    g_prof.pool.push_back(p.a);
    g_prof.pool.push_back(p.b);
  }
  g_prof.pending.clear();
}

// ---- device buffers ---------------------------------------------------------
// Freed stream-ordered memory stays cached in the device's default pool --
// up to an eighth of the device's memory, at most 32 GiB -- instead of going
// back to the driver at every synchronization: a fit allocates and frees its
// buffers between several synchronizations, and remapping them each time
// costs more than the kernels that use them.  Set once per device; a
// property of this process's pool, not of the GPU.
static void keep_pool_memory() {
  static std::atomic<int> done[64];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return;
  if (done[dev].load(std::memory_order_relaxed)) return;
  done[dev].store(1, std::memory_order_relaxed);
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, dev) != cudaSuccess) {
    cudaGetLastError();
    return;
  }
  size_t free_b = 0, total_b = 0;
  if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
    cudaGetLastError();
    return;
  }
  uint64_t keep = std::min<uint64_t>(uint64_t(total_b) / 8, uint64_t(32) << 30);
  if (cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep) != cudaSuccess)
    cudaGetLastError();
}

// Stream-ordered allocation; freed on the same stream when the owner goes
// out of scope (or kept by release()).
template <class T>
struct DevBuf {
  T* p = nullptr;
  cudaStream_t s = nullptr;
  DevBuf() = default;
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
  ~DevBuf() { reset(); }
  void reset() {
    if (p) cudaFreeAsync(p, s);
    p = nullptr;
  }
  cudaError_t alloc(size_t count, cudaStream_t stream) {
    reset();
    keep_pool_memory();
    s = stream;
    if (count == 0) count = 1;
    return cudaMallocAsync(reinterpret_cast<void**>(&p), count * sizeof(T), stream);
  }
  T* release() {
    T* q = p;
    p = nullptr;
    return q;
  }
};

// Pinned host words for size read-backs, one block per host thread.
unsigned long long* thread_pinned() {
  static thread_local unsigned long long* p = nullptr;
  if (!p && cudaMallocHost(&p, 8 * sizeof(unsigned long long)) != cudaSuccess) p = nullptr;
  return p;
}

// One persistent helper thread that runs a task while the caller runs
// another (used to fit the two classes concurrently).  Detached and never
// destroyed: it idles on a condition variable until the process exits.
class Worker {
 public:
  Worker() {
    std::thread([this] { loop(); }).detach();
  }
  void run(std::function<void()> f) {
    std::lock_guard<std::mutex> lk(mu_);
    task_ = std::move(f);
    pending_ = true;
    finished_ = false;
    cv_.notify_all();
  }
  void wait() {
    std::unique_lock<std::mutex> lk(mu_);
    cv_.wait(lk, [this] { return finished_; });
  }

 private:
  void loop() {
    for (;;) {
      std::function<void()> f;
      {
        std::unique_lock<std::mutex> lk(mu_);
        cv_.wait(lk, [this] { return pending_; });
        f = std::move(task_);
        pending_ = false;
      }
      f();
      std::lock_guard<std::mutex> lk(mu_);
      finished_ = true;
      cv_.notify_all();
    }
  }
  std::mutex mu_;
  std::condition_variable cv_;
  std::function<void()> task_;
  bool pending_ = false, finished_ = false;
};

// Idle helper threads, reused across calls (created on demand).
std::mutex g_pool_mu;
std::vector<Worker*> g_pool;

Worker* acquire_worker() {
  std::lock_guard<std::mutex> lk(g_pool_mu);
  if (g_pool.empty()) return new Worker();
  Worker* w = g_pool.back();
  g_pool.pop_back();
  return w;
}

void release_worker(Worker* w) {
  std::lock_guard<std::mutex> lk(g_pool_mu);
  g_pool.push_back(w);
}

// Smallest scoring batch that uses the item index (item-index models).
constexpr int64_t kIndexMinRows = 512;

// Owns a record index for the duration of a call.
struct IndexHolder {
  igk::RecordIndex idx;
  cudaStream_t s = nullptr;
  ~IndexHolder() { igk::release_record_index(&idx, s); }
};

// An input array as a device pointer: either the caller's own device array,
// or a stream-ordered device copy of the caller's host array.
template <class T>
struct InputView {
  const T* d = nullptr;
  DevBuf<T> copy;
  int bind(const T* p, size_t count, cudaStream_t s, const char* what) {
    if (count == 0) {
      d = p;
      return IG_OK;
    }
    if (igk::is_device_pointer(p)) {
      d = p;
      return IG_OK;
    }
    IG_CUDA(copy.alloc(count, s), what);
    IG_CUDA(cudaMemcpyAsync(copy.p, p, count * sizeof(T), cudaMemcpyHostToDevice, s), what);
    d = copy.p;
    return IG_OK;
  }
};

// An output array: written in place when it is on the device, otherwise
// produced in a device buffer and copied back by finish().
template <class T>
struct OutputView {
  T* user = nullptr;
  T* d = nullptr;
  size_t count = 0;
  bool host = false;
  DevBuf<T> buf;
  int bind(T* p, size_t n, cudaStream_t s, const char* what) {
    user = p;
    count = n;
    if (p && igk::is_device_pointer(p)) {
      d = p;
      return IG_OK;
    }
    host = p != nullptr;
    IG_CUDA(buf.alloc(n, s), what);
    d = buf.p;
    return IG_OK;
  }
  int finish(cudaStream_t s, const char* what) {
    if (host && count)
      IG_CUDA(cudaMemcpyAsync(user, d, count * sizeof(T), cudaMemcpyDeviceToHost, s), what);
    return IG_OK;
  }
};

int read_status(int* d_status, cudaStream_t s, const char* where) {
  int st = 0;
  IG_CUDA(cudaMemcpyAsync(&st, d_status, sizeof(int), cudaMemcpyDeviceToHost, s), where);
  IG_CUDA(cudaStreamSynchronize(s), where);
  if (st & igk::ST_BAD_INPUT)
    return fail(IG_E_INVAL, "%s: input value out of range (code >= card or label > 1)", where);
  if (st & igk::ST_TIMEOUT) return fail(IG_E_TIMEOUT, "%s: a bounded device wait ran out", where);
  if (st & igk::ST_TABLE_FULL) return fail(IG_E_INTERNAL, "%s: hash table full", where);
  if (st & igk::ST_COUNT) return fail(IG_E_INTERNAL, "%s: hash table key count mismatch", where);
  return IG_OK;
}

std::atomic<long long> g_launches{0};

}  // namespace

void* igk::prof_begin(int stage, cudaStream_t s) {
  std::lock_guard<std::mutex> lk(g_prof.mu);
  if (!g_prof.on || stage < 0 || stage >= IG_PROF_STAGES || !((g_prof.mask >> stage) & 1u))
    return nullptr;
  ProfToken* t = new ProfToken{stage, s, prof_event()};
  cudaEventRecord(t->a, s);
  return t;
}

void igk::prof_add_work(int stage, int64_t tests) {
  std::lock_guard<std::mutex> lk(g_prof.mu);
  if (g_prof.on && stage >= 0 && stage < IG_PROF_STAGES) g_prof.work[stage] += tests;
}

void igk::prof_end(void* token) {
  if (!token) return;
  ProfToken* t = static_cast<ProfToken*>(token);
  std::lock_guard<std::mutex> lk(g_prof.mu);
  cudaEvent_t b = prof_event();
  cudaEventRecord(b, t->s);
  g_prof.pending.push_back({t->stage, t->s, t->a, b});
  delete t;
}

void igk::count_launches(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

int igk::num_sms() {
  // Filled by whichever thread asks first; concurrent fillers store the same
  // value (relaxed atomics: the class and server threads call this too).
  static std::atomic<int> cached[64];
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) return 148;
  int v = cached[dev].load(std::memory_order_relaxed);
  if (!v) {
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    if (v <= 0) v = 148;
    cached[dev].store(v, std::memory_order_relaxed);
  }
  return v;
}

bool igk::device_of(const void* p, int* dev) {
  if (!p) return false;
  cudaPointerAttributes attr;
  if (cudaPointerGetAttributes(&attr, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (attr.type != cudaMemoryTypeDevice && attr.type != cudaMemoryTypeManaged) return false;
  if (attr.device < 0) return false;
  *dev = attr.device;
  return true;
}

bool igk::is_device_pointer(const void* p) {
  int owner = -1;
  if (!device_of(p, &owner)) return false;
  int cur = -1;
  if (cudaGetDevice(&cur) == cudaSuccess && cur != owner) cudaSetDevice(owner);
  return true;
}

namespace {
// A second stream for work that can overlap the caller's, with the two
// events that join it: one per host thread and device, created on first use
// and kept for the life of the process.
struct AuxStream {
  cudaStream_t s = nullptr;
  cudaEvent_t ready = nullptr, done = nullptr;
  cudaError_t error = cudaSuccess;
};
AuxStream& aux_stream() {
  static thread_local AuxStream per_dev[64];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) dev = 0;
  AuxStream& a = per_dev[dev];
  if (!a.s && a.error == cudaSuccess) {
    a.error = cudaStreamCreateWithFlags(&a.s, cudaStreamNonBlocking);
    if (a.error == cudaSuccess)
      a.error = cudaEventCreateWithFlags(&a.ready, cudaEventDisableTiming);
    if (a.error == cudaSuccess) a.error = cudaEventCreateWithFlags(&a.done, cudaEventDisableTiming);
  }
  return a;
}
}  // namespace

namespace {
// The two class streams of a fit and the three events that fork and join
// them, one set per host thread and device, created on first use and kept
// for the life of the process.
struct FitStreams {
  cudaStream_t cs[2] = {nullptr, nullptr};
  cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
  cudaError_t error = cudaSuccess;
};
FitStreams& fit_streams() {
  static thread_local FitStreams per_dev[64];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) dev = 0;
  FitStreams& f = per_dev[dev];
  if (!f.cs[0] && f.error == cudaSuccess) {
    for (int i = 0; i < 2 && f.error == cudaSuccess; ++i)
      f.error = cudaStreamCreateWithFlags(&f.cs[i], cudaStreamNonBlocking);
    for (int i = 0; i < 3 && f.error == cudaSuccess; ++i)
      f.error = cudaEventCreateWithFlags(&f.ev[i], cudaEventDisableTiming);
  }
  return f;
}
}  // namespace

struct ig_model {
  int K = 0, KT = 0;
  int64_t n_train[2] = {0, 0}, n_cand[2] = {0, 0}, n_pat[2] = {0, 0}, n_pairs[2] = {0, 0};
  uint64_t* words[2] = {nullptr, nullptr};     // stride K (API view)
  uint64_t* words_kt[2] = {nullptr, nullptr};  // stride KT, pad_rows rows
  uint32_t* support[2] = {nullptr, nullptr};
  uint64_t* score[2] = {nullptr, nullptr};     // pad_rows entries
  int reg3 = 0;
  double mu = 0, sigma = 0, r = 0, thr = 0;
  int subset_kernel = 1;  // 1 integer pipe, 2 tensor cores, 3 item index, 4 item index on tensor cores
  uint8_t* pat_img[2] = {nullptr, nullptr};    // tensor-core images of P^c
  int64_t coh_tests[2] = {0, 0};               // coherence tests executed
  int64_t coh_tests_tc[2] = {0, 0};            // ... of which on the tensor cores
  int64_t coh_tests_pruned[2] = {0, 0};        // ... of which through the item index
  int64_t sup_tests[2] = {0, 0};               // support tests executed
  igk::KeyedIndex* pidx[2] = {nullptr, nullptr};  // patterns by key item, for scoring
  int index_max_q = 4, index_flip = 2;            // item-index tiling
  uint64_t score_max[2] = {~uint64_t(0), ~uint64_t(0)};  // largest S per class (bound)
};

static void model_release(ig_model* m) {
  if (!m) return;
  for (int c = 0; c < 2; ++c) {
    if (m->pidx[c]) {
      igk::release_keyed_index(m->pidx[c], nullptr);
      delete m->pidx[c];
    }
    if (m->pat_img[c]) cudaFree(m->pat_img[c]);
    if (m->words[c] && m->words[c] != m->words_kt[c]) cudaFree(m->words[c]);
    if (m->words_kt[c]) cudaFree(m->words_kt[c]);
    if (m->support[c]) cudaFree(m->support[c]);
    if (m->score[c]) cudaFree(m->score[c]);
  }
  delete m;
}

// Files both classes' patterns under their key items for scoring: the key
// of a pattern is its item held by the fewest records according to freq
// (device, 64K entries).  Any choice keeps scoring exact; this one keeps the
// item-index work small for records like those freq was counted on.
static cudaError_t build_pattern_indexes(ig_model* m, const uint32_t* freq, cudaStream_t s) {
  for (int c = 0; c < 2; ++c) {
    if (m->n_pat[c] == 0) continue;
    igk::KeyedIndex* k = new igk::KeyedIndex;
    cudaError_t e = igk::build_keyed_index(m->words_kt[c], m->n_pat[c], m->KT, m->K, m->KT, freq,
                                           m->score[c], k, s);
    if (e != cudaSuccess) {
      delete k;
      return e;
    }
    m->pidx[c] = k;
  }
  return cudaSuccess;
}

// Item counts over the patterns of both classes (for models whose records
// are not at hand).
static cudaError_t pattern_item_freq(const ig_model* m, uint32_t* freq, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(freq, 0, sizeof(uint32_t) * 64 * m->K, s);
  for (int c = 0; c < 2 && e == cudaSuccess; ++c)
    if (m->n_pat[c])
      e = igk::launch_item_histogram(m->words_kt[c], m->n_pat[c], m->KT, m->K, 64 * m->K, freq, s);
  return e;
}

void igk::model_view(const ig_model* m, igk::ModelView* v) {
  v->K = m->K;
  v->KT = m->KT;
  for (int c = 0; c < 2; ++c) {
    v->words_kt[c] = m->words_kt[c];
    v->score[c] = m->score[c];
    v->n_pat[c] = m->n_pat[c];
  }
  v->reg3 = m->reg3;
  v->thr = m->thr;
}

int igk::report_error(int code, const char* msg) { return fail(code, "%s", msg); }

int igk::report_exception(const char* where, bool out_of_memory) noexcept {
  const int code = out_of_memory ? IG_E_NOMEM : IG_E_INTERNAL;
  try {
    return fail(code, "%s: %s", where,
                out_of_memory ? "host memory allocation failed" : "unexpected host exception");
  } catch (...) {
    return code;
  }
}

namespace {

// The distinct rows of X[0, n) (stride KT), in any order, into Xu, their
// number into *d_nu (on the device).  B^c of Eq. 1 is a set: a repeated
// record adds no intersection its first copy does not (x AND x = x), so the
// pair stage needs each record once -- at NSL-KDD shape a quarter of the
// training records repeat, and the pairs fall to about 55%.
int unique_rows(const uint64_t* X, int64_t n, int KT, DevBuf<uint64_t>& Xu,
                unsigned long long* d_nu, cudaStream_t s) {
  uint64_t cap = 1024;
  while (cap < 2 * uint64_t(n)) cap <<= 1;
  DevBuf<uint32_t> table, flag;
  IG_CUDA(table.alloc(cap, s), "ig_fit: distinct records");
  IG_CUDA(flag.alloc(size_t(n), s), "ig_fit: distinct records");
  IG_CUDA(Xu.alloc(size_t(n) * KT, s), "ig_fit: distinct records");
  IG_CUDA(cudaMemsetAsync(table.p, 0xff, cap * sizeof(uint32_t), s), "ig_fit");
  IG_CUDA(cudaMemsetAsync(d_nu, 0, sizeof(unsigned long long), s), "ig_fit");
  ProfScope ps(S_SPLIT, s);
  IG_CUDA(igk::launch_mark_repeats(X, n, KT, table.p, cap, flag.p, s), "ig_fit: distinct records");
  IG_CUDA(igk::launch_select_unflagged(X, n, KT, flag.p, Xu.p, d_nu, s),
          "ig_fit: distinct records");
  return IG_OK;
}

// Candidate generation (Eq. 1) for one class, deduplicated on the device.
// One launch covers every pair band; if the table runs out of room the
// launch records the lowest band that failed, and the table is doubled,
// rehashed and the bands from that one on are replayed (inserts are
// idempotent).  The table starts at twice a guess of |B^c| (an eighth of the
// pairs, at least 16 keys per record), so typical workloads need one launch.
struct TableCounters {
  unsigned long long count;
  int failed_band;
  int pad;
};

// Slots one pair insert may probe before its band is replayed on a grown
// table.  At the load factors used (at most one half) linear probing
// almost never comes near it.
constexpr uint64_t kMaxProbe = 512;

// Hand-over between the two class threads of a fit: each prepares its own
// side (record index, image), records an event on its stream and marks
// itself ready; a thread that needs the other side waits for that mark
// (bounded) and orders its stream after the event.  A thread that fails
// before it is ready marks itself failed, so the other never waits in vain.
struct SideSync {
  std::mutex mu;
  std::condition_variable cv;
  int state[2] = {0, 0};  // 0 pending, 1 ready, -1 failed
  cudaEvent_t ev[2] = {nullptr, nullptr};
  ~SideSync() {
    for (cudaEvent_t e : ev)
      if (e) cudaEventDestroy(e);
  }
  void mark(int c, int st) {
    {
      std::lock_guard<std::mutex> lk(mu);
      if (state[c] == 0) state[c] = st;
    }
    cv.notify_all();
  }
  int wait(int c, cudaStream_t s) {
    std::unique_lock<std::mutex> lk(mu);
    if (!cv.wait_for(lk, std::chrono::seconds(600), [&] { return state[c] != 0; }))
      return fail(IG_E_TIMEOUT, "ig_fit: the other class's record index never came");
    if (state[c] < 0) return fail(IG_E_INTERNAL, "ig_fit: the other class failed");
    IG_CUDA(cudaStreamWaitEvent(s, ev[c], 0), "ig_fit");
    return IG_OK;
  }
};

struct SideSignal {
  SideSync* sync;
  int c;
  cudaError_t ready(cudaStream_t s) {
    cudaError_t e = cudaEventCreateWithFlags(&sync->ev[c], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventRecord(sync->ev[c], s);
    sync->mark(c, e == cudaSuccess ? 1 : -1);
    return e;
  }
  ~SideSignal() { sync->mark(c, -1); }  // no effect once ready
};

constexpr int kNoBand = 0x7f7f7f7f;  // failed_band after a 0x7f byte fill

// One class's hash set of candidate keys (Eq. 1) between its pair stage and
// its compaction.
struct CandTable {
  DevBuf<uint64_t> slots;
  uint64_t cap = 0;
};

igk::PairTable make_table(uint64_t* slots, uint64_t cap, TableCounters* t, uint64_t max_probe) {
  igk::PairTable pt;
  pt.slots = slots;
  pt.mask = cap - 1;
  pt.count = &t->count;
  pt.limit = cap / 2;
  pt.max_probe = max_probe;
  pt.failed_band = &t->failed_band;
  return pt;
}

// The table's first capacity: twice a guess of |B^c| (an eighth of the
// pairs, at least 16 keys per record), a power of two.
uint64_t initial_cap(int64_t n) {
  const int64_t pairs = n * (n + 1) / 2;
  const int64_t guess = std::max<int64_t>(pairs / 8, 16 * n);
  uint64_t cap = 1u << 12;
  while (cap < uint64_t(2 * guess)) cap <<= 1;
  return cap;
}

cudaError_t alloc_table(CandTable& tab, uint64_t cap, cudaStream_t s) {
  tab.cap = cap;
  cudaError_t e = tab.slots.alloc(cap, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(tab.slots.p, 0, cap * sizeof(uint64_t), s);
  return e;
}

// After a pair launch whose band `failed` ran out of room: a larger table,
// rehashed from the old one.  The bands before the failed one held
// `pairs_before` pairs and gave `count` keys; the new table is sized for
// twice the count projected at that rate over all pairs (at least doubling),
// so that one growth is usually enough.  The table's counters (d_ctr) are
// reused: they count the rehashed keys, and failed_band must be reset
// before the replay.
int grow_table(const uint64_t* X, int64_t n, int KT, CandTable& tab, TableCounters* d_ctr,
               int64_t failed, unsigned long long count, int* d_status, cudaStream_t s) {
  const int64_t pairs = n * (n + 1) / 2;
  const int64_t T = igk::kPairTile, nt = igk::ceil_div(n, T);
  int64_t pairs_before = 0, pairs_all = 0;  // tile-granular pair counts
  for (int64_t r = 0; r < nt; ++r) {
    const int64_t band = (nt - r) * T * T;
    pairs_all += band;
    if (r < failed) pairs_before += band;
  }
  const double rate = double(count) / double(std::max<int64_t>(1, pairs_before));
  const double projected = std::min(double(pairs), rate * double(pairs_all)) * 1.25;
  uint64_t ncap = tab.cap << 1;
  while (double(ncap) < 2.0 * projected && ncap < (uint64_t(1) << 36)) ncap <<= 1;
  CandTable grown;
  IG_CUDA(alloc_table(grown, ncap, s), "ig_fit: hash table");
  IG_CUDA(cudaMemsetAsync(d_ctr, 0, sizeof(TableCounters), s), "ig_fit");
  {
    ProfScope ps(S_REHASH, s);
    // The grown table is at most a quarter full: every rehashed key finds
    // a slot (probing is unbounded here).
    IG_CUDA(igk::launch_rehash(X, tab.slots.p, tab.cap, make_table(grown.slots.p, ncap, d_ctr, ncap),
                               KT, d_status, s),
            "ig_fit: rehash");
  }
  std::swap(tab.slots.p, grown.slots.p);  // the old slots are freed (after the rehash) on s
  tab.cap = ncap;
  return IG_OK;
}

// Appends the U keys of a finished table to `cand` (canonical order comes
// later) and frees the table.
int compact_table(const uint64_t* X, int KT, CandTable& tab, int64_t U, int* d_status,
                  DevBuf<uint64_t>& cand, cudaStream_t s) {
  if (U > int64_t(0xffffffffll)) return fail(IG_E_OVERFLOW, "ig_fit: too many candidates");
  IG_CUDA(cand.alloc(size_t(igk::pad_rows(U)) * KT, s), "ig_fit: candidates");
  DevBuf<unsigned long long> out_count;
  IG_CUDA(out_count.alloc(1, s), "ig_fit");
  IG_CUDA(cudaMemsetAsync(out_count.p, 0, sizeof(unsigned long long), s), "ig_fit");
  {
    ProfScope ps(S_COMPACT, s);
    IG_CUDA(igk::launch_compact(X, tab.slots.p, tab.cap, KT, cand.p, U, out_count.p, d_status, s),
            "ig_fit: compact");
  }
  tab.slots.s = s;
  tab.slots.reset();
  return IG_OK;
}

// Candidate generation (Eq. 1) for one class, deduplicated on the device.
// One launch covers every pair band; if the table runs out of room the
// launch records the lowest band that failed, and the table is grown,
// rehashed and the bands from that one on are replayed (inserts are
// idempotent).  Typical workloads need one launch.
int build_candidates(const uint64_t* Xall, int64_t n, int KT, cudaStream_t s, int* d_status,
                     TableCounters* h_counters, DevBuf<uint64_t>& cand, int64_t* U_out) {
  if (n > int64_t(65535) * igk::kPairTile)
    return fail(IG_E_OVERFLOW, "ig_fit: more than 4,194,240 records in one class");
  // Pairs of distinct records only; their count stays on the device (n
  // sizes the grids).
  DevBuf<uint64_t> Xu;
  DevBuf<unsigned long long> d_nu;
  IG_CUDA(d_nu.alloc(1, s), "ig_fit: distinct records");
  IG_CHECK(unique_rows(Xall, n, KT, Xu, d_nu.p, s));
  const uint64_t* X = Xu.p;
  CandTable tab;
  DevBuf<TableCounters> ctr;
  IG_CUDA(ctr.alloc(1, s), "ig_fit: table counters");
  IG_CUDA(cudaMemsetAsync(ctr.p, 0, sizeof(TableCounters), s), "ig_fit");
  IG_CUDA(alloc_table(tab, initial_cap(n), s), "ig_fit: hash table");
  int64_t band_lo = 0;
  for (;;) {
    // failed_band = none, then insert the bands.
    IG_CUDA(cudaMemsetAsync(&ctr.p->failed_band, 0x7f, sizeof(int), s), "ig_fit");
    {
      ProfScope ps(S_PAIR, s);
      IG_CUDA(igk::launch_pair_insert(X, n, KT, band_lo,
                                      make_table(tab.slots.p, tab.cap, ctr.p, kMaxProbe), d_status,
                                      s, d_nu.p),
              "ig_fit: pair intersection");
    }
    IG_CUDA(cudaMemcpyAsync(h_counters, ctr.p, sizeof(TableCounters), cudaMemcpyDeviceToHost, s),
            "ig_fit");
    IG_CUDA(cudaStreamSynchronize(s), "ig_fit");
    if (h_counters->failed_band == kNoBand) break;
    band_lo = h_counters->failed_band;
    IG_CHECK(grow_table(X, n, KT, tab, ctr.p, band_lo, h_counters->count, d_status, s));
  }
  IG_CHECK(read_status(d_status, s, "ig_fit: candidate generation"));
  const int64_t U = int64_t(h_counters->count);
  IG_CHECK(compact_table(X, KT, tab, U, d_status, cand, s));
  *U_out = U;
  return IG_OK;
}

// What the batched candidate stage hands to a problem's fit: its class
// matrices and, per class, the finished table of candidate keys.
struct FitPrep {
  bool ready = false;
  DevBuf<uint64_t> X[2];
  DevBuf<uint64_t> Xu[2];  // the distinct records of each class (the pair stage's rows)
  int64_t nc[2] = {0, 0};
  CandTable tab[2];
  int64_t count[2] = {0, 0};
};

}  // namespace

extern "C" {

const char* ig_last_error(void) { return g_last_error.c_str(); }

int ig_encode(const uint16_t* codes, int64_t n, int32_t F, const uint16_t* cards,
              uint64_t* words_out, int32_t K, ig_stream_t stream) {
  return igk::guarded("ig_encode", [&]() -> int {
    igk::DeviceRestore restore_device;  // the caller's device, put back on return
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (n < 0 || F <= 0 || !cards || (n > 0 && (!codes || !words_out)))
      return fail(IG_E_INVAL, "ig_encode: bad arguments");
    std::vector<uint32_t> offsets(F + 1, 0);
    for (int f = 0; f < F; ++f) {
      if (cards[f] == 0) return fail(IG_E_INVAL, "ig_encode: feature %d has cardinality 0", f);
      offsets[f + 1] = offsets[f] + cards[f];
    }
    const int64_t L = offsets[F];
    if (K != int32_t((L + 63) / 64))
      return fail(IG_E_INVAL, "ig_encode: K = %d but ceil(L/64) = %lld", K, (long long)((L + 63) / 64));
    if (K < 1 || K > IG_MAX_WORDS) return fail(IG_E_INVAL, "ig_encode: K = %d out of range", K);
    if (n == 0) return IG_OK;
    InputView<uint16_t> in;
    IG_CHECK(in.bind(codes, size_t(n) * F, s, "ig_encode: codes"));
    OutputView<uint64_t> out;
    IG_CHECK(out.bind(words_out, size_t(n) * K, s, "ig_encode: output"));
    DevBuf<uint32_t> d_off;
    DevBuf<int> d_status;
    IG_CUDA(d_off.alloc(F + 1, s), "ig_encode");
    IG_CUDA(d_status.alloc(1, s), "ig_encode");
    IG_CUDA(cudaMemcpyAsync(d_off.p, offsets.data(), sizeof(uint32_t) * (F + 1),
                            cudaMemcpyHostToDevice, s),
            "ig_encode");
    IG_CUDA(cudaMemsetAsync(d_status.p, 0, sizeof(int), s), "ig_encode");
    {
      ProfScope ps(S_ENCODE, s);
      IG_CUDA(igk::launch_encode(in.d, n, F, d_off.p, nullptr, out.d, K, d_status.p, s),
              "ig_encode: kernel");
    }
    IG_CHECK(out.finish(s, "ig_encode: copy back"));
    return read_status(d_status.p, s, "ig_encode");
  });
}

}  // extern "C"

namespace {

// ig_fit's body.  With `prep` (from ig_fit_batched's candidate stage) the
// class matrices and the candidate tables are already built: the split and
// the pair stage are skipped and each class starts at its compaction.
int fit_impl(const uint64_t* rows, const uint8_t* labels, int64_t n, int32_t K,
             const ig_params* params, ig_model** out, cudaStream_t s, FitPrep* prep) {
  if (!out) return fail(IG_E_INVAL, "ig_fit: out is NULL");
  *out = nullptr;
  if (!rows || !labels || n < 2) return fail(IG_E_INVAL, "ig_fit: need at least two records");
  if (K < 1 || K > IG_MAX_WORDS) return fail(IG_E_INVAL, "ig_fit: K = %d out of range", K);
  if (n > int64_t(0x7fffffff)) return fail(IG_E_OVERFLOW, "ig_fit: too many records");
  ig_params prm{0.0, 0, 0, 0, 0};
  if (params) prm = *params;
  if (prm.index_max_q != 0 && prm.index_max_q != 1 && prm.index_max_q != 2 &&
      prm.index_max_q != 4)
    return fail(IG_E_INVAL, "ig_fit: index_max_q must be 0, 1, 2 or 4");
  if (prm.index_flip_factor < 0) return fail(IG_E_INVAL, "ig_fit: negative index_flip_factor");
  if (prm.subset_kernel < 0 || prm.subset_kernel > 4)
    return fail(IG_E_INVAL, "ig_fit: unknown subset_kernel %d", prm.subset_kernel);
  if (prm.reg3_enabled && !std::isfinite(prm.r))
    return fail(IG_E_INVAL, "ig_fit: Regulation 3 needs a finite r");
  const int KT = igk::padded_words(K);

  InputView<uint64_t> in_rows;
  InputView<uint8_t> in_lab;
  if (!prep) {
    IG_CHECK(in_rows.bind(rows, size_t(n) * K, s, "ig_fit: rows"));
    IG_CHECK(in_lab.bind(labels, size_t(n), s, "ig_fit: labels"));
  }

  DevBuf<int> d_status;
  DevBuf<unsigned long long> d_counts;
  IG_CUDA(d_status.alloc(1, s), "ig_fit");
  IG_CUDA(d_counts.alloc(2, s), "ig_fit");
  IG_CUDA(cudaMemsetAsync(d_status.p, 0, sizeof(int), s), "ig_fit");
  // Pinned host words for read-backs: [0..1] class counts, [2..3] the
  // classes' largest scores, [4..5] and [6..7] the coherence and support
  // tests of the item-index rounds (the tensor-core form copies them when
  // its stream gets there), [8] those of the Regulation 3 evidence.
  static thread_local unsigned long long* h_pinned = nullptr;
  if (!h_pinned) IG_CUDA(cudaMallocHost(&h_pinned, 16 * sizeof(unsigned long long)), "ig_fit");
  // [2 + c]: the largest score of class c, copied back by its class stream.
  unsigned long long* const h_smax = h_pinned + 2;
  int64_t* const h_tests = reinterpret_cast<int64_t*>(h_pinned + 4);
  for (int i = 0; i < 5; ++i) h_tests[i] = 0;
  bool sup_idx_ran[2] = {false, false};

  // Section 3.2: class-stacked row matrices (normal -> X[0], attack -> X[1]).
  DevBuf<uint64_t> X[2];
  int64_t nc[2];
  if (prep) {
    for (int c = 0; c < 2; ++c) {
      X[c].p = prep->X[c].release();
      X[c].s = s;
      nc[c] = prep->nc[c];
    }
  } else {
    // One spare tile of rows beyond the padding: record windows of the
    // coherence rounds may start at any multiple of 32 rows.
    for (int c = 0; c < 2; ++c)
      IG_CUDA(X[c].alloc(size_t(igk::pad_rows(n) + igk::kRowPad) * KT, s), "ig_fit: rows");
    {
      ProfScope ps(S_SPLIT, s);
      IG_CUDA(igk::launch_split(in_rows.d, in_lab.d, n, K, KT, X[0].p, X[1].p, d_counts.p,
                                d_status.p, s),
              "ig_fit: split");
    }
    IG_CUDA(cudaMemcpyAsync(h_pinned, d_counts.p, 2 * sizeof(unsigned long long),
                            cudaMemcpyDeviceToHost, s),
            "ig_fit");
    IG_CHECK(read_status(d_status.p, s, "ig_fit: labels"));
    nc[0] = int64_t(h_pinned[0]);
    nc[1] = int64_t(h_pinned[1]);
  }
  if (nc[0] == 0 || nc[1] == 0) return fail(IG_E_INVAL, "ig_fit: both classes must be non-empty");

  ig_model* m = new ig_model;
  struct ModelGuard {
    ig_model* m;
    ~ModelGuard() { model_release(m); }
  } guard{m};
  m->K = K;
  m->KT = KT;
  // Subset-test form: the item index (default, and where K allows it), the
  // tensor-core GEMM, or the plain integer-pipe kernel.  Dense steps of the
  // index form run on the tensor cores where K allows.
  const bool pruned =
      (prm.subset_kernel == 0 || prm.subset_kernel == 3 || prm.subset_kernel == 4) && KT >= 2;
  const bool tc = prm.subset_kernel != 1 && igk::tc_supported(KT);
  const bool index_tc =
      (prm.subset_kernel == 0 || prm.subset_kernel == 4) && igk::tc_supported(KT);
  m->subset_kernel = pruned ? (index_tc ? 4 : 3) : (tc ? 2 : 1);
  m->index_max_q = prm.index_max_q ? prm.index_max_q : 4;
  m->index_flip = prm.index_flip_factor ? prm.index_flip_factor : 2;
  // Item indexes of both classes' records: used by the other class's
  // coherence, this class's support and (normal class) Regulation 3.  And
  // complemented images of the records for the tensor cores: the stream
  // operand of the other class's coherence and of this class's support, and
  // the own operand of the Regulation 3 evidence; with the item index they
  // are only needed where an index could not be used.  Each class thread
  // prepares its own side first, then tells the other (side_ready).
  IndexHolder rec_idx[2];
  DevBuf<uint8_t> rec_img[2];
  SideSync side_sync;

  // The two classes are fitted concurrently, each on its own stream (class
  // + on a worker thread, class - on the calling thread), so that the
  // kernels of one class run while the other waits for a size read-back.
  auto fit_class = [&](int c, cudaStream_t s) -> int {
    const int o = 1 - c;
    SideSignal signal{&side_sync, c};
    // This class's record index and image, for both classes' later steps.
    if (pruned) {
      rec_idx[c].s = s;
      IG_CUDA(igk::build_record_index(X[c].p, nc[c], KT, K, KT, 0.25, &rec_idx[c].idx, s),
              "ig_fit: record index");
    }
    if (tc && !(pruned && rec_idx[c].idx.usable)) {
      IG_CUDA(rec_img[c].alloc(igk::tc_image_bytes(nc[c], KT, false), s), "ig_fit: images");
      ProfScope ps(S_EXPAND, s);
      IG_CUDA(igk::launch_expand(X[c].p, nc[c], KT, KT, true, false, rec_img[c].p, s),
              "ig_fit: expand");
    }
    IG_CUDA(signal.ready(s), "ig_fit");
    bool other_ready = false;
    unsigned long long* h_own = thread_pinned();  // this class thread's pinned words
    if (!h_own) return fail(IG_E_CUDA, "ig_fit: pinned host allocation failed");
    TableCounters* h_counters = reinterpret_cast<TableCounters*>(h_own + 4);
    m->n_train[c] = nc[c];
    m->n_pairs[c] = nc[c] * (nc[c] - 1) / 2;
    // Eq. 1: B^c, deduplicated on the device.
    DevBuf<uint64_t> cand;
    int64_t U = 0;
    if (prep) {
      U = prep->count[c];
      prep->Xu[c].s = s;
      IG_CHECK(compact_table(prep->Xu[c].p, KT, prep->tab[c], U, d_status.p, cand, s));
      prep->Xu[c].reset();
    } else {
      IG_CHECK(build_candidates(X[c].p, nc[c], KT, s, d_status.p, h_counters, cand, &U));
    }
    m->n_cand[c] = U;
    // Eq. 3 (tested as Eq. 6): drop candidates inside any opposite record.
    // The opposite records are tested in growing windows; after each window
    // the candidates already found inside a record are dropped, so the long
    // tail of records is only tested against the candidates still standing.
    // Row counts stay on the device between rounds.
    DevBuf<uint32_t> covered;
    DevBuf<uint64_t> surv;
    DevBuf<unsigned long long> d_kept;
    const int64_t windows[] = {0, 32, 128, 512, 2048};
    const int nwin = int(sizeof(windows) / sizeof(windows[0]));
    // With tensor cores the last window starts at 512 (a whole number of
    // 128-row tiles) and runs as one 0/1 GEMM.
    const int64_t tc_from = 512;
    IG_CUDA(covered.alloc(size_t(U), s), "ig_fit");
    IG_CUDA(surv.alloc(size_t(igk::pad_rows(U)) * KT, s), "ig_fit");
    IG_CUDA(d_kept.alloc(nwin, s), "ig_fit");
    IG_CUDA(cudaMemsetAsync(d_kept.p, 0, sizeof(unsigned long long) * nwin, s), "ig_fit");
    uint64_t* cur = cand.p;
    uint64_t* nxt = surv.p;
    const unsigned long long* cur_n_dev = nullptr;
    int64_t win_lo[8], win_hi[8];
    int rounds = 0;
    // With the item index, records from 128 on are tested in one indexed
    // round; with tensor cores (and no index), from 512 on in one GEMM round.
    const int64_t pruned_from = 128;
    int64_t round_tests[8];   // tests of an indexed round, or -1 for dense
    for (int wi = 0; wi < nwin && windows[wi] < nc[o]; ++wi) {
      const int64_t lo = windows[wi];
      int64_t hi = (wi + 1 < nwin && windows[wi + 1] < nc[o]) ? windows[wi + 1] : nc[o];
      const bool pruned_round = pruned && lo == pruned_from;
      const bool tc_round = !pruned && tc && lo >= tc_from;
      if (pruned_round || tc_round) hi = nc[o];
      if ((pruned_round || tc_round) && !other_ready) {
        // The other class's record index / image, prepared by its thread.
        IG_CHECK(side_sync.wait(o, s));
        other_ready = true;
      }
      unsigned long long* kept = d_kept.p + rounds;
      round_tests[rounds] = -1;
      IG_CUDA(cudaMemsetAsync(covered.p, 0, sizeof(uint32_t) * U, s), "ig_fit");
      bool done_round = false;
      if (pruned_round) {
        // The candidates left are counted on the device (U bounds them).
        if (rec_idx[o].idx.usable) {
          igk::IndexedArgs a;
          a.mode = igk::MODE_ANY;
          a.index = &rec_idx[o].idx;
          a.keyed = cur;
          a.n_keyed = U;
          a.n_keyed_dev = cur_n_dev;
          a.keyed_stride = KT;
          a.keyed_score = nullptr;
          a.out_u32 = covered.p;
          a.out_u64 = nullptr;
          a.status = d_status.p;
          a.tests_out = h_tests + c;  // read after the round's read-back below
          a.prof_stage = S_COHERENCE_IDX;
          a.max_q = m->index_max_q;
          a.flip_factor = m->index_flip;
          a.tc = m->subset_kernel == 4 ? 1 : 0;
          IG_CUDA(igk::indexed_subset(a, s), "ig_fit: coherence");
          round_tests[rounds] = -2;  // in h_tests[c]
          done_round = true;
        }
      }
      if (!done_round && rec_img[o].p && (tc_round || (pruned_round && tc && lo % 128 == 0))) {
        DevBuf<uint8_t> own_img;
        IG_CUDA(own_img.alloc(igk::tc_image_bytes(U, KT, true), s), "ig_fit: images");
        {
          ProfScope pe(S_EXPAND, s);
          IG_CUDA(igk::launch_expand(cur, U, KT, KT, false, true, own_img.p, s), "ig_fit: expand");
        }
        ProfScope ps(S_COHERENCE_TC, s);
        igk::TcArgs a{igk::MODE_ANY, KT,        own_img.p, U,       cur_n_dev, rec_img[o].p,
                      lo / 128,      hi - lo,   nullptr,   covered.p, nullptr, d_status.p};
        IG_CUDA(igk::launch_subset_tc(a, s), "ig_fit: coherence");
        done_round = true;
      }
      if (!done_round) {
        ProfScope ps(S_COHERENCE, s);
        igk::SubsetArgs a{igk::MODE_ANY, KT,      cur,     U,          KT,       X[o].p + lo * KT,
                          nullptr,        hi - lo, covered.p, nullptr, d_status.p, cur_n_dev};
        IG_CUDA(igk::launch_subset(a, s), "ig_fit: coherence");
      }
      {
        ProfScope ps(S_SELECT, s);
        IG_CUDA(igk::launch_select_unflagged(cur, U, KT, covered.p, nxt, kept, s, cur_n_dev),
                "ig_fit: select");
      }
      win_lo[rounds] = lo;
      win_hi[rounds] = hi;
      ++rounds;
      cur_n_dev = kept;
      std::swap(cur, nxt);
      if (hi == nc[o]) break;
    }
    unsigned long long kept_h[8] = {0};
    IG_CUDA(cudaMemcpyAsync(kept_h, d_kept.p, sizeof(unsigned long long) * rounds,
                            cudaMemcpyDeviceToHost, s),
            "ig_fit");
    IG_CHECK(read_status(d_status.p, s, "ig_fit: coherence"));
    h_own[2] = kept_h[rounds - 1];
    m->coh_tests[c] = m->coh_tests_tc[c] = m->coh_tests_pruned[c] = 0;
    for (int r = 0; r < rounds; ++r) {
      if (round_tests[r] == -2) {
        m->coh_tests[c] += h_tests[c];
        m->coh_tests_pruned[c] += h_tests[c];
        continue;
      }
      const int64_t t = int64_t(r == 0 ? U : kept_h[r - 1]) * (win_hi[r] - win_lo[r]);
      m->coh_tests[c] += t;
      if (tc && win_lo[r] >= (pruned ? pruned_from : tc_from)) m->coh_tests_tc[c] += t;
    }
    const int64_t P = int64_t(h_own[2]);
    m->n_pat[c] = P;
    covered.reset();
    // Canonical order of P^c (the other buffer serves as sort workspace).
    uint64_t* spare = (cur == cand.p) ? surv.p : cand.p;
    IG_CUDA(cudaMallocAsync(reinterpret_cast<void**>(&m->words_kt[c]),
                            sizeof(uint64_t) * std::max<int64_t>(1, igk::pad_rows(P)) * KT, s),
            "ig_fit: patterns");
    {
      ProfScope ps(S_SORT, s);
      IG_CUDA(igk::canonical_sort(cur, P, KT, m->words_kt[c], spare, s), "ig_fit: canonical sort");
    }
    cand.reset();
    surv.reset();
    // Eq. 2: support f_c and score S_c = f_c * |b|^2.
    IG_CUDA(cudaMallocAsync(reinterpret_cast<void**>(&m->support[c]),
                            sizeof(uint32_t) * std::max<int64_t>(1, P), s),
            "ig_fit: supports");
    IG_CUDA(cudaMemsetAsync(m->support[c], 0, sizeof(uint32_t) * std::max<int64_t>(1, P), s),
            "ig_fit");
    bool support_done = false;
    m->sup_tests[c] = P * nc[c];
    if (pruned) {
      if (rec_idx[c].idx.usable) {
        igk::IndexedArgs a;
        a.mode = igk::MODE_COUNT;
        a.index = &rec_idx[c].idx;
        a.keyed = m->words_kt[c];
        a.n_keyed = P;
        a.keyed_stride = KT;
        a.keyed_score = nullptr;
        a.out_u32 = m->support[c];
        a.out_u64 = nullptr;
        a.status = d_status.p;
        a.tests_out = h_tests + 2 + c;  // read after the fit's last read-back
        a.prof_stage = S_SUPPORT_IDX;
        a.max_q = m->index_max_q;
        a.flip_factor = m->index_flip;
        a.tc = m->subset_kernel == 4 ? 1 : 0;
        IG_CUDA(igk::indexed_subset(a, s), "ig_fit: support");
        support_done = true;
        sup_idx_ran[c] = true;
      }
    }
    if (support_done) {
    } else if (tc && rec_img[c].p) {
      DevBuf<uint8_t> own_img;
      IG_CUDA(own_img.alloc(igk::tc_image_bytes(P, KT, true), s), "ig_fit: images");
      {
        ProfScope pe(S_EXPAND, s);
        IG_CUDA(igk::launch_expand(m->words_kt[c], P, KT, KT, false, true, own_img.p, s),
                "ig_fit: expand");
      }
      igk::prof_add_work(S_SUPPORT_TC, P * nc[c]);
      ProfScope ps(S_SUPPORT_TC, s);
      igk::TcArgs a{igk::MODE_COUNT, KT,      own_img.p,      P,       nullptr, rec_img[c].p,
                    0,               nc[c],   nullptr,        m->support[c], nullptr,
                    d_status.p};
      IG_CUDA(igk::launch_subset_tc(a, s), "ig_fit: support");
    } else {
      igk::prof_add_work(S_SUPPORT, P * nc[c]);
      ProfScope ps(S_SUPPORT, s);
      igk::SubsetArgs a{igk::MODE_COUNT, KT, m->words_kt[c], P, KT, X[c].p, nullptr, nc[c],
                        m->support[c], nullptr, d_status.p};
      IG_CUDA(igk::launch_subset(a, s), "ig_fit: support");
    }
    if (tc && P && !pruned) {  // stream image of P^c for the evidence kernels
      IG_CUDA(cudaMallocAsync(reinterpret_cast<void**>(&m->pat_img[c]),
                              igk::tc_image_bytes(P, KT, false), s),
              "ig_fit: images");
      ProfScope pe(S_EXPAND, s);
      IG_CUDA(igk::launch_expand(m->words_kt[c], P, KT, KT, false, false, m->pat_img[c], s),
              "ig_fit: expand");
    }
    const size_t npad = size_t(std::max<int64_t>(1, igk::pad_rows(P)));
    IG_CUDA(cudaMallocAsync(reinterpret_cast<void**>(&m->score[c]), sizeof(uint64_t) * npad, s),
            "ig_fit: scores");
    IG_CUDA(cudaMemsetAsync(m->score[c], 0, sizeof(uint64_t) * npad, s), "ig_fit");
    {
      DevBuf<unsigned long long> d_smax;
      IG_CUDA(d_smax.alloc(1, s), "ig_fit");
      IG_CUDA(cudaMemsetAsync(d_smax.p, 0, sizeof(unsigned long long), s), "ig_fit");
      ProfScope ps(S_PSCORE, s);
      IG_CUDA(igk::launch_pattern_score(m->words_kt[c], P, KT, m->support[c], m->score[c], s,
                                        d_smax.p),
              "ig_fit: score");
      IG_CUDA(cudaMemcpyAsync(h_smax + c, d_smax.p, sizeof(unsigned long long),
                              cudaMemcpyDeviceToHost, s),
              "ig_fit");
    }
    if (K == KT) {
      m->words[c] = m->words_kt[c];
    } else {
      IG_CUDA(cudaMallocAsync(reinterpret_cast<void**>(&m->words[c]),
                              sizeof(uint64_t) * std::max<int64_t>(1, P) * K, s),
              "ig_fit");
      if (P)
        IG_CUDA(cudaMemcpy2DAsync(m->words[c], K * sizeof(uint64_t), m->words_kt[c],
                                  KT * sizeof(uint64_t), K * sizeof(uint64_t), P,
                                  cudaMemcpyDeviceToDevice, s),
                "ig_fit");
    }
    // Scoring's pattern index of this class, keyed by the item counts of
    // both classes' training records (from the two record indexes).
    if (pruned && P) {
      if (!other_ready) {
        IG_CHECK(side_sync.wait(o, s));
        other_ready = true;
      }
      if (rec_idx[0].idx.usable && rec_idx[1].idx.usable) {
        const int L = 64 * K;
        std::vector<uint32_t> f(L);
        for (int l = 0; l < L; ++l)
          f[l] = (rec_idx[0].idx.h_off[l + 1] - rec_idx[0].idx.h_off[l]) +
                 (rec_idx[1].idx.h_off[l + 1] - rec_idx[1].idx.h_off[l]);
        DevBuf<uint32_t> d_f;
        IG_CUDA(d_f.alloc(L, s), "ig_fit");
        IG_CUDA(cudaMemcpyAsync(d_f.p, f.data(), sizeof(uint32_t) * L, cudaMemcpyHostToDevice, s),
                "ig_fit");
        igk::KeyedIndex* k = new igk::KeyedIndex;
        // The tensor-core scoring builds its work items on the device and
        // needs no host offsets (and this fit no read-back).
        const cudaError_t e = igk::build_keyed_index(m->words_kt[c], P, KT, K, KT, d_f.p,
                                                     m->score[c], k, s, nullptr,
                                                     !(m->subset_kernel == 4 &&
                                                       igk::tc_supported(KT)));
        if (e != cudaSuccess) delete k;
        IG_CUDA(e, "ig_fit: pattern index");
        m->pidx[c] = k;
      }
    }
    return IG_OK;
  };
  {
    int dev = 0;
    IG_CUDA(cudaGetDevice(&dev), "ig_fit");
    FitStreams& fs = fit_streams();
    IG_CUDA(fs.error, "ig_fit: class streams");
    cudaStream_t* cs = fs.cs;
    cudaEvent_t* ev = fs.ev;
    IG_CUDA(cudaEventRecord(ev[2], s), "ig_fit");
    for (int i = 0; i < 2; ++i) IG_CUDA(cudaStreamWaitEvent(cs[i], ev[2], 0), "ig_fit");
    int rc[2] = {IG_OK, IG_OK};
    std::string msg[2];
    {
      Worker* w = acquire_worker();
      w->run([&] {
        cudaSetDevice(dev);
        rc[1] = igk::guarded("ig_fit", [&]() -> int {
          const int r = fit_class(1, cs[1]);
          if (r != IG_OK) msg[1] = g_last_error;
          return r;
        });
      });
      // Guarded on this thread too: nothing may unwind this frame while the
      // helper thread still uses it.
      rc[0] = igk::guarded("ig_fit", [&]() -> int {
        const int r = fit_class(0, cs[0]);
        if (r != IG_OK) msg[0] = g_last_error;
        return r;
      });
      w->wait();
      release_worker(w);
    }
    for (int i = 0; i < 2; ++i) {
      cudaEventRecord(ev[i], cs[i]);
      cudaStreamWaitEvent(s, ev[i], 0);
      // What the class streams allocated for later steps is freed on s.
      rec_idx[i].s = s;
      rec_img[i].s = s;
    }
    // Report a class's own failure before one that only saw the other fail.
    int first = -1;
    for (int i = 1; i >= 0; --i)
      if (rc[i] != IG_OK && (first < 0 || msg[first].find("the other class failed") !=
                                              std::string::npos))
        first = i;
    if (first >= 0) {
      g_last_error = msg[first];
      return rc[first];
    }
  }

  // Regulation 3: mean and population std of N over the training normals,
  // in double precision and record order.
  if (prm.reg3_enabled) {
    DevBuf<unsigned long long> d_n;
    IG_CUDA(d_n.alloc(size_t(nc[0]), s), "ig_fit");
    IG_CUDA(cudaMemsetAsync(d_n.p, 0, sizeof(unsigned long long) * nc[0], s), "ig_fit");
    bool done_idx = false;
    if (pruned && m->n_pat[0] && rec_idx[0].idx.usable) {
      igk::IndexedArgs a;
      a.mode = igk::MODE_SUM;
      a.index = &rec_idx[0].idx;
      a.keyed = m->words_kt[0];
      a.n_keyed = m->n_pat[0];
      a.keyed_stride = KT;
      a.keyed_score = m->score[0];
      a.out_u32 = nullptr;
      a.out_u64 = d_n.p;
      a.status = d_status.p;
      a.tests_out = h_tests + 4;
      a.prof_stage = S_EVIDENCE_IDX;
      a.max_q = m->index_max_q;
      a.flip_factor = m->index_flip;
      a.tc = m->subset_kernel == 4 ? 1 : 0;
      IG_CUDA(igk::indexed_subset(a, s), "ig_fit: Regulation 3 evidence");
      done_idx = true;
    }
    if (done_idx) {
    } else if (tc && m->n_pat[0] && rec_img[0].p && m->pat_img[0]) {
      ProfScope ps(S_EVIDENCE_TC, s);
      igk::TcArgs a{igk::MODE_SUM, KT,           rec_img[0].p, nc[0],   nullptr, m->pat_img[0],
                    0,             m->n_pat[0],  m->score[0],  nullptr, d_n.p,   d_status.p};
      IG_CUDA(igk::launch_subset_tc(a, s), "ig_fit: Regulation 3 evidence");
    } else {
      ProfScope ps(S_EVIDENCE, s);
      igk::SubsetArgs a{igk::MODE_SUM, KT, X[0].p, nc[0], KT, m->words_kt[0], m->score[0],
                        m->n_pat[0], nullptr, d_n.p, d_status.p};
      IG_CUDA(igk::launch_subset(a, s), "ig_fit: Regulation 3 evidence");
    }
    std::vector<unsigned long long> hn(static_cast<size_t>(nc[0]));
    IG_CUDA(cudaMemcpyAsync(hn.data(), d_n.p, sizeof(unsigned long long) * nc[0],
                            cudaMemcpyDeviceToHost, s),
            "ig_fit");
    IG_CHECK(read_status(d_status.p, s, "ig_fit: Regulation 3"));
    double sum = 0.0;
    for (int64_t i = 0; i < nc[0]; ++i) sum += double(int64_t(hn[i]));
    const double mean = sum / double(nc[0]);
    double ss = 0.0;
    for (int64_t i = 0; i < nc[0]; ++i) {
      const double d = double(int64_t(hn[i])) - mean;
      ss += d * d;
    }
    m->reg3 = 1;
    m->mu = mean;
    m->sigma = std::sqrt(ss / double(nc[0]));
    m->r = prm.r;
    const double scaled = prm.r * m->sigma;
    m->thr = m->mu - scaled;
  }
  IG_CHECK(read_status(d_status.p, s, "ig_fit"));
  for (int c = 0; c < 2; ++c) {
    m->score_max[c] = h_smax[c];
    if (sup_idx_ran[c]) {
      m->sup_tests[c] = h_tests[2 + c];
      igk::prof_add_work(S_SUPPORT_IDX, h_tests[2 + c]);
    }
  }
  guard.m = nullptr;
  *out = m;
  return IG_OK;
}

// Pinned host scratch of at least `bytes`, one block per host thread.
void* pinned_scratch(size_t bytes) {
  static thread_local void* p = nullptr;
  static thread_local size_t cap = 0;
  if (bytes > cap) {
    if (p) cudaFreeHost(p);
    p = nullptr;
    cap = 0;
    if (cudaMallocHost(&p, bytes) != cudaSuccess) return nullptr;
    cap = bytes;
  }
  return p;
}

// The candidate stage (Eq. 1) of every problem of a batch at once: the
// class split of every problem, one read-back of all class sizes, then the
// pair tiles of every class of every problem, all word counts, in one launch
// (a persistent grid drawing tiles from a device-side queue), one read-back
// of all tables' counters, and replays of the tables that ran out of room
// (grown and rehashed one by one, replayed together).  A problem that this
// stage cannot prepare (bad arguments, bad labels, an empty class) is left
// unprepared: its own fit then runs every step and reports the error.
int batched_candidates(const ig_problem* problems, int32_t np, const ig_params* params,
                       std::vector<FitPrep>& prep, cudaStream_t s) {
  struct Inputs {
    InputView<uint64_t> rows;
    InputView<uint8_t> lab;
  };
  std::unique_ptr<Inputs[]> in(new Inputs[np]);
  std::vector<char> ok(np, 0);
  DevBuf<unsigned long long> d_counts;
  DevBuf<int> d_status;
  IG_CUDA(d_counts.alloc(size_t(2) * np, s), "ig_fit_batched");
  // Status words: one per problem (its split), and one for the pair stage.
  IG_CUDA(d_status.alloc(size_t(np) + 1, s), "ig_fit_batched");
  IG_CUDA(cudaMemsetAsync(d_counts.p, 0, sizeof(unsigned long long) * 2 * np, s), "ig_fit_batched");
  IG_CUDA(cudaMemsetAsync(d_status.p, 0, sizeof(int) * (np + 1), s), "ig_fit_batched");
  int* const pair_status = d_status.p + np;
  for (int32_t i = 0; i < np; ++i) {
    const ig_problem& pr = problems[i];
    const ig_params* prm = pr.params ? pr.params : params;
    if (!pr.rows || !pr.labels || pr.n < 2 || pr.K < 1 || pr.K > IG_MAX_WORDS ||
        pr.n > int64_t(0x7fffffff) || (prm && prm->subset_kernel < 0))
      continue;
    const int KT = igk::padded_words(pr.K);
    if (in[i].rows.bind(pr.rows, size_t(pr.n) * pr.K, s, "ig_fit_batched: rows") != IG_OK ||
        in[i].lab.bind(pr.labels, size_t(pr.n), s, "ig_fit_batched: labels") != IG_OK)
      continue;
    for (int c = 0; c < 2; ++c)
      IG_CUDA(prep[i].X[c].alloc(size_t(igk::pad_rows(pr.n) + igk::kRowPad) * KT, s),
              "ig_fit_batched: rows");
    {
      ProfScope ps(S_SPLIT, s);
      IG_CUDA(igk::launch_split(in[i].rows.d, in[i].lab.d, pr.n, pr.K, KT, prep[i].X[0].p,
                                prep[i].X[1].p, d_counts.p + 2 * i, d_status.p + i, s),
              "ig_fit_batched: split");
    }
    ok[i] = 1;
  }
  const size_t n_ctr = size_t(2) * np;
  char* h = static_cast<char*>(pinned_scratch(n_ctr * sizeof(TableCounters) +
                                              n_ctr * sizeof(unsigned long long) +
                                              (size_t(np) + 1) * sizeof(int)));
  if (!h) return fail(IG_E_CUDA, "ig_fit_batched: pinned host allocation failed");
  TableCounters* h_ctr = reinterpret_cast<TableCounters*>(h);
  unsigned long long* h_counts = reinterpret_cast<unsigned long long*>(h_ctr + n_ctr);
  int* h_status = reinterpret_cast<int*>(h_counts + n_ctr);
  IG_CUDA(cudaMemcpyAsync(h_counts, d_counts.p, sizeof(unsigned long long) * n_ctr,
                          cudaMemcpyDeviceToHost, s),
          "ig_fit_batched");
  IG_CUDA(cudaMemcpyAsync(h_status, d_status.p, sizeof(int) * np, cudaMemcpyDeviceToHost, s),
          "ig_fit_batched");
  IG_CUDA(cudaStreamSynchronize(s), "ig_fit_batched");

  // Tables of the problems whose split succeeded with both classes present.
  struct Job {
    int32_t i;
    int c;
    int KT;
  };
  std::vector<Job> jobs;
  for (int32_t i = 0; i < np; ++i) {
    if (!ok[i]) continue;
    const int64_t nc[2] = {int64_t(h_counts[2 * i]), int64_t(h_counts[2 * i + 1])};
    if (h_status[i] != 0 || nc[0] == 0 || nc[1] == 0 ||
        std::max(nc[0], nc[1]) > int64_t(65535) * igk::kPairTile) {
      ok[i] = 0;
      continue;
    }
    for (int c = 0; c < 2; ++c) {
      prep[i].nc[c] = nc[c];
      jobs.push_back(Job{i, c, igk::padded_words(problems[i].K)});
    }
  }
  // The pair stage runs over each class's distinct records: their counts
  // are read back together (one synchronization for the batch).
  std::vector<int64_t> nu(jobs.size(), 0);
  if (!jobs.empty()) {
    DevBuf<unsigned long long> d_nu;
    IG_CUDA(d_nu.alloc(jobs.size(), s), "ig_fit_batched");
    for (size_t k = 0; k < jobs.size(); ++k) {
      FitPrep& pp = prep[jobs[k].i];
      IG_CHECK(unique_rows(pp.X[jobs[k].c].p, pp.nc[jobs[k].c], jobs[k].KT, pp.Xu[jobs[k].c],
                           d_nu.p + k, s));
    }
    unsigned long long* h_nu = reinterpret_cast<unsigned long long*>(h_ctr);
    IG_CUDA(cudaMemcpyAsync(h_nu, d_nu.p, sizeof(unsigned long long) * jobs.size(),
                            cudaMemcpyDeviceToHost, s),
            "ig_fit_batched");
    IG_CUDA(cudaStreamSynchronize(s), "ig_fit_batched");
    for (size_t k = 0; k < jobs.size(); ++k) nu[k] = int64_t(h_nu[k]);
  }
  // Table sizes.  A table with room for every pair (a key per pair at half
  // load) never has to grow, so the stage needs one launch; that is the
  // size while all tables together stay within an eighth of the device's
  // memory, and the usual guess (which may grow) otherwise.
  {
    size_t free_b = 0, total_b = 0;
    IG_CUDA(cudaMemGetInfo(&free_b, &total_b), "ig_fit_batched");
    uint64_t room = 0;
    std::vector<uint64_t> cap(jobs.size());
    for (size_t k = 0; k < jobs.size(); ++k) {
      const int64_t n = nu[k];
      const uint64_t pairs = uint64_t(n) * uint64_t(n + 1) / 2;
      uint64_t c = 1u << 12;
      while (c < 2 * pairs) c <<= 1;
      cap[k] = c;
      room += c * sizeof(uint64_t);
    }
    // IG_TEST_SMALL_TABLES=1 (a test hook) takes the usual guess always, so
    // that tables grow and their bands are replayed.
    const char* small = std::getenv("IG_TEST_SMALL_TABLES");
    const bool roomy = room <= total_b / 8 && !(small && small[0] == '1');
    for (size_t k = 0; k < jobs.size(); ++k)
      IG_CUDA(alloc_table(prep[jobs[k].i].tab[jobs[k].c], roomy ? cap[k] : initial_cap(nu[k]), s),
              "ig_fit_batched: hash table");
  }
  DevBuf<TableCounters> d_ctr;
  IG_CUDA(d_ctr.alloc(std::max<size_t>(1, jobs.size()), s), "ig_fit_batched");
  for (size_t k = 0; k < jobs.size(); ++k) h_ctr[k] = TableCounters{0ull, kNoBand, 0};
  IG_CUDA(cudaMemcpyAsync(d_ctr.p, h_ctr, sizeof(TableCounters) * jobs.size(),
                          cudaMemcpyHostToDevice, s),
          "ig_fit_batched");
  std::vector<int64_t> band_lo(jobs.size(), 0);
  std::vector<size_t> todo(jobs.size());
  for (size_t k = 0; k < jobs.size(); ++k) todo[k] = k;
  DevBuf<igk::PairJob> d_jobs;
  DevBuf<int64_t> d_off;
  DevBuf<unsigned long long> d_next;
  const int warps = igk::pair_multi_grid_warps();
  while (!todo.empty()) {
    // One launch over every table still to do.
    std::vector<igk::PairJob> pj;
    std::vector<int64_t> off{0};
    for (size_t k : todo) {
      const Job& jb = jobs[k];
      FitPrep& pp = prep[jb.i];
      igk::PairJob j;
      j.X = pp.Xu[jb.c].p;
      j.n = nu[k];
      j.band_lo = band_lo[k];
      j.KT = jb.KT;
      j.t = make_table(pp.tab[jb.c].slots.p, pp.tab[jb.c].cap, d_ctr.p + k, kMaxProbe);
      // Warps add their keys to the count often enough that it lags the
      // table by at most about a quarter of the limit over the whole grid.
      j.t.flush = uint32_t(
          std::max<int64_t>(1, std::min<int64_t>(256, int64_t(j.t.limit) / (4 * int64_t(warps)))));
      const int64_t nt = igk::ceil_div(j.n, igk::kPairTile), rows = nt - j.band_lo;
      pj.push_back(j);
      off.push_back(off.back() + rows * (rows + 1) / 2);
    }
    // Buffers of the previous launch are freed in stream order first.
    IG_CUDA(d_jobs.alloc(pj.size(), s), "ig_fit_batched");
    IG_CUDA(d_off.alloc(off.size(), s), "ig_fit_batched");
    IG_CUDA(d_next.alloc(1, s), "ig_fit_batched");
    IG_CUDA(cudaMemcpyAsync(d_jobs.p, pj.data(), sizeof(igk::PairJob) * pj.size(),
                            cudaMemcpyHostToDevice, s),
            "ig_fit_batched");
    IG_CUDA(cudaMemcpyAsync(d_off.p, off.data(), sizeof(int64_t) * off.size(),
                            cudaMemcpyHostToDevice, s),
            "ig_fit_batched");
    IG_CUDA(cudaMemsetAsync(d_next.p, 0, sizeof(unsigned long long), s), "ig_fit_batched");
    {
      ProfScope ps(S_PAIR, s);
      IG_CUDA(igk::launch_pair_insert_multi(d_jobs.p, int(pj.size()), d_off.p, d_next.p,
                                            pair_status, s),
              "ig_fit_batched: pair intersection");
    }
    IG_CUDA(cudaMemcpyAsync(h_ctr, d_ctr.p, sizeof(TableCounters) * jobs.size(),
                            cudaMemcpyDeviceToHost, s),
            "ig_fit_batched");
    IG_CUDA(cudaStreamSynchronize(s), "ig_fit_batched");
    std::vector<size_t> again;
    for (size_t k : todo) {
      if (h_ctr[k].failed_band == kNoBand) continue;
      const Job& jb = jobs[k];
      FitPrep& pp = prep[jb.i];
      band_lo[k] = h_ctr[k].failed_band;
      IG_CHECK(grow_table(pp.Xu[jb.c].p, nu[k], jb.KT, pp.tab[jb.c], d_ctr.p + k, band_lo[k],
                          h_ctr[k].count, pair_status, s));
      IG_CUDA(cudaMemsetAsync(&d_ctr.p[k].failed_band, 0x7f, sizeof(int), s), "ig_fit_batched");
      again.push_back(k);
    }
    todo.swap(again);
  }
  IG_CUDA(cudaMemcpyAsync(h_status, d_status.p, sizeof(int) * (np + 1), cudaMemcpyDeviceToHost,
                          s),
          "ig_fit_batched");
  IG_CUDA(cudaStreamSynchronize(s), "ig_fit_batched");
  for (size_t k = 0; k < jobs.size(); ++k) prep[jobs[k].i].count[jobs[k].c] = int64_t(h_ctr[k].count);
  // A pair-stage status (which no table should raise) leaves every problem
  // to its own fit.
  for (int32_t i = 0; i < np; ++i) prep[i].ready = ok[i] && h_status[i] == 0 && h_status[np] == 0;
  return IG_OK;
}

// Runs fn(k, stream) for k = order[0], order[1], ... on `lanes` streams,
// each with a host thread pulling the next item when it finishes one.  The
// streams start after what `s` holds and `s` waits for all of them.  The
// first failure (by the order in which lanes saw them) is kept, its message
// prefixed with `what` and the item's number.
template <class Fn>
int run_lanes(const std::vector<int32_t>& order, int lanes, cudaStream_t s, const char* what,
              Fn fn) {
  const int32_t n = int32_t(order.size());
  if (n == 0) return IG_OK;
  if (lanes <= 0) lanes = 8;
  if (lanes > n) lanes = n;
  int dev = 0;
  IG_CUDA(cudaGetDevice(&dev), what);
  cudaEvent_t ready = nullptr;
  std::vector<cudaStream_t> ls(lanes, nullptr);
  std::vector<cudaEvent_t> done(lanes, nullptr);
  // Destroys what was created (a stream is released once its work is done).
  auto release = [&] {
    for (int l = 0; l < lanes; ++l) {
      if (done[l]) cudaEventDestroy(done[l]);
      if (ls[l]) cudaStreamDestroy(ls[l]);
    }
    if (ready) cudaEventDestroy(ready);
  };
  cudaError_t e = cudaEventCreateWithFlags(&ready, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventRecord(ready, s);
  for (int l = 0; l < lanes && e == cudaSuccess; ++l) {
    e = cudaStreamCreateWithFlags(&ls[l], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&done[l], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(ls[l], ready, 0);
  }
  if (e != cudaSuccess) {
    release();
    return fail_cuda(e, what);
  }
  std::atomic<int32_t> next{0};
  std::mutex err_mu;
  int first_rc = IG_OK;
  std::string first_msg;
  auto lane = [&](int l) {
    cudaSetDevice(dev);
    for (;;) {
      const int32_t k = next.fetch_add(1);
      if (k >= n) break;
      const int rc = igk::guarded(what, [&]() -> int { return fn(order[k], ls[l]); });
      if (rc != IG_OK) {
        std::lock_guard<std::mutex> lk(err_mu);
        if (first_rc == IG_OK) {
          first_rc = rc;
          try {
            first_msg = std::string(what) + " " + std::to_string(order[k]) + ": " + g_last_error;
          } catch (...) {
          }
        }
      }
    }
    cudaEventRecord(done[l], ls[l]);
  };
  std::vector<Worker*> ws;
  for (int l = 1; l < lanes; ++l) {
    Worker* w = acquire_worker();
    w->run([&, l] { lane(l); });
    ws.push_back(w);
  }
  lane(0);
  for (Worker* w : ws) {
    w->wait();
    release_worker(w);
  }
  for (int l = 0; l < lanes; ++l) cudaStreamWaitEvent(s, done[l], 0);
  release();
  if (first_rc != IG_OK) g_last_error = first_msg;
  return first_rc;
}

}  // namespace

extern "C" {

int ig_fit(const uint64_t* rows, const uint8_t* labels, int64_t n, int32_t K,
           const ig_params* params, ig_model** out, ig_stream_t stream) {
  return igk::guarded("ig_fit", [&]() -> int {
    igk::DeviceRestore restore_device;  // the caller's device, put back on return
    return fit_impl(rows, labels, n, K, params, out, reinterpret_cast<cudaStream_t>(stream),
                    nullptr);
  });
}

int ig_fit_batched(const ig_problem* problems, int32_t n_problems, const ig_params* params,
                   int32_t lanes, ig_model** out, ig_stream_t stream) {
  return igk::guarded("ig_fit_batched", [&]() -> int {
    igk::DeviceRestore restore_device;  // the caller's device, put back on return
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (n_problems < 0 || (n_problems > 0 && (!problems || !out)))
      return fail(IG_E_INVAL, "ig_fit_batched: bad arguments");
    for (int32_t i = 0; i < n_problems; ++i) out[i] = nullptr;
    if (n_problems == 0) return IG_OK;
    // Largest problems first (pairs grow as n^2), each lane pulling the next.
    std::vector<int32_t> order(n_problems);
    for (int32_t i = 0; i < n_problems; ++i) order[i] = i;
    std::sort(order.begin(), order.end(), [&](int32_t a, int32_t b) {
      return problems[a].n > problems[b].n || (problems[a].n == problems[b].n && a < b);
    });
    std::vector<FitPrep> prep(n_problems);
    IG_CHECK(batched_candidates(problems, n_problems, params, prep, s));
    const int rc = run_lanes(order, lanes, s, "problem", [&](int32_t k, cudaStream_t ls) {
      const ig_problem& pr = problems[k];
      return fit_impl(pr.rows, pr.labels, pr.n, pr.K, pr.params ? pr.params : params, &out[k], ls,
                      prep[k].ready ? &prep[k] : nullptr);
    });
    if (rc != IG_OK) {
      for (int32_t i = 0; i < n_problems; ++i) {
        ig_model_free(out[i]);
        out[i] = nullptr;
      }
    }
    return rc;
  });
}

int ig_score_batched(const ig_score_job* jobs, int32_t n_jobs, int32_t lanes,
                     ig_stream_t stream) {
  return igk::guarded("ig_score_batched", [&]() -> int {
    igk::DeviceRestore restore_device;  // the caller's device, put back on return
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (n_jobs < 0 || (n_jobs > 0 && !jobs)) return fail(IG_E_INVAL, "ig_score_batched: bad arguments");
    // Largest batches first, each lane pulling the next.
    std::vector<int32_t> order(n_jobs);
    for (int32_t i = 0; i < n_jobs; ++i) order[i] = i;
    std::sort(order.begin(), order.end(), [&](int32_t a, int32_t b) {
      return jobs[a].m > jobs[b].m || (jobs[a].m == jobs[b].m && a < b);
    });
    return run_lanes(order, lanes, s, "job", [&](int32_t k, cudaStream_t ls) {
      const ig_score_job& j = jobs[k];
      return ig_score(j.model, j.rows, j.m, j.A_out, j.N_out, j.label_out,
                      reinterpret_cast<ig_stream_t>(ls));
    });
  });
}

int ig_model_from_patterns(int32_t K, const uint64_t* const* words, const uint32_t* const* support,
                           const int64_t* n_patterns, ig_model** out, ig_stream_t stream) {
  return igk::guarded("ig_model_from_patterns", [&]() -> int {
    igk::DeviceRestore restore_device;  // the caller's device, put back on return
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (!out || !words || !support || !n_patterns)
      return fail(IG_E_INVAL, "ig_model_from_patterns: NULL argument");
    *out = nullptr;
    if (K < 1 || K > IG_MAX_WORDS)
      return fail(IG_E_INVAL, "ig_model_from_patterns: K = %d out of range", K);
    const int KT = igk::padded_words(K);
    ig_model* m = new ig_model;
    struct ModelGuard {
      ig_model* m;
      ~ModelGuard() { model_release(m); }
    } guard{m};
    m->K = K;
    m->KT = KT;
    DevBuf<int> d_status;
    IG_CUDA(d_status.alloc(1, s), "ig_model_from_patterns");
    IG_CUDA(cudaMemsetAsync(d_status.p, 0, sizeof(int), s), "ig_model_from_patterns");
    for (int c = 0; c < 2; ++c) {
      const int64_t P = n_patterns[c];
      if (P < 0 || (P > 0 && (!words[c] || !support[c])))
        return fail(IG_E_INVAL, "ig_model_from_patterns: bad class %d arrays", c);
      if (P > int64_t(0xffffffffll)) return fail(IG_E_OVERFLOW, "ig_model_from_patterns: too many");
      m->n_pat[c] = P;
      const size_t npad = size_t(std::max<int64_t>(1, igk::pad_rows(P)));
      InputView<uint64_t> in_w;
      InputView<uint32_t> in_f;
      IG_CHECK(in_w.bind(words[c], size_t(P) * K, s, "ig_model_from_patterns: words"));
      IG_CHECK(in_f.bind(support[c], size_t(P), s, "ig_model_from_patterns: supports"));
      DevBuf<uint64_t> raw, work;
      IG_CUDA(raw.alloc(npad * KT, s), "ig_model_from_patterns");
      IG_CUDA(work.alloc(npad * KT, s), "ig_model_from_patterns");
      IG_CUDA(cudaMemsetAsync(raw.p, 0, npad * KT * 8, s), "ig_model_from_patterns");
      if (P)
        IG_CUDA(cudaMemcpy2DAsync(raw.p, KT * 8, in_w.d, K * 8, K * 8, P, cudaMemcpyDeviceToDevice, s),
                "ig_model_from_patterns");
      IG_CUDA(cudaMallocAsync(reinterpret_cast<void**>(&m->words_kt[c]), npad * KT * 8, s),
              "ig_model_from_patterns");
      IG_CUDA(cudaMemsetAsync(m->words_kt[c], 0, npad * KT * 8, s), "ig_model_from_patterns");
      IG_CUDA(cudaMemcpyAsync(work.p, raw.p, npad * KT * 8, cudaMemcpyDeviceToDevice, s),
              "ig_model_from_patterns");
      {
        ProfScope ps(S_SORT, s);
        IG_CUDA(igk::canonical_sort(work.p, P, KT, m->words_kt[c], work.p, s),
                "ig_model_from_patterns: sort");
      }
      IG_CUDA(igk::launch_check_strict(m->words_kt[c], P, KT, d_status.p, s),
              "ig_model_from_patterns");
      IG_CUDA(cudaMallocAsync(reinterpret_cast<void**>(&m->support[c]),
                              sizeof(uint32_t) * std::max<int64_t>(1, P), s),
              "ig_model_from_patterns");
      IG_CUDA(igk::launch_place_payload(m->words_kt[c], P, KT, raw.p, in_f.d, m->support[c],
                                        d_status.p, s),
              "ig_model_from_patterns");
      IG_CUDA(cudaMallocAsync(reinterpret_cast<void**>(&m->score[c]), sizeof(uint64_t) * npad, s),
              "ig_model_from_patterns");
      IG_CUDA(cudaMemsetAsync(m->score[c], 0, sizeof(uint64_t) * npad, s), "ig_model_from_patterns");
      DevBuf<unsigned long long> d_smax;
      IG_CUDA(d_smax.alloc(1, s), "ig_model_from_patterns");
      IG_CUDA(cudaMemsetAsync(d_smax.p, 0, sizeof(unsigned long long), s), "ig_model_from_patterns");
      IG_CUDA(igk::launch_pattern_score(m->words_kt[c], P, KT, m->support[c], m->score[c], s,
                                        d_smax.p),
              "ig_model_from_patterns: score");
      unsigned long long smax = 0;
      IG_CUDA(cudaMemcpyAsync(&smax, d_smax.p, sizeof(smax), cudaMemcpyDeviceToHost, s),
              "ig_model_from_patterns");
      if (K == KT) {
        m->words[c] = m->words_kt[c];
      } else {
        IG_CUDA(cudaMallocAsync(reinterpret_cast<void**>(&m->words[c]),
                                sizeof(uint64_t) * std::max<int64_t>(1, P) * K, s),
                "ig_model_from_patterns");
        if (P)
          IG_CUDA(cudaMemcpy2DAsync(m->words[c], K * 8, m->words_kt[c], KT * 8, K * 8, P,
                                    cudaMemcpyDeviceToDevice, s),
                  "ig_model_from_patterns");
      }
      IG_CHECK(read_status(d_status.p, s, "ig_model_from_patterns"));
      m->score_max[c] = smax;
    }
    m->subset_kernel = KT >= 2 ? 3 : 1;
    if (KT >= 2) {
      DevBuf<uint32_t> d_f;
      IG_CUDA(d_f.alloc(64 * K, s), "ig_model_from_patterns");
      IG_CUDA(pattern_item_freq(m, d_f.p, s), "ig_model_from_patterns");
      IG_CUDA(build_pattern_indexes(m, d_f.p, s), "ig_model_from_patterns: pattern index");
    }
    guard.m = nullptr;
    *out = m;
    return IG_OK;
  });
}

int ig_model_info(const ig_model* m, ig_model_info_t* info) {
  if (!m || !info) return fail(IG_E_INVAL, "ig_model_info: NULL argument");
  info->K = m->K;
  info->reg3_enabled = m->reg3;
  for (int c = 0; c < 2; ++c) {
    info->n_train[c] = m->n_train[c];
    info->n_candidates[c] = m->n_cand[c];
    info->n_patterns[c] = m->n_pat[c];
    info->n_pairs[c] = m->n_pairs[c];
  }
  info->reg3_mu = m->mu;
  info->reg3_sigma = m->sigma;
  info->reg3_r = m->r;
  info->reg3_threshold = m->thr;
  info->coherence_tests[0] = m->coh_tests[0];
  info->coherence_tests[1] = m->coh_tests[1];
  info->coherence_tests_tc[0] = m->coh_tests_tc[0];
  info->coherence_tests_tc[1] = m->coh_tests_tc[1];
  info->coherence_tests_idx[0] = m->coh_tests_pruned[0];
  info->coherence_tests_idx[1] = m->coh_tests_pruned[1];
  info->support_tests[0] = m->sup_tests[0];
  info->support_tests[1] = m->sup_tests[1];
  info->subset_kernel = m->subset_kernel;
  info->reserved = 0;
  return IG_OK;
}

int ig_model_patterns(const ig_model* m, int32_t cls, const uint64_t** words,
                      const uint32_t** support, const uint64_t** score) {
  if (!m || (cls != 0 && cls != 1)) return fail(IG_E_INVAL, "ig_model_patterns: bad arguments");
  if (words) *words = m->words[cls];
  if (support) *support = m->support[cls];
  if (score) *score = m->score[cls];
  return IG_OK;
}

int ig_model_copy_patterns(const ig_model* m, int32_t cls, uint64_t* words_out,
                           uint32_t* support_out, uint64_t* score_out,
                           ig_stream_t stream) {
  return igk::guarded("ig_model_copy_patterns", [&]() -> int {
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (!m || (cls != 0 && cls != 1)) return fail(IG_E_INVAL, "ig_model_copy_patterns: bad arguments");
    const int64_t P = m->n_pat[cls];
    if (P == 0) return IG_OK;
    if (words_out)
      IG_CUDA(cudaMemcpyAsync(words_out, m->words[cls], sizeof(uint64_t) * P * m->K,
                              cudaMemcpyDefault, s), "ig_model_copy_patterns");
    if (support_out)
      IG_CUDA(cudaMemcpyAsync(support_out, m->support[cls], sizeof(uint32_t) * P,
                              cudaMemcpyDefault, s), "ig_model_copy_patterns");
    if (score_out)
      IG_CUDA(cudaMemcpyAsync(score_out, m->score[cls], sizeof(uint64_t) * P, cudaMemcpyDefault, s),
              "ig_model_copy_patterns");
    IG_CUDA(cudaStreamSynchronize(s), "ig_model_copy_patterns");
    return IG_OK;
  });
}

int ig_score(const ig_model* m, const uint64_t* rows, int64_t n_rows, int64_t* A_out,
             int64_t* N_out, uint8_t* label_out, ig_stream_t stream) {
  return igk::guarded("ig_score", [&]() -> int {
    igk::DeviceRestore restore_device;  // the caller's device, put back on return
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (!m || n_rows < 0 || (n_rows > 0 && !rows)) return fail(IG_E_INVAL, "ig_score: bad arguments");
    // Pinned words for the tensor-core evidence's executed tests (one pair
    // per host thread), copied when the stream gets there.
    static thread_local int64_t* h_tests = nullptr;
    int tc_tests = 0;
    if (n_rows == 0) return IG_OK;
    InputView<uint64_t> in;
    IG_CHECK(in.bind(rows, size_t(n_rows) * m->K, s, "ig_score: rows"));
    OutputView<unsigned long long> A, N;
    OutputView<uint8_t> lab;
    IG_CHECK(A.bind(reinterpret_cast<unsigned long long*>(A_out), size_t(n_rows), s, "ig_score"));
    IG_CHECK(N.bind(reinterpret_cast<unsigned long long*>(N_out), size_t(n_rows), s, "ig_score"));
    if (label_out) IG_CHECK(lab.bind(label_out, size_t(n_rows), s, "ig_score"));
    DevBuf<int> d_status;
    IG_CUDA(d_status.alloc(1, s), "ig_score");
    IG_CUDA(cudaMemsetAsync(d_status.p, 0, sizeof(int), s), "ig_score");
    IG_CUDA(cudaMemsetAsync(A.d, 0, sizeof(unsigned long long) * n_rows, s), "ig_score");
    IG_CUDA(cudaMemsetAsync(N.d, 0, sizeof(unsigned long long) * n_rows, s), "ig_score");
    DevBuf<uint8_t> test_img;
    // The item index pays for its build (and its host round trips) only on
    // batches of some size; smaller batches stream the patterns densely.
    const bool pruned = m->subset_kernel >= 3 && n_rows >= kIndexMinRows;
    bool tc = m->subset_kernel >= 2 && igk::tc_supported(m->KT) && m->pat_img[0] && m->pat_img[1];
    bool done[2] = {false, false};
    IndexHolder test_idx;
    test_idx.s = s;
    DevBuf<uint64_t> sorted_rows;
    DevBuf<uint32_t> perm;
    if (pruned && m->subset_kernel == 4) {
      // The tensor-core evidence kernel reads records in canonical order: the
      // neighbouring rows of an item group then hold similar itemsets, so the
      // patterns inside them fall into fewer 32 x 32 accumulator chunks, and
      // its epilogue skips every chunk without one.  The index files each copy
      // under the caller's row number (perm), so results land in place.
      const int KT = m->KT;
      const uint64_t* keys = in.d;
      DevBuf<uint64_t> padded;
      if (m->K != KT) {
        IG_CUDA(padded.alloc(size_t(n_rows) * KT, s), "ig_score");
        IG_CUDA(cudaMemsetAsync(padded.p, 0, sizeof(uint64_t) * n_rows * KT, s), "ig_score");
        IG_CUDA(cudaMemcpy2DAsync(padded.p, KT * 8, in.d, m->K * 8, m->K * 8, n_rows,
                                  cudaMemcpyDeviceToDevice, s),
                "ig_score");
        keys = padded.p;
      }
      IG_CUDA(sorted_rows.alloc(size_t(n_rows) * KT, s), "ig_score");
      IG_CUDA(perm.alloc(size_t(n_rows), s), "ig_score");
      {
        ProfScope ps(igk::kStageIndexBuild, s);
        IG_CUDA(igk::canonical_sort(keys, n_rows, KT, sorted_rows.p, nullptr, s, perm.p),
                "ig_score: record order");
      }
      IG_CUDA(igk::build_record_index(sorted_rows.p, n_rows, KT, m->K, KT, 0.25, &test_idx.idx, s,
                                      perm.p),
              "ig_score: record index");
    } else if (pruned) {
      IG_CUDA(igk::build_record_index(in.d, n_rows, m->K, m->K, m->KT, 0.25, &test_idx.idx, s),
              "ig_score: record index");
    }
    if (pruned && test_idx.idx.usable && m->subset_kernel == 4 && igk::tc_supported(m->KT)) {
      // Tensor-core form: both classes' patterns against the batch's records
      // in one launch of the fused kernel (one schedule, one tail).  Small
      // batches reuse the model's pattern index; larger ones re-key the
      // patterns by the batch's own item counts.
      igk::KeyedIndex own[2];
      const igk::KeyedIndex* kx[2];
      unsigned long long* outs[2];
      uint64_t smax[2];
      int n = 0;
      cudaError_t e = cudaSuccess;
      if (!h_tests) e = cudaMallocHost(&h_tests, 2 * sizeof(int64_t));
      for (int c = 1; c >= 0 && e == cudaSuccess; --c) {
        done[c] = true;
        if (m->n_pat[c] == 0) continue;
        if (m->pidx[c] && n_rows * 8 < m->n_pat[c]) {
          kx[n] = m->pidx[c];
        } else {
          // Work items are built on the device: no host offsets, no read-back.
          e = igk::build_keyed_index(m->words_kt[c], m->n_pat[c], m->KT, m->K, m->KT,
                                     test_idx.idx.freq, m->score[c], &own[n], s, nullptr, false);
          kx[n] = &own[n];
        }
        outs[n] = c == 1 ? A.d : N.d;
        smax[n] = m->score_max[c];
        ++n;
      }
      if (e == cudaSuccess && n > 0) {
        h_tests[0] = h_tests[1] = 0;
        e = igk::indexed_subset_tc_classes(igk::MODE_SUM, test_idx.idx, kx, n, nullptr, outs,
                                           d_status.p, h_tests, S_EVIDENCE_IDX, smax, s);
        tc_tests = n;  // counted after the last read-back below
      }
      for (int i = 0; i < 2; ++i) igk::release_keyed_index(&own[i], s);
      IG_CUDA(e, "ig_score: evidence");
    } else if (pruned && test_idx.idx.usable) {
      // A (class 1) on the caller's stream and N (class 0) on this thread's
      // auxiliary stream, concurrently: both only read the indexes.
      AuxStream& aux = aux_stream();
      IG_CUDA(aux.error, "ig_score: auxiliary stream");
      IG_CUDA(cudaEventRecord(aux.ready, s), "ig_score");
      IG_CUDA(cudaStreamWaitEvent(aux.s, aux.ready, 0), "ig_score");
      for (int c = 1; c >= 0; --c) {
        if (m->n_pat[c] == 0) {
          done[c] = true;
          continue;
        }
        const cudaStream_t sc = c == 1 ? s : aux.s;
        int64_t t = 0;
        // Small batches reuse the model's pattern index; larger ones re-key
        // the patterns by the batch's own item counts (fewer tests, and
        // patterns holding an item absent from the batch drop out at once).
        if (m->pidx[c] && n_rows * 8 < m->n_pat[c]) {
          IG_CUDA(igk::indexed_subset_prebuilt(igk::MODE_SUM, test_idx.idx, *m->pidx[c], nullptr,
                                               c == 1 ? A.d : N.d, d_status.p, &t, S_EVIDENCE_IDX,
                                               m->index_max_q, m->index_flip,
                                               m->subset_kernel == 4 ? 1 : 0, sc, m->score_max[c]),
                  "ig_score: evidence");
          done[c] = true;
          igk::prof_add_work(S_EVIDENCE_IDX, t);
          continue;
        }
        igk::IndexedArgs a;
        a.mode = igk::MODE_SUM;
        a.index = &test_idx.idx;
        a.keyed = m->words_kt[c];
        a.n_keyed = m->n_pat[c];
        a.keyed_stride = m->KT;
        a.keyed_score = m->score[c];
        a.out_u32 = nullptr;
        a.out_u64 = c == 1 ? A.d : N.d;
        a.status = d_status.p;
        a.tests_out = &t;
        a.prof_stage = S_EVIDENCE_IDX;
        a.score_max = m->score_max[c];
        a.max_q = m->index_max_q;
        a.flip_factor = m->index_flip;
        a.tc = m->subset_kernel == 4 ? 1 : 0;
        IG_CUDA(igk::indexed_subset(a, sc), "ig_score: evidence");
        done[c] = true;
        igk::prof_add_work(S_EVIDENCE_IDX, t);
      }
      IG_CUDA(cudaEventRecord(aux.done, aux.s), "ig_score");
      IG_CUDA(cudaStreamWaitEvent(s, aux.done, 0), "ig_score");
    }
    if (done[0] && done[1]) tc = false;
    if (tc) {
      IG_CUDA(test_img.alloc(igk::tc_image_bytes(n_rows, m->KT, true), s), "ig_score: images");
      ProfScope pe(S_EXPAND, s);
      IG_CUDA(igk::launch_expand(in.d, n_rows, m->K, m->KT, true, true, test_img.p, s),
              "ig_score: expand");
    }
    for (int c = 1; c >= 0; --c) {  // A from P+, then N from P- (Eq. 4)
      if (done[c]) continue;
      igk::prof_add_work(tc && m->n_pat[c] ? S_EVIDENCE_TC : S_EVIDENCE, n_rows * m->n_pat[c]);
      ProfScope ps(tc && m->n_pat[c] ? S_EVIDENCE_TC : S_EVIDENCE, s);
      if (tc && m->n_pat[c]) {
        igk::TcArgs a{igk::MODE_SUM, m->KT,      test_img.p,  n_rows,  nullptr,
                      m->pat_img[c], 0,          m->n_pat[c], m->score[c], nullptr,
                      c == 1 ? A.d : N.d,        d_status.p};
        IG_CUDA(igk::launch_subset_tc(a, s), "ig_score: evidence");
      } else {
        igk::SubsetArgs a{igk::MODE_SUM, m->KT, in.d, n_rows, m->K, m->words_kt[c], m->score[c],
                          m->n_pat[c], nullptr, c == 1 ? A.d : N.d, d_status.p};
        IG_CUDA(igk::launch_subset(a, s), "ig_score: evidence");
      }
    }
    if (label_out) {
      ProfScope ps(S_LABELS, s);
      IG_CUDA(igk::launch_labels(A.d, N.d, n_rows, m->reg3, m->thr, lab.d, s), "ig_score: labels");
    }
    IG_CHECK(A.finish(s, "ig_score"));
    IG_CHECK(N.finish(s, "ig_score"));
    if (label_out) IG_CHECK(lab.finish(s, "ig_score"));
    const int rc = read_status(d_status.p, s, "ig_score");
    if (rc == IG_OK && tc_tests) igk::prof_add_work(S_EVIDENCE_IDX, h_tests[0] + h_tests[1]);
    return rc;
  });
}

// ---- persistence ------------------------------------------------------------
static const char kMagic[8] = {'I', 'G', 'G', 'B', '3', '0', '0', 0};
static const uint32_t kVersion = 1;

int ig_model_save(const ig_model* m, const char* path) {
  return igk::guarded("ig_model_save", [&]() -> int {
    if (!m || !path) return fail(IG_E_INVAL, "ig_model_save: NULL argument");
    FILE* f = fopen(path, "wb");
    if (!f) return fail(IG_E_IO, "ig_model_save: cannot open %s", path);
    bool ok = true;
    auto put = [&](const void* p, size_t n) { ok = ok && fwrite(p, 1, n, f) == n; };
    uint32_t hdr[4] = {kVersion, uint32_t(m->K), uint32_t(m->reg3), 0};
    double st[4] = {m->mu, m->sigma, m->r, m->thr};
    put(kMagic, 8);
    put(hdr, sizeof(hdr));
    put(st, sizeof(st));
    put(m->n_train, sizeof(m->n_train));
    put(m->n_cand, sizeof(m->n_cand));
    put(m->n_pairs, sizeof(m->n_pairs));
    put(m->n_pat, sizeof(m->n_pat));
    for (int c = 0; c < 2 && ok; ++c) {
      const int64_t P = m->n_pat[c];
      std::vector<uint64_t> w(size_t(P) * m->K);
      std::vector<uint32_t> sup(static_cast<size_t>(P));
      std::vector<uint64_t> sc(static_cast<size_t>(P));
      if (P) {
        if (cudaMemcpy(w.data(), m->words[c], w.size() * 8, cudaMemcpyDeviceToHost) != cudaSuccess ||
            cudaMemcpy(sup.data(), m->support[c], sup.size() * 4, cudaMemcpyDeviceToHost) != cudaSuccess ||
            cudaMemcpy(sc.data(), m->score[c], sc.size() * 8, cudaMemcpyDeviceToHost) != cudaSuccess) {
          fclose(f);
          return fail(IG_E_CUDA, "ig_model_save: copy from device failed");
        }
      }
      put(w.data(), w.size() * 8);
      put(sup.data(), sup.size() * 4);
      put(sc.data(), sc.size() * 8);
    }
    if (fclose(f) != 0) ok = false;
    return ok ? IG_OK : fail(IG_E_IO, "ig_model_save: write to %s failed", path);
  });
}

int ig_model_load(const char* path, ig_model** out) {
  return igk::guarded("ig_model_load", [&]() -> int {
    if (!path || !out) return fail(IG_E_INVAL, "ig_model_load: NULL argument");
    *out = nullptr;
    FILE* f = fopen(path, "rb");
    if (!f) return fail(IG_E_IO, "ig_model_load: cannot open %s", path);
    bool ok = true;
    auto get = [&](void* p, size_t n) { ok = ok && fread(p, 1, n, f) == n; };
    char magic[8];
    uint32_t hdr[4];
    double st[4];
    ig_model* m = new ig_model;
    get(magic, 8);
    get(hdr, sizeof(hdr));
    get(st, sizeof(st));
    get(m->n_train, sizeof(m->n_train));
    get(m->n_cand, sizeof(m->n_cand));
    get(m->n_pairs, sizeof(m->n_pairs));
    get(m->n_pat, sizeof(m->n_pat));
    if (!ok || memcmp(magic, kMagic, 8) != 0 || hdr[0] != kVersion || hdr[1] < 1 ||
        hdr[1] > IG_MAX_WORDS || m->n_pat[0] < 0 || m->n_pat[1] < 0) {
      fclose(f);
      model_release(m);
      return fail(IG_E_IO, "ig_model_load: %s is not an IG model file", path);
    }
    {
      // The pattern counts must account for the rest of the file exactly
      // (words, supports and scores of both classes) before anything is sized
      // by them: a damaged header must not drive a huge allocation.
      const off_t here = ftello(f);
      bool sized = here >= 0 && fseeko(f, 0, SEEK_END) == 0;
      const off_t end = sized ? ftello(f) : off_t(-1);
      const int64_t per = 8 * int64_t(hdr[1]) + 4 + 8;
      const int64_t left = int64_t(end) - int64_t(here);
      sized = sized && end >= here && m->n_pat[0] <= left / per && m->n_pat[1] <= left / per &&
              (m->n_pat[0] + m->n_pat[1]) * per == left && fseeko(f, here, SEEK_SET) == 0;
      if (!sized) {
        fclose(f);
        model_release(m);
        return fail(IG_E_IO, "ig_model_load: %s is truncated or its counts do not match its size",
                    path);
      }
    }
    m->K = int(hdr[1]);
    m->KT = igk::padded_words(m->K);
    m->reg3 = int(hdr[2]);
    m->mu = st[0];
    m->sigma = st[1];
    m->r = st[2];
    m->thr = st[3];
    for (int c = 0; c < 2 && ok; ++c) {
      const int64_t P = m->n_pat[c];
      std::vector<uint64_t> w(size_t(P) * m->K), wk(size_t(std::max<int64_t>(1, igk::pad_rows(P))) * m->KT, 0);
      std::vector<uint32_t> sup(static_cast<size_t>(P));
      std::vector<uint64_t> sc(size_t(std::max<int64_t>(1, igk::pad_rows(P))), 0);
      get(w.data(), w.size() * 8);
      get(sup.data(), sup.size() * 4);
      get(sc.data(), size_t(P) * 8);
      if (!ok) break;
      m->score_max[c] = P ? *std::max_element(sc.begin(), sc.begin() + P) : 0;
      for (int64_t i = 0; i < P; ++i)
        for (int k = 0; k < m->K; ++k) wk[size_t(i) * m->KT + k] = w[size_t(i) * m->K + k];
      bool cu = cudaMalloc(&m->words_kt[c], wk.size() * 8) == cudaSuccess &&
                cudaMemcpy(m->words_kt[c], wk.data(), wk.size() * 8, cudaMemcpyHostToDevice) == cudaSuccess &&
                cudaMalloc(&m->support[c], std::max<size_t>(1, sup.size()) * 4) == cudaSuccess &&
                (sup.empty() || cudaMemcpy(m->support[c], sup.data(), sup.size() * 4, cudaMemcpyHostToDevice) == cudaSuccess) &&
                cudaMalloc(&m->score[c], sc.size() * 8) == cudaSuccess &&
                cudaMemcpy(m->score[c], sc.data(), sc.size() * 8, cudaMemcpyHostToDevice) == cudaSuccess;
      if (cu && m->K == m->KT) {
        m->words[c] = m->words_kt[c];
      } else if (cu) {
        cu = cudaMalloc(&m->words[c], std::max<size_t>(1, w.size()) * 8) == cudaSuccess &&
             (w.empty() || cudaMemcpy(m->words[c], w.data(), w.size() * 8, cudaMemcpyHostToDevice) == cudaSuccess);
      }
      if (!cu) {
        fclose(f);
        model_release(m);
        return fail(IG_E_CUDA, "ig_model_load: device allocation or copy failed");
      }
    }
    fclose(f);
    if (!ok) {
      model_release(m);
      return fail(IG_E_IO, "ig_model_load: %s is truncated", path);
    }
    if (m->KT >= 2) {
      uint32_t* d_f = nullptr;
      cudaError_t e = cudaMalloc(&d_f, sizeof(uint32_t) * 64 * m->K);
      if (e == cudaSuccess) e = pattern_item_freq(m, d_f, nullptr);
      if (e == cudaSuccess) e = build_pattern_indexes(m, d_f, nullptr);
      if (d_f) cudaFree(d_f);
      if (e != cudaSuccess) {
        model_release(m);
        return fail_cuda(e, "ig_model_load: pattern index");
      }
      m->subset_kernel = 3;
    }
    *out = m;
    return IG_OK;
  });
}

void ig_model_free(ig_model* m) {
  if (!m) return;
  cudaDeviceSynchronize();
  model_release(m);
}

int ig_prof_enable(int32_t on) {
  std::lock_guard<std::mutex> lk(g_prof.mu);
  g_prof.on = on != 0;
  return IG_OK;
}

int ig_prof_select(uint32_t stage_mask) {
  std::lock_guard<std::mutex> lk(g_prof.mu);
  g_prof.mask = stage_mask;
  return IG_OK;
}

int ig_prof_reset(void) {
  std::lock_guard<std::mutex> lk(g_prof.mu);
  prof_drain_locked();
  for (int i = 0; i < IG_PROF_STAGES; ++i) {
    g_prof.ms[i] = 0;
    g_prof.launches[i] = 0;
    g_prof.work[i] = 0;
  }
  g_prof.spans.clear();
  if (!g_prof.ref && cudaEventCreate(&g_prof.ref) != cudaSuccess) {
    g_prof.ref = nullptr;
    cudaGetLastError();
  }
  if (g_prof.ref && cudaEventRecord(g_prof.ref, nullptr) != cudaSuccess) cudaGetLastError();
  return IG_OK;
}

int ig_prof_timeline(int32_t* stage, uint64_t* stream, double* t0_ms, double* t1_ms,
                     int64_t cap, int64_t* n_out) {
  return igk::guarded("ig_prof_timeline", [&]() -> int {
    std::lock_guard<std::mutex> lk(g_prof.mu);
    prof_drain_locked();
    const int64_t n = int64_t(g_prof.spans.size());
    if (n_out) *n_out = n;
    for (int64_t i = 0; i < n && i < cap; ++i) {
      const auto& sp = g_prof.spans[size_t(i)];
      if (stage) stage[i] = sp.stage;
      if (stream) stream[i] = uint64_t(reinterpret_cast<uintptr_t>(sp.s));
      if (t0_ms) t0_ms[i] = sp.t0;
      if (t1_ms) t1_ms[i] = sp.t1;
    }
    return IG_OK;
  });
}

int ig_prof_read_work(int64_t* tests) {
  std::lock_guard<std::mutex> lk(g_prof.mu);
  for (int i = 0; i < IG_PROF_STAGES; ++i)
    if (tests) tests[i] = g_prof.work[i];
  return IG_OK;
}

int ig_prof_read(double* ms, int64_t* launches) {
  std::lock_guard<std::mutex> lk(g_prof.mu);
  prof_drain_locked();
  for (int i = 0; i < IG_PROF_STAGES; ++i) {
    if (ms) ms[i] = g_prof.ms[i];
    if (launches) launches[i] = g_prof.launches[i];
  }
  return IG_OK;
}

int64_t ig_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

const char* ig_prof_stage_name(int32_t stage) {
  if (stage < 0 || stage >= IG_PROF_STAGES) return "";
  return kStageNames[stage];
}

}  // extern "C"
