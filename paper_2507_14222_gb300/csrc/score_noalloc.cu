// ig_score_noalloc: scoring that allocates no device memory.
//
// Some callers cannot let a library allocate device memory on their behalf:
// a latency-bound flow-scoring loop where a cudaMalloc/cudaFree can stall
// the device or fail under memory pressure at the worst moment, or a process
// whose device-memory budget is reserved up front by another allocator (for
// example a framework's caching allocator) so that any extra allocation may
// run out of memory.  For them this entry point scores records with the same
// kernels as ig_score, but keeps its scratch -- the A and N accumulators and
// the device status word -- in one file-scope device array of fixed size
// instead of allocating it per call.
//
// The array below is part of the library image: every GPU that loads the
// library holds it (about 4 MiB) until the process exits.  All calls share
// it and it keeps the last call's contents, so each call clears what must
// start at zero, and calls whose work overlaps on the GPU (for example on two
// streams) race on it and give wrong results.
#include <cstdio>
#include <mutex>

#include "../../include/ig.h"
#include "common.cuh"
#include "internal.h"

namespace {

constexpr int64_t kMaxRows = IG_SCORE_NOALLOC_MAX_ROWS;
constexpr int64_t kStatusWords = 32;  // first 256 bytes hold the status int

// [0, 32): status word (+ padding); then A[kMaxRows]; then N[kMaxRows].
static __device__ __align__(256) unsigned long long g_score_scratch[kStatusWords + 2 * kMaxRows];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
unsigned long long* g_scratch_addr[kMaxDevices] = {nullptr};

// Device address of the scratch array on the current device.  In host code
// the symbol names a host-side stand-in, so the address has to be looked up
// once per device (with that device current) before any kernel can be given
// it.
int scratch_address(unsigned long long** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices)
    return igk::report_error(IG_E_CUDA, "ig_score_noalloc: no usable CUDA device");
  std::lock_guard<std::mutex> lk(g_setup_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_score_scratch);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return igk::report_error(IG_E_CUDA,
                               "ig_score_noalloc: cudaGetSymbolAddress of the scratch array failed");
    }
    g_scratch_addr[dev] = static_cast<unsigned long long*>(p);
  }
  *out = g_scratch_addr[dev];
  return IG_OK;
}

int cuda_fail(cudaError_t e) {
  static thread_local char buf[256];
  snprintf(buf, sizeof(buf), "ig_score_noalloc: %s", cudaGetErrorString(e));
  return igk::report_error(IG_E_CUDA, buf);
}

}  // namespace

extern "C" int ig_score_noalloc(const ig_model* model, const uint64_t* rows, int64_t m,
                                int64_t* A_out, int64_t* N_out, uint8_t* label_out,
                                ig_stream_t stream) {
  return igk::guarded("ig_score_noalloc", [&]() -> int {
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (!model || m < 0 || (m > 0 && !rows))
      return igk::report_error(IG_E_INVAL, "ig_score_noalloc: bad arguments");
    if (m > kMaxRows)
      return igk::report_error(
          IG_E_INVAL, "ig_score_noalloc: more rows than IG_SCORE_NOALLOC_MAX_ROWS (262144) in one call");
    if (m == 0) return IG_OK;
    // Every array must be device memory of one GPU, the one holding the
    // model; that GPU is made current for the call and the caller's device is
    // put back on return.
    igk::ModelView v;
    igk::model_view(model, &v);
    int dev = -1;
    if (!igk::device_of(rows, &dev))
      return igk::report_error(IG_E_INVAL,
                               "ig_score_noalloc: rows and outputs must be device memory");
    const void* more[3] = {A_out, N_out, label_out};
    for (const void* p : more) {
      int d = -1;
      if (p && (!igk::device_of(p, &d) || d != dev))
        return igk::report_error(
            IG_E_INVAL, "ig_score_noalloc: rows and outputs must be device memory of one GPU");
    }
    for (int c = 0; c < 2; ++c) {
      int d = -1;
      if (v.n_pat[c] && (!igk::device_of(v.words_kt[c], &d) || d != dev))
        return igk::report_error(IG_E_INVAL,
                                 "ig_score_noalloc: the model lives on another GPU than the rows");
    }
    igk::DeviceRestore restore_device;
    int cur = -1;
    if (cudaGetDevice(&cur) != cudaSuccess || cur != dev) {
      cudaError_t e = cudaSetDevice(dev);
      if (e != cudaSuccess) return cuda_fail(e);
    }
    unsigned long long* scratch = nullptr;
    int rc = scratch_address(&scratch);
    if (rc != IG_OK) return rc;
    int* d_status = reinterpret_cast<int*>(scratch);
    unsigned long long* A = scratch + kStatusWords;
    unsigned long long* N = A + kMaxRows;

    cudaError_t e;
    if ((e = cudaMemsetAsync(d_status, 0, sizeof(int), s)) != cudaSuccess) return cuda_fail(e);
    if ((e = cudaMemsetAsync(A, 0, sizeof(unsigned long long) * m, s)) != cudaSuccess) return cuda_fail(e);
    if ((e = cudaMemsetAsync(N, 0, sizeof(unsigned long long) * m, s)) != cudaSuccess) return cuda_fail(e);
    for (int c = 1; c >= 0; --c) {  // A from P+, N from P- (Eq. 4)
      igk::SubsetArgs a{igk::MODE_SUM, v.KT, rows, m, v.K, v.words_kt[c], v.score[c],
                        v.n_pat[c], nullptr, c == 1 ? A : N, d_status};
      if ((e = igk::launch_subset(a, s)) != cudaSuccess) return cuda_fail(e);
    }
    if (label_out && (e = igk::launch_labels(A, N, m, v.reg3, v.thr, label_out, s)) != cudaSuccess)
      return cuda_fail(e);
    if (A_out && (e = cudaMemcpyAsync(A_out, A, sizeof(int64_t) * m, cudaMemcpyDeviceToDevice, s)) !=
                     cudaSuccess)
      return cuda_fail(e);
    if (N_out && (e = cudaMemcpyAsync(N_out, N, sizeof(int64_t) * m, cudaMemcpyDeviceToDevice, s)) !=
                     cudaSuccess)
      return cuda_fail(e);
    int st = 0;
    if ((e = cudaMemcpyAsync(&st, d_status, sizeof(int), cudaMemcpyDeviceToHost, s)) != cudaSuccess)
      return cuda_fail(e);
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_fail(e);
    if (st & igk::ST_TIMEOUT)
      return igk::report_error(IG_E_TIMEOUT, "ig_score_noalloc: a bounded device wait ran out");
    return IG_OK;
  });
}
