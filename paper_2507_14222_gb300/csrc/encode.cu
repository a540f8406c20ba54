// Record encoding (Section 3.1, Eq. 5) and the class split of Section 3.2.
#include "common.cuh"
#include "internal.h"

namespace igk {

// One thread per output word (record i, word k): OR in the item bit of
// every feature whose item range [offsets[f], offsets[f+1]) reaches word k.
// Consecutive threads write consecutive words of the same record.
__global__ void encode_kernel(const uint16_t* __restrict__ codes, int64_t n,
                              int F, const uint32_t* __restrict__ offsets,
                              uint64_t* __restrict__ out, int K, int* status) {
  int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t >= n * K) return;
  int64_t i = t / K;
  int k = int(t - i * K);
  const uint16_t* c = codes + i * F;
  uint64_t w = 0;
  bool bad = false;
  for (int f = 0; f < F; ++f) {
    uint32_t lo = offsets[f], hi = offsets[f + 1];
    if (hi <= uint32_t(k) * 64u || lo >= uint32_t(k + 1) * 64u) continue;
    uint32_t v = c[f];
    if (v == 0xffffu) continue;  // missing value: no item for this feature
    if (v >= hi - lo) {
      bad = true;
      continue;
    }
    uint32_t item = lo + v;
    if ((item >> 6) == uint32_t(k)) w |= 1ull << (item & 63u);
  }
  if (bad) set_status(status, ST_BAD_INPUT);
  out[t] = w;
}

cudaError_t launch_encode(const uint16_t* codes, int64_t n, int F,
                          const uint32_t* offsets, const uint16_t* /*cards*/,
                          uint64_t* out, int K, int* status, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  int64_t total = n * K;
  int threads = 256;
  int64_t blocks = ceil_div(total, threads);
  encode_kernel<<<unsigned(blocks), threads, 0, s>>>(codes, n, F, offsets, out,
                                                    K, status);
  count_launches(1);
  return cudaGetLastError();
}

// Stable partition of the records by label (one block; the order of the
// records within each class is kept).  A block-wide exclusive scan of the
// attack flags gives each record its slot in x1 (attack) or x0 (normal).
constexpr int kSplitThreads = 1024;

__global__ void __launch_bounds__(kSplitThreads)
    split_kernel(const uint64_t* __restrict__ rows, const uint8_t* __restrict__ labels,
                 int64_t n, int K, int KT, uint64_t* __restrict__ x0,
                 uint64_t* __restrict__ x1, unsigned long long* counts,
                 int* status) {
  __shared__ uint32_t warp_sum[kSplitThreads / 32];
  __shared__ int64_t base1;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) base1 = 0;
  __syncthreads();
  for (int64_t start = 0; start < n; start += kSplitThreads) {
    int64_t i = start + threadIdx.x;
    bool valid = i < n;
    uint8_t lab = valid ? labels[i] : 0;
    if (lab > 1) {
      set_status(status, ST_BAD_INPUT);
      lab = 1;
    }
    bool att = valid && lab == 1;
    uint32_t ballot = __ballot_sync(0xffffffffu, att);
    if (lane == 0) warp_sum[warp] = __popc(ballot);
    __syncthreads();
    uint32_t before = 0, total = 0;
    for (int w = 0; w < kSplitThreads / 32; ++w) {
      uint32_t v = warp_sum[w];
      if (w < warp) before += v;
      total += v;
    }
    int64_t r1 = base1 + before + __popc(ballot & ((1u << lane) - 1u));
    int64_t r0 = (start - base1) + (threadIdx.x - (before + __popc(ballot & ((1u << lane) - 1u))));
    if (valid) {
      uint64_t* dst = att ? x1 + r1 * KT : x0 + r0 * KT;
      const uint64_t* src = rows + i * K;
      for (int k = 0; k < KT; ++k) dst[k] = k < K ? src[k] : 0ull;
    }
    __syncthreads();
    if (threadIdx.x == 0) base1 += total;
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    counts[1] = (unsigned long long)base1;
    counts[0] = (unsigned long long)(n - base1);
  }
}

cudaError_t launch_split(const uint64_t* rows, const uint8_t* labels, int64_t n,
                         int K, int KT, uint64_t* x0, uint64_t* x1,
                         unsigned long long* counts, int* status, cudaStream_t s) {
  split_kernel<<<1, kSplitThreads, 0, s>>>(rows, labels, n, K, KT, x0, x1,
                                           counts, status);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace igk
