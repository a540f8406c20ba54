// Canonical order of pattern lists: ascending as KT-word unsigned integers,
// word KT-1 most significant.  The hash table hands out patterns in an
// arbitrary order; this sort makes the library's output byte-identical
// across runs (the paper's requirement that GPU and CPU pattern evidence
// agree exactly, Section 4).
//
// LSD radix sort of a uint32 index permutation on 8-bit digits, least
// significant digit first.  Digits whose value is the same in every key
// (found from an OR- and an AND-reduction of all keys) cannot change the
// order and are skipped.  Each pass is three kernels: a per-block digit
// histogram, one exclusive scan of the (digit, block) matrix in digit-major
// order, and a stable scatter in which each block ranks its items per digit
// with warp match-any votes, round by round in item order.
#include "common.cuh"
#include "internal.h"

namespace igk {

constexpr int kSortThreads = 256;
constexpr int kSortRounds = 8;
constexpr int kSortTile = kSortThreads * kSortRounds;
constexpr int kScanThreads = 1024;

__global__ void key_or_and_kernel(const uint64_t* __restrict__ keys, int64_t n,
                                  int KT, unsigned long long* or_and) {
  uint64_t o[IG_MAX_KT_WORDS], a[IG_MAX_KT_WORDS];
  for (int k = 0; k < KT; ++k) {
    o[k] = 0ull;
    a[k] = ~0ull;
  }
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += stride)
    for (int k = 0; k < KT; ++k) {
      uint64_t w = keys[i * KT + k];
      o[k] |= w;
      a[k] &= w;
    }
  for (int k = 0; k < KT; ++k) {
    uint64_t ok = o[k], ak = a[k];
    for (int d = 16; d > 0; d >>= 1) {
      ok |= __shfl_xor_sync(0xffffffffu, ok, d);
      ak &= __shfl_xor_sync(0xffffffffu, ak, d);
    }
    if ((threadIdx.x & 31) == 0) {
      atomicOr(or_and + k, (unsigned long long)ok);
      atomicAnd(or_and + IG_MAX_KT_WORDS + k, (unsigned long long)ak);
    }
  }
}

__global__ void iota_kernel(uint32_t* idx, int64_t n) {
  int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i < n) idx[i] = uint32_t(i);
}

__device__ __forceinline__ uint32_t key_digit(const uint64_t* keys, int KT,
                                              uint32_t id, int word, int shift) {
  return uint32_t((keys[int64_t(id) * KT + word] >> shift) & 0xffu);
}

__global__ void __launch_bounds__(kSortThreads)
    radix_hist_kernel(const uint64_t* __restrict__ keys, int KT, int word, int shift,
                      const uint32_t* __restrict__ idx, int64_t n,
                      uint32_t* __restrict__ hist, int nblocks) {
  __shared__ uint32_t cnt[256];
  cnt[threadIdx.x] = 0;
  __syncthreads();
  const int64_t base = int64_t(blockIdx.x) * kSortTile;
  for (int r = 0; r < kSortRounds; ++r) {
    int64_t i = base + r * kSortThreads + threadIdx.x;
    if (i < n) atomicAdd(&cnt[key_digit(keys, KT, idx[i], word, shift)], 1u);
  }
  __syncthreads();
  hist[int64_t(threadIdx.x) * nblocks + blockIdx.x] = cnt[threadIdx.x];
}

// Exclusive scan of len values in place, by one block: each thread sums a
// contiguous chunk, the chunk sums are scanned across the block, and the
// chunks are rewritten with their running offsets.
__global__ void __launch_bounds__(kScanThreads)
    exclusive_scan_kernel(uint32_t* __restrict__ v, int64_t len) {
  __shared__ uint32_t part[kScanThreads];
  const int64_t chunk = ceil_div(len, kScanThreads);
  const int64_t lo = int64_t(threadIdx.x) * chunk;
  const int64_t hi = lo + chunk < len ? lo + chunk : len;
  uint32_t s = 0;
  for (int64_t i = lo; i < hi; ++i) s += v[i];
  part[threadIdx.x] = s;
  __syncthreads();
  for (int off = 1; off < kScanThreads; off <<= 1) {
    uint32_t add = threadIdx.x >= off ? part[threadIdx.x - off] : 0u;
    __syncthreads();
    part[threadIdx.x] += add;
    __syncthreads();
  }
  uint32_t run = part[threadIdx.x] - s;
  for (int64_t i = lo; i < hi; ++i) {
    uint32_t x = v[i];
    v[i] = run;
    run += x;
  }
}

__global__ void __launch_bounds__(kSortThreads)
    radix_scatter_kernel(const uint64_t* __restrict__ keys, int KT, int word, int shift,
                         const uint32_t* __restrict__ idx_in,
                         uint32_t* __restrict__ idx_out, int64_t n,
                         const uint32_t* __restrict__ offsets, int nblocks) {
  constexpr int W = kSortThreads / 32;
  __shared__ uint32_t run[256];
  __shared__ uint32_t wcnt[W][256];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  run[threadIdx.x] = offsets[int64_t(threadIdx.x) * nblocks + blockIdx.x];
  const int64_t base = int64_t(blockIdx.x) * kSortTile;
  for (int r = 0; r < kSortRounds; ++r) {
    const int64_t i = base + r * kSortThreads + threadIdx.x;
    const bool valid = i < n;
    const uint32_t id = valid ? idx_in[i] : 0u;
    const uint32_t d = valid ? key_digit(keys, KT, id, word, shift) : 256u;
#pragma unroll
    for (int w = 0; w < W; ++w) wcnt[w][threadIdx.x] = 0;
    __syncthreads();
    const unsigned peers = __match_any_sync(0xffffffffu, d);
    const uint32_t rank = __popc(peers & ((1u << lane) - 1u));
    if (valid && rank == 0) wcnt[warp][d] = __popc(peers);
    __syncthreads();
    {  // column threadIdx.x: offsets of each warp's group of this digit
      uint32_t acc = run[threadIdx.x];
#pragma unroll
      for (int w = 0; w < W; ++w) {
        uint32_t c = wcnt[w][threadIdx.x];
        wcnt[w][threadIdx.x] = acc;
        acc += c;
      }
      run[threadIdx.x] = acc;
    }
    __syncthreads();
    if (valid) idx_out[wcnt[warp][d] + rank] = id;
    __syncthreads();
  }
}

__global__ void gather_rows_kernel(const uint64_t* __restrict__ keys, int KT,
                                   const uint32_t* __restrict__ idx, int64_t n,
                                   uint64_t* __restrict__ out) {
  int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t >= n * KT) return;
  int64_t i = t / KT;
  int k = int(t - i * KT);
  out[t] = keys[int64_t(idx[i]) * KT + k];
}

cudaError_t canonical_sort(const uint64_t* keys, int64_t n, int KT,
                           uint64_t* keys_out, int* /*status*/, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  if (n > int64_t(0xffffffffu)) return cudaErrorInvalidValue;
  cudaError_t e;
  const int nblocks = int(ceil_div(n, kSortTile));
  uint32_t *idx_a = nullptr, *idx_b = nullptr, *hist = nullptr;
  unsigned long long* or_and = nullptr;
  unsigned long long host_or_and[2 * IG_MAX_KT_WORDS];
  auto cleanup = [&]() {
    if (idx_a) cudaFreeAsync(idx_a, s);
    if (idx_b) cudaFreeAsync(idx_b, s);
    if (hist) cudaFreeAsync(hist, s);
    if (or_and) cudaFreeAsync(or_and, s);
  };
#define IG_SORT_TRY(x)      \
  if ((e = (x)) != cudaSuccess) { \
    cleanup();              \
    return e;               \
  }
  IG_SORT_TRY(cudaMallocAsync(&idx_a, sizeof(uint32_t) * n, s));
  IG_SORT_TRY(cudaMallocAsync(&idx_b, sizeof(uint32_t) * n, s));
  IG_SORT_TRY(cudaMallocAsync(&hist, sizeof(uint32_t) * 256 * nblocks, s));
  IG_SORT_TRY(cudaMallocAsync(&or_and, sizeof(host_or_and), s));
  IG_SORT_TRY(cudaMemsetAsync(or_and, 0, sizeof(unsigned long long) * IG_MAX_KT_WORDS, s));
  IG_SORT_TRY(cudaMemsetAsync(or_and + IG_MAX_KT_WORDS, 0xff,
                              sizeof(unsigned long long) * IG_MAX_KT_WORDS, s));
  {
    int64_t blocks = ceil_div(n, 256);
    if (blocks > 1024) blocks = 1024;
    key_or_and_kernel<<<unsigned(blocks), 256, 0, s>>>(keys, n, KT, or_and);
    count_launches(1);
    IG_SORT_TRY(cudaGetLastError());
  }
  IG_SORT_TRY(cudaMemcpyAsync(host_or_and, or_and, sizeof(host_or_and),
                              cudaMemcpyDeviceToHost, s));
  iota_kernel<<<unsigned(ceil_div(n, 256)), 256, 0, s>>>(idx_a, n);
  count_launches(1);
  IG_SORT_TRY(cudaGetLastError());
  IG_SORT_TRY(cudaStreamSynchronize(s));
  for (int word = 0; word < KT; ++word) {
    const uint64_t varies = host_or_and[word] ^ host_or_and[IG_MAX_KT_WORDS + word];
    for (int shift = 0; shift < 64; shift += 8) {
      if (((varies >> shift) & 0xffull) == 0) continue;
      radix_hist_kernel<<<nblocks, kSortThreads, 0, s>>>(keys, KT, word, shift, idx_a,
                                                         n, hist, nblocks);
      IG_SORT_TRY(cudaGetLastError());
      exclusive_scan_kernel<<<1, kScanThreads, 0, s>>>(hist, int64_t(256) * nblocks);
      IG_SORT_TRY(cudaGetLastError());
      radix_scatter_kernel<<<nblocks, kSortThreads, 0, s>>>(keys, KT, word, shift, idx_a,
                                                            idx_b, n, hist, nblocks);
      IG_SORT_TRY(cudaGetLastError());
      count_launches(3);
      uint32_t* t = idx_a;
      idx_a = idx_b;
      idx_b = t;
    }
  }
  gather_rows_kernel<<<unsigned(ceil_div(n * KT, 256)), 256, 0, s>>>(keys, KT, idx_a, n,
                                                                     keys_out);
  IG_SORT_TRY(cudaGetLastError());
  count_launches(1);
  cleanup();
  return cudaSuccess;
#undef IG_SORT_TRY
}

}  // namespace igk
