// Canonical order of pattern lists: ascending as KT-word unsigned integers,
// word KT-1 most significant.  The hash set hands out patterns in an
// arbitrary order; this sort makes the library's output byte-identical
// across runs (the paper's requirement that GPU and CPU pattern evidence
// agree exactly, Section 4).
//
//  1. each block sorts a tile of T keys held in shared memory with a bitonic
//     network over 16-bit indices (full KT-word comparisons);
//  2. merge passes double the sorted run length: every key finds its output
//     slot directly as (its index in its own run) + (number of keys of the
//     partner run before it), the latter by binary search -- keys of the
//     right run count equal keys of the left run as before them -- so the
//     slots form a permutation without merge-path partitioning, also when
//     keys repeat.
#include "common.cuh"
#include "internal.h"

namespace igk {

constexpr int kSortBlockThreads = 512;

template <int KT>
struct SortShape {
  // 64 KiB of keys per tile, at most 4096 keys (16-bit indices).
  static constexpr int T = (8192 / KT) > 4096 ? 4096 : (8192 / KT);
  static constexpr size_t kSmem = size_t(T) * KT * 8 + size_t(T) * 2;
};

template <int KT>
__device__ __forceinline__ bool key_less(const uint64_t* a, const uint64_t* b) {
#pragma unroll
  for (int k = KT - 1; k >= 0; --k) {
    const uint64_t x = a[k], y = b[k];
    if (x != y) return x < y;
  }
  return false;
}

template <int KT>
__global__ void __launch_bounds__(kSortBlockThreads)
    block_sort_kernel(const uint64_t* keys, int64_t n, uint64_t* out) {
  constexpr int T = SortShape<KT>::T;
  extern __shared__ __align__(16) uint64_t sk[];
  uint16_t* idx = reinterpret_cast<uint16_t*>(sk + T * KT);
  const int64_t base = int64_t(blockIdx.x) * T;
  const int nv = int((n - base) < T ? (n - base) : T);
  for (int e = threadIdx.x; e < nv * KT; e += blockDim.x) sk[e] = keys[base * KT + e];
  for (int r = threadIdx.x; r < T; r += blockDim.x) idx[r] = uint16_t(r);
  __syncthreads();
  // Indices >= nv stand for +infinity (the tile's missing tail).
  auto greater = [&](int a, int b) -> bool {
    if (a >= nv) return b < nv;
    if (b >= nv) return false;
    return key_less<KT>(sk + b * KT, sk + a * KT);
  };
  for (int k = 2; k <= T; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int t = threadIdx.x; t < T / 2; t += blockDim.x) {
        const int i = (t / j) * 2 * j + (t % j), l = i + j;
        const int a = idx[i], b = idx[l];
        const bool up = (i & k) == 0;
        if (up ? greater(a, b) : greater(b, a)) {
          idx[i] = uint16_t(b);
          idx[l] = uint16_t(a);
        }
      }
      __syncthreads();
    }
  }
  for (int e = threadIdx.x; e < nv * KT; e += blockDim.x) {
    const int r = e / KT, k = e - r * KT;
    out[base * KT + e] = sk[idx[r] * KT + k];
  }
}

template <int KT>
__global__ void merge_pass_kernel(const uint64_t* __restrict__ in, uint64_t* __restrict__ out,
                                  int64_t n, int64_t run) {
  const int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (e >= n) return;
  const int64_t r = e / run;
  const int64_t own_lo = r * run;
  const int64_t pair_lo = (r & ~int64_t(1)) * run;
  const int64_t o_lo = (r ^ 1) * run;
  const int64_t o_hi = o_lo + run < n ? o_lo + run : n;
  uint64_t key[KT];
#pragma unroll
  for (int k = 0; k < KT; ++k) key[k] = in[e * KT + k];
  // A key of the left run goes before equal keys of the right run: it counts
  // the partner's keys strictly below it, a right-run key those not above it
  // (a stable merge, so equal keys cannot collide on one slot).
  const bool left = (r & 1) == 0;
  int64_t below = 0;
  if (o_lo < n) {
    int64_t lo = o_lo, hi = o_hi;
    while (lo < hi) {
      const int64_t mid = (lo + hi) >> 1;
      const bool before = left ? key_less<KT>(in + mid * KT, key)
                               : !key_less<KT>(key, in + mid * KT);
      if (before)
        lo = mid + 1;
      else
        hi = mid;
    }
    below = lo - o_lo;
  }
  const int64_t pos = pair_lo + (e - own_lo) + below;
#pragma unroll
  for (int k = 0; k < KT; ++k) out[pos * KT + k] = key[k];
}

template <int KT>
static cudaError_t sort_t(const uint64_t* keys, int64_t n, uint64_t* keys_out, uint64_t* work,
                          cudaStream_t s) {
  using S = SortShape<KT>;
  cudaError_t e = cudaFuncSetAttribute(block_sort_kernel<KT>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, int(S::kSmem));
  if (e != cudaSuccess) return e;
  int passes = 0;
  for (int64_t run = S::T; run < n; run *= 2) ++passes;
  uint64_t* cur = (passes % 2 == 0) ? keys_out : work;
  uint64_t* other = (cur == keys_out) ? work : keys_out;
  const int64_t tiles = ceil_div(n, S::T);
  block_sort_kernel<KT><<<unsigned(tiles), kSortBlockThreads, S::kSmem, s>>>(keys, n, cur);
  count_launches(1);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  for (int64_t run = S::T; run < n; run *= 2) {
    merge_pass_kernel<KT><<<unsigned(ceil_div(n, 256)), 256, 0, s>>>(cur, other, n, run);
    count_launches(1);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    uint64_t* t = cur;
    cur = other;
    other = t;
  }
  return cudaSuccess;
}

// payload_sorted[position of keys[i] in sorted] = payload[i], found by
// binary search (sorted holds the same rows in canonical order, distinct).
template <int KT>
__global__ void place_payload_kernel(const uint64_t* __restrict__ sorted, int64_t n,
                                     const uint64_t* __restrict__ keys,
                                     const uint32_t* __restrict__ payload,
                                     uint32_t* __restrict__ payload_sorted, int* status) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  uint64_t key[KT];
#pragma unroll
  for (int k = 0; k < KT; ++k) key[k] = keys[i * KT + k];
  int64_t lo = 0, hi = n;
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (key_less<KT>(sorted + mid * KT, key))
      lo = mid + 1;
    else
      hi = mid;
  }
  if (lo >= n || key_less<KT>(key, sorted + lo * KT)) {
    set_status(status, ST_BAD_INPUT);
    return;
  }
  payload_sorted[lo] = payload[i];
}

// Flags (ST_BAD_INPUT) an empty row or two equal neighbours in a sorted list.
template <int KT>
__global__ void check_strict_kernel(const uint64_t* __restrict__ sorted, int64_t n, int* status) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  bool empty = true, same = i + 1 < n;
#pragma unroll
  for (int k = 0; k < KT; ++k) {
    const uint64_t w = sorted[i * KT + k];
    empty &= w == 0ull;
    if (i + 1 < n) same &= w == sorted[(i + 1) * KT + k];
  }
  if (empty || same) set_status(status, ST_BAD_INPUT);
}

cudaError_t launch_place_payload(const uint64_t* sorted, int64_t n, int KT, const uint64_t* keys,
                                 const uint32_t* payload, uint32_t* payload_sorted, int* status,
                                 cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  IG_DISPATCH_KT(KT, (place_payload_kernel<KTC><<<unsigned(ceil_div(n, 256)), 256, 0, s>>>(
                         sorted, n, keys, payload, payload_sorted, status)));
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_check_strict(const uint64_t* sorted, int64_t n, int KT, int* status,
                                cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  IG_DISPATCH_KT(KT, (check_strict_kernel<KTC><<<unsigned(ceil_div(n, 256)), 256, 0, s>>>(
                         sorted, n, status)));
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t canonical_sort(const uint64_t* keys, int64_t n, int KT, uint64_t* keys_out,
                           uint64_t* work, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  IG_DISPATCH_KT(KT, return sort_t<KTC>(keys, n, keys_out, work, s));
  return cudaErrorInvalidValue;
}

}  // namespace igk
