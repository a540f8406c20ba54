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

// Stable partition of the records by label (the order of the records
// within each class is kept), in three launches:
//   1. each block of kSplitRows records counts its attack records;
//   2. an exclusive scan of the block counts gives every block its first
//      attack slot (and its first normal slot: block start - attack slots);
//   3. each block ranks its records by a block-wide scan of the attack flags
//      and copies all their words together, so reads are coalesced and each
//      warp store covers consecutive words of one or a few rows.
constexpr int kSplitRows = 1024;

__global__ void __launch_bounds__(kSplitRows)
    split_count_kernel(const uint8_t* __restrict__ labels, int64_t n,
                       uint32_t* __restrict__ block_att, int* status) {
  __shared__ uint32_t warp_sum[kSplitRows / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t i = int64_t(blockIdx.x) * kSplitRows + threadIdx.x;
  uint8_t lab = i < n ? labels[i] : 0;
  if (lab > 1) {
    set_status(status, ST_BAD_INPUT);
    lab = 1;
  }
  const uint32_t ballot = __ballot_sync(0xffffffffu, lab == 1);
  if (lane == 0) warp_sum[warp] = __popc(ballot);
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t t = 0;
    for (int w = 0; w < kSplitRows / 32; ++w) t += warp_sum[w];
    block_att[blockIdx.x] = t;
  }
}

__global__ void __launch_bounds__(kSplitRows)
    split_scatter_kernel(const uint64_t* __restrict__ rows, const uint8_t* __restrict__ labels,
                         int64_t n, int K, int KT, const uint32_t* __restrict__ att_before,
                         int n_blocks, uint64_t* __restrict__ x0, uint64_t* __restrict__ x1,
                         unsigned long long* counts) {
  __shared__ uint32_t warp_sum[kSplitRows / 32];
  __shared__ int64_t slot[kSplitRows];  // >= 0: row of x1; < 0: ~row of x0
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t start = int64_t(blockIdx.x) * kSplitRows;
  const int64_t i = start + threadIdx.x;
  const bool att = i < n && labels[i] >= 1;  // labels > 1 were reported by the count
  const uint32_t ballot = __ballot_sync(0xffffffffu, att);
  if (lane == 0) warp_sum[warp] = __popc(ballot);
  __syncthreads();
  uint32_t before = 0;
  for (int w = 0; w < warp; ++w) before += warp_sum[w];
  const uint32_t mine = before + __popc(ballot & ((1u << lane) - 1u));
  const int64_t a = int64_t(att_before[blockIdx.x]) + mine;  // attack records before i
  slot[threadIdx.x] = att ? a : ~(i - a);
  __syncthreads();
  const int nv = int(n - start < kSplitRows ? n - start : kSplitRows);
  for (int e = threadIdx.x; e < nv * KT; e += kSplitRows) {
    const int r = e / KT, k = e - r * KT;
    const int64_t sl = slot[r];
    const uint64_t v = k < K ? rows[(start + r) * K + k] : 0ull;
    if (sl >= 0)
      x1[sl * KT + k] = v;
    else
      x0[(~sl) * KT + k] = v;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    counts[1] = (unsigned long long)att_before[n_blocks];
    counts[0] = (unsigned long long)(n - int64_t(att_before[n_blocks]));
  }
}

cudaError_t launch_split(const uint64_t* rows, const uint8_t* labels, int64_t n,
                         int K, int KT, uint64_t* x0, uint64_t* x1,
                         unsigned long long* counts, int* status, cudaStream_t s) {
  const int nb = int(ceil_div(n, kSplitRows));
  if (nb == 0) return cudaMemsetAsync(counts, 0, 2 * sizeof(unsigned long long), s);
  void* mem = nullptr;
  cudaError_t e = cudaMallocAsync(&mem, size_t(2 * nb + 1) * 4, s);
  if (e != cudaSuccess) return e;
  uint32_t* block_att = static_cast<uint32_t*>(mem);
  uint32_t* att_before = block_att + nb;  // nb + 1 entries
  split_count_kernel<<<nb, kSplitRows, 0, s>>>(labels, n, block_att, status);
  e = launch_small_scan(block_att, nb, att_before, s);
  if (e == cudaSuccess) {
    split_scatter_kernel<<<nb, kSplitRows, 0, s>>>(rows, labels, n, K, KT, att_before, nb, x0, x1,
                                                   counts);
    count_launches(2);
    e = cudaGetLastError();
  }
  cudaFreeAsync(mem, s);
  return e;
}

}  // namespace igk
