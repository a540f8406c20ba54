// Canonical order of pattern lists: ascending as KT-word unsigned integers,
// word KT-1 most significant.  The hash set hands out patterns in an
// arbitrary order; this sort makes the library's output byte-identical
// across runs (the paper's requirement that GPU and CPU pattern evidence
// agree exactly, Section 4).
//
//  1. every key is represented while it is sorted by (prefix, index): an
//     order-preserving 128-bit prefix (its ten highest items), so the merge
//     passes move 20 bytes per key and their searches run over arrays that
//     fit in L2; full keys are read only when two prefixes tie;
//  2. each CTA sorts a tile of kSortTile keys with a bitonic network whose
//     elements stay in registers (thread t holds tile positions t,
//     t + 1024, ...), exchanged by warp shuffles where the partner is less
//     than 32 positions away and through shared memory otherwise; the
//     tile's keys are staged in shared memory (K <= 8 words) for prefix
//     ties.  The prefixes are computed here, from the staged keys;
//  3. merge passes multiply the sorted run length by kMergeFan (4): every
//     element finds its output slot directly as (its index in its own run)
//     + (the number of elements of each other run of its group before it),
//     by binary searches advanced in lockstep so that their loads overlap;
//     equal keys of lower runs count as before it, so the slots form a
//     permutation without merge-path partitioning, also when keys repeat;
//  4. the keys are gathered in the final order.
#include "common.cuh"
#include "internal.h"

namespace igk {

constexpr int kSortThreads = 1024;
constexpr int kSortPerThread = 1;                             // tile positions per thread
constexpr int kSortTile = kSortThreads * kSortPerThread;      // elements per block-sorted tile
// Runs merged per pass.  Eight runs per pass (two passes fewer at 148k)
// measured slower than four: seven lockstep searches per element cost more
// than the passes they save.
constexpr int kMergeFan = 4;

template <int KT>
__device__ __forceinline__ bool key_less(const uint64_t* a, const uint64_t* b) {
#pragma unroll
  for (int k = KT - 1; k >= 0; --k) {
    const uint64_t x = a[k], y = b[k];
    if (x != y) return x < y;
  }
  return false;
}

// Order-preserving prefix of a key: its ten highest items, from the top,
// each as (item + 1) in a 12-bit field (0 = no further item), five per
// word.  Comparing (p0, p1) lexicographically agrees with comparing the keys
// (word KT-1 most significant): two keys first differ at the highest bit
// where one has an item and the other not, and that is the first position
// where their descending item lists differ.  Keys with equal prefixes are
// compared in full.  Every prefix word is below 2^60.
template <int KT>
__device__ __forceinline__ void key_prefix(const uint64_t* key, uint64_t& a, uint64_t& b) {
  a = 0;
  b = 0;
  int taken = 0;
  for (int w = KT - 1; w >= 0 && taken < 10; --w) {
    uint64_t x = key[w];
    while (x && taken < 10) {
      const int bit = 63 - __clzll(static_cast<long long>(x));
      x &= ~(1ull << bit);
      const uint64_t field = uint64_t(w * 64 + bit + 1);
      if (taken < 5)
        a |= field << (12 * (4 - taken));
      else
        b |= field << (12 * (9 - taken));
      ++taken;
    }
  }
}

template <int KT>
__device__ __forceinline__ bool elem_less(const uint64_t* keys, uint64_t a0, uint64_t a1,
                                          uint32_t ai, uint64_t b0, uint64_t b1, uint32_t bi) {
  if (a0 != b0) return a0 < b0;
  if (a1 != b1) return a1 < b1;
  return key_less<KT>(keys + int64_t(ai) * KT, keys + int64_t(bi) * KT);
}

struct SortArrays {
  uint64_t* p0;
  uint64_t* p1;
  uint32_t* idx;
};

// Keys staged in shared memory for the block sort's prefix ties where they
// fit beside the exchange arrays.
template <int KT>
constexpr bool kSortStageKeys = KT <= 8;
template <int KT>
constexpr size_t sort_smem_bytes() {
  return size_t(kSortTile) * (8 + 8 + 4) + (kSortStageKeys<KT> ? size_t(kSortTile) * KT * 8 : 0);
}

// One element of the block sort's network, in registers: its prefix, its
// key's index and the tile slot of its staged key.  Tile positions past the
// keys hold +inf (prefix words of all ones, above every real prefix).
struct Elem {
  uint64_t p0, p1;
  uint32_t idx;
};

// The element that position `pos` keeps from its comparator with position
// q: the smaller one at the lower position, the larger at the upper, in the
// order of (prefix, key, index), which is strict for distinct elements.  Keys
// are read at kbase + (index - base) * KT: the staged tile when kbase is
// the shared copy, else global memory.
template <int KT>
__device__ __forceinline__ Elem keep(const Elem& mine, const Elem& other, bool lower,
                                     const uint64_t* kbase, int64_t base) {
  bool other_first;
  if (other.p0 != mine.p0) {
    other_first = other.p0 < mine.p0;
  } else if (other.p1 != mine.p1) {
    other_first = other.p1 < mine.p1;
  } else if (other.idx == 0xffffffffu || mine.idx == 0xffffffffu) {
    other_first = mine.idx == 0xffffffffu && other.idx != 0xffffffffu;
  } else {
    // Equal keys order by index: the comparator must be strict, or both
    // positions would keep the same element.
    const uint64_t* ko = kbase + (int64_t(other.idx) - base) * KT;
    const uint64_t* km = kbase + (int64_t(mine.idx) - base) * KT;
    other_first = key_less<KT>(ko, km) || (!key_less<KT>(km, ko) && other.idx < mine.idx);
  }
  return lower == other_first ? other : mine;
}

// Sorts tile blockIdx.x (keys [base, base + kSortTile)) and writes its
// elements (prefix, index) in order.  The network: for each block size
// k = 2, 4, ..., kSortTile, a "flip" step pairs position i with its mirror
// i ^ (k - 1) in its k-block, then "disperse" steps pair i with i ^ j for
// j = k/4, ..., 1; every comparator puts the smaller element at the lower
// position, so the +inf positions past the tile's keys never move.
template <int KT>
__global__ void __launch_bounds__(kSortThreads, 1)
    block_sort_kernel(const uint64_t* __restrict__ keys, int64_t n, SortArrays out) {
  constexpr int E = kSortPerThread, T = kSortThreads, C = kSortTile;
  extern __shared__ __align__(16) uint8_t sh_raw[];
  uint64_t* x0 = reinterpret_cast<uint64_t*>(sh_raw);  // exchange arrays [C]
  uint64_t* x1 = x0 + C;
  uint64_t* sk = x1 + C;                                // staged keys [C][KT] (K <= 8)
  uint32_t* xi = reinterpret_cast<uint32_t*>(sk + (kSortStageKeys<KT> ? size_t(C) * KT : 0));
  const int64_t base = int64_t(blockIdx.x) * C;
  const int nv = int((n - base) < C ? (n - base) : C);
  const uint64_t* kbase = keys + base * KT;
  if constexpr (kSortStageKeys<KT>) {
    for (int q = threadIdx.x; q < nv * KT; q += T) sk[q] = kbase[q];
    __syncthreads();
    kbase = sk;
  }
  Elem el[E];
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const int pos = threadIdx.x + e * T;
    if (pos < nv) {
      key_prefix<KT>(kbase + int64_t(pos) * KT, el[e].p0, el[e].p1);
      el[e].idx = uint32_t(base + pos);
    } else {
      el[e].p0 = ~0ull;
      el[e].p1 = ~0ull;
      el[e].idx = 0xffffffffu;
    }
  }
  const int lane = threadIdx.x & 31;
  for (int k = 2; k <= C; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      const int d = j == (k >> 1) ? k - 1 : j;  // partner = position ^ d
      if (d < 32) {
#pragma unroll
        for (int e = 0; e < E; ++e) {
          Elem o;
          o.p0 = __shfl_xor_sync(0xffffffffu, el[e].p0, d);
          o.p1 = __shfl_xor_sync(0xffffffffu, el[e].p1, d);
          o.idx = __shfl_xor_sync(0xffffffffu, el[e].idx, d);
          el[e] = keep<KT>(el[e], o, lane < (lane ^ d), kbase, base);
        }
      } else {
#pragma unroll
        for (int e = 0; e < E; ++e) {
          const int pos = threadIdx.x + e * T;
          x0[pos] = el[e].p0;
          x1[pos] = el[e].p1;
          xi[pos] = el[e].idx;
        }
        __syncthreads();
#pragma unroll
        for (int e = 0; e < E; ++e) {
          const int pos = threadIdx.x + e * T, q = pos ^ d;
          Elem o;
          o.p0 = x0[q];
          o.p1 = x1[q];
          o.idx = xi[q];
          el[e] = keep<KT>(el[e], o, pos < q, kbase, base);
        }
        __syncthreads();
      }
    }
  }
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const int pos = threadIdx.x + e * T;
    if (pos < nv) {
      out.p0[base + pos] = el[e].p0;
      out.p1[base + pos] = el[e].p1;
      out.idx[base + pos] = el[e].idx;
    }
  }
}

// Merge pass over groups of kMergeFan runs: element e of run q of its group
// goes to (its index in its run) + (the number of elements of each other
// run of the group that come before it).  Equal keys order by run (those of
// lower runs first), so the slots form a permutation even when keys repeat.
// The binary searches advance in lockstep, so their loads overlap.
template <int KT>
__global__ void merge_pass_kernel(const uint64_t* __restrict__ keys, SortArrays in,
                                  SortArrays out, int64_t n, int64_t run) {
  constexpr int F = kMergeFan;
  const int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (e >= n) return;
  const int64_t r = e / run;
  const int64_t own_lo = r * run;
  const int64_t grp_lo = (r / F) * F * run;
  const int q = int(r % F);
  const uint64_t k0 = in.p0[e], k1 = in.p1[e];
  const uint32_t ki = in.idx[e];
  int64_t lo[F - 1], hi[F - 1], base[F - 1];
  bool before_eq[F - 1];  // partner run lower than q: its equal keys come first
#pragma unroll
  for (int s = 0; s < F - 1; ++s) {
    const int qq = s < q ? s : s + 1;
    const int64_t a = grp_lo + int64_t(qq) * run;
    base[s] = a < n ? a : n;
    lo[s] = base[s];
    hi[s] = a + run < n ? a + run : n;
    before_eq[s] = qq < q;
  }
  bool more = true;
  while (more) {
    more = false;
#pragma unroll
    for (int s = 0; s < F - 1; ++s) {
      if (lo[s] < hi[s]) {
        const int64_t mid = (lo[s] + hi[s]) >> 1;
        const uint64_t m0 = in.p0[mid], m1 = in.p1[mid];
        const uint32_t mi = in.idx[mid];
        const bool before = before_eq[s] ? !elem_less<KT>(keys, k0, k1, ki, m0, m1, mi)
                                         : elem_less<KT>(keys, m0, m1, mi, k0, k1, ki);
        if (before)
          lo[s] = mid + 1;
        else
          hi[s] = mid;
        more |= lo[s] < hi[s];
      }
    }
  }
  int64_t pos = grp_lo + (e - own_lo);
#pragma unroll
  for (int s = 0; s < F - 1; ++s) pos += lo[s] - base[s];
  out.p0[pos] = k0;
  out.p1[pos] = k1;
  out.idx[pos] = ki;
}

__global__ void gather_rows_kernel(const uint64_t* __restrict__ keys, int KT,
                                   const uint32_t* __restrict__ idx, int64_t n,
                                   uint64_t* __restrict__ out) {
  const int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t >= n * KT) return;
  const int64_t i = t / KT;
  const int k = int(t - i * KT);
  out[t] = keys[int64_t(idx[i]) * KT + k];
}

template <int KT>
static cudaError_t sort_t(const uint64_t* keys, int64_t n, uint64_t* keys_out, uint32_t* perm_out,
                          cudaStream_t s) {
  // Two sets of (p0, p1, idx) arrays, ping-ponged by the passes.
  void* mem = nullptr;
  cudaError_t e = cudaMallocAsync(&mem, size_t(n) * 40, s);
  if (e != cudaSuccess) return e;
  uint8_t* m = static_cast<uint8_t*>(mem);
  SortArrays A{reinterpret_cast<uint64_t*>(m), reinterpret_cast<uint64_t*>(m + 8 * n),
               reinterpret_cast<uint32_t*>(m + 32 * n)};
  SortArrays B{reinterpret_cast<uint64_t*>(m + 16 * n), reinterpret_cast<uint64_t*>(m + 24 * n),
               reinterpret_cast<uint32_t*>(m + 36 * n)};
  constexpr size_t smem = sort_smem_bytes<KT>();
  e = cudaFuncSetAttribute(block_sort_kernel<KT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           int(smem));
  if (e != cudaSuccess) {
    cudaFreeAsync(mem, s);
    return e;
  }
  block_sort_kernel<KT><<<unsigned(ceil_div(n, kSortTile)), kSortThreads, smem, s>>>(keys, n, A);
  count_launches(1);
  SortArrays cur = A, other = B;
  const unsigned g = unsigned(ceil_div(n, 256));
  for (int64_t run = kSortTile; run < n; run *= kMergeFan) {
    merge_pass_kernel<KT><<<g, 256, 0, s>>>(keys, cur, other, n, run);
    count_launches(1);
    const SortArrays t = cur;
    cur = other;
    other = t;
  }
  gather_rows_kernel<<<unsigned(ceil_div(n * KT, 256)), 256, 0, s>>>(keys, KT, cur.idx, n,
                                                                     keys_out);
  count_launches(1);
  e = cudaGetLastError();
  if (e == cudaSuccess && perm_out)
    e = cudaMemcpyAsync(perm_out, cur.idx, size_t(n) * 4, cudaMemcpyDeviceToDevice, s);
  cudaFreeAsync(mem, s);
  return e;
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
                           uint64_t* /*work*/, cudaStream_t s, uint32_t* perm_out) {
  if (n == 0) return cudaSuccess;
  if (n >= int64_t(0xffffffffll)) return cudaErrorInvalidValue;
  IG_DISPATCH_KT(KT, return sort_t<KTC>(keys, n, keys_out, perm_out, s));
  return cudaErrorInvalidValue;
}

}  // namespace igk
