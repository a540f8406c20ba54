// Canonical order of pattern lists: ascending as KT-word unsigned integers,
// word KT-1 most significant.  The hash set hands out patterns in an
// arbitrary order; this sort makes the library's output byte-identical
// across runs (the paper's requirement that GPU and CPU pattern evidence
// agree exactly, Section 4).
//
//  1. every key gets an order-preserving 128-bit prefix (its ten highest
//     items) and is represented by (prefix, index) while it is sorted, so the
//     passes move 20 bytes per key and their searches run over arrays that
//     fit in L2; full keys are read only when two prefixes tie;
//  2. each block sorts a tile of 1,024 elements in shared memory with a
//     bitonic network (one compare-exchange per thread and stage; two
//     blocks fit an SM);
//  3. merge passes quadruple the sorted run length: every element finds its
//     output slot directly as (its index in its own run) + (number of
//     elements of the three other runs of its group before it), by binary
//     searches -- equal keys of lower runs count as before it -- so the
//     slots form a permutation without merge-path partitioning, also when
//     keys repeat;
//  4. the keys are gathered in the final order.
#include "common.cuh"
#include "internal.h"

namespace igk {

constexpr int kSortBlockThreads = 512;
constexpr int kSortTile = 1024;  // elements per block-sorted tile (one pair per thread)

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
// compared in full.
template <int KT>
__global__ void prefix_kernel(const uint64_t* __restrict__ keys, int64_t n,
                              uint64_t* __restrict__ p0, uint64_t* __restrict__ p1,
                              uint32_t* __restrict__ idx) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  uint64_t a = 0, b = 0;
  int taken = 0;
  for (int w = KT - 1; w >= 0 && taken < 10; --w) {
    uint64_t x = keys[i * KT + w];
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
  p0[i] = a;
  p1[i] = b;
  idx[i] = uint32_t(i);
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

// Bitonic network over a tile of kSortTile elements in shared memory.  The
// tile holds keys [base, base + kSortTile) (this is the first pass, so the
// element of key i carries index i); with KT <= 8 words those keys are
// staged in shared memory too, so that elements whose prefixes tie are
// compared there rather than by loads from global memory that every thread
// of the block would wait for at the next barrier.
template <int KT>
constexpr bool kSortStageKeys = KT <= 8;
template <int KT>
constexpr size_t sort_stage_bytes() {
  return kSortStageKeys<KT> ? size_t(kSortTile) * KT * 8 : 0;
}

template <int KT>
__global__ void __launch_bounds__(kSortBlockThreads)
    block_sort_kernel(const uint64_t* __restrict__ keys, int64_t n, SortArrays in,
                      SortArrays out) {
  __shared__ uint64_t s0[kSortTile];
  __shared__ uint64_t s1[kSortTile];
  __shared__ uint32_t si[kSortTile];
  extern __shared__ uint64_t tile_keys[];  // [kSortTile][KT] when staged
  const int64_t base = int64_t(blockIdx.x) * kSortTile;
  const int nv = int((n - base) < kSortTile ? (n - base) : kSortTile);
  if constexpr (kSortStageKeys<KT>) {
    for (int e = threadIdx.x; e < nv * KT; e += blockDim.x) tile_keys[e] = keys[base * KT + e];
  }
  for (int r = threadIdx.x; r < kSortTile; r += blockDim.x) {
    if (r < nv) {
      s0[r] = in.p0[base + r];
      s1[r] = in.p1[base + r];
      si[r] = in.idx[base + r];
    } else {  // +infinity: after every key
      s0[r] = ~0ull;
      s1[r] = ~0ull;
      si[r] = 0xffffffffu;
    }
  }
  __syncthreads();
  auto greater = [&](int x, int y) -> bool {
    if (si[x] == 0xffffffffu) return si[y] != 0xffffffffu;
    if (si[y] == 0xffffffffu) return false;
    if constexpr (kSortStageKeys<KT>) {
      if (s0[y] != s0[x]) return s0[y] < s0[x];
      if (s1[y] != s1[x]) return s1[y] < s1[x];
      return key_less<KT>(tile_keys + int64_t(si[y] - base) * KT,
                          tile_keys + int64_t(si[x] - base) * KT);
    } else {
      return elem_less<KT>(keys, s0[y], s1[y], si[y], s0[x], s1[x], si[x]);
    }
  };
  // k = 2^lk, j = 2^lj: pair t compares i = (t with a zero bit inserted at
  // lj) and l = i + j, in ascending order where bit lk of i is 0.
  for (int lk = 1; (1 << lk) <= kSortTile; ++lk) {
    for (int lj = lk - 1; lj >= 0; --lj) {
      const int j = 1 << lj;
      for (int t = threadIdx.x; t < kSortTile / 2; t += blockDim.x) {
        const int i = ((t >> lj) << (lj + 1)) | (t & (j - 1)), l = i + j;
        const bool up = ((i >> lk) & 1) == 0;
        if (up ? greater(i, l) : greater(l, i)) {
          const uint64_t a0 = s0[i], a1 = s1[i];
          const uint32_t ai = si[i];
          s0[i] = s0[l];
          s1[i] = s1[l];
          si[i] = si[l];
          s0[l] = a0;
          s1[l] = a1;
          si[l] = ai;
        }
      }
      __syncthreads();
    }
  }
  for (int r = threadIdx.x; r < nv; r += blockDim.x) {
    out.p0[base + r] = s0[r];
    out.p1[base + r] = s1[r];
    out.idx[base + r] = si[r];
  }
}

// Merge pass over groups of four runs: element e of run q of its group
// goes to (its index in its run) + (the number of elements of each other
// run of the group that come before it).  Equal keys order by run (those of
// lower runs first), so the slots form a permutation even when keys repeat.
// The three binary searches advance in lockstep, so their loads overlap.
template <int KT>
__global__ void merge4_pass_kernel(const uint64_t* __restrict__ keys, SortArrays in,
                                   SortArrays out, int64_t n, int64_t run) {
  const int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (e >= n) return;
  const int64_t r = e / run;
  const int64_t own_lo = r * run;
  const int64_t grp_lo = (r & ~int64_t(3)) * run;
  const int q = int(r & 3);
  const uint64_t k0 = in.p0[e], k1 = in.p1[e];
  const uint32_t ki = in.idx[e];
  int64_t lo[3], hi[3], base[3];
  bool before_eq[3];  // partner run lower than q: its equal keys come first
#pragma unroll
  for (int s = 0; s < 3; ++s) {
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
    for (int s = 0; s < 3; ++s) {
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
  const int64_t pos = grp_lo + (e - own_lo) + (lo[0] - base[0]) + (lo[1] - base[1]) +
                      (lo[2] - base[2]);
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
  const unsigned g = unsigned(ceil_div(n, 256));
  prefix_kernel<KT><<<g, 256, 0, s>>>(keys, n, A.p0, A.p1, A.idx);
  count_launches(1);
  constexpr size_t stage = sort_stage_bytes<KT>();
  if (stage > 0) {
    e = cudaFuncSetAttribute(block_sort_kernel<KT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             int(stage));
    if (e != cudaSuccess) {
      cudaFreeAsync(mem, s);
      return e;
    }
  }
  block_sort_kernel<KT><<<unsigned(ceil_div(n, kSortTile)), kSortBlockThreads, stage, s>>>(
      keys, n, A, B);
  count_launches(1);
  SortArrays cur = B, other = A;
  for (int64_t run = kSortTile; run < n; run *= 4) {
    merge4_pass_kernel<KT><<<g, 256, 0, s>>>(keys, cur, other, n, run);
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
