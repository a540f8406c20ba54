// Candidate generation and deduplication (Eq. 1; pairwise intersection as
// in Section 3.3).
//
// Every pair i <= j of one class's records is ANDed (i == j yields the record
// itself, the "union X^c" term of Eq. 1) and the non-empty results are
// inserted into an open-addressing hash table keyed on all KT words, so
// B^c is formed as a set on the device without materialising the O(n^2)
// intersections.
//
// Table layout: tags[cap] (uint32: 0 empty, 1 claimed and being written,
// otherwise 0x80000000 | 31 fingerprint bits) and keys[cap][KT].  A slot is
// claimed by CAS on its tag, its key written, then the tag is published with
// a release store; readers load tags with acquire semantics, so a published
// fingerprint guarantees the key words are visible.  Linear probing; the
// host keeps the load factor below 0.7 so every probe sequence ends at an
// empty slot, and waits on a claimed slot are bounded.
#include "common.cuh"
#include "internal.h"

namespace igk {

constexpr uint32_t kTagBusy = 1u;
constexpr uint32_t kTagReady = 0x80000000u;

struct TableView {
  uint32_t* tags;
  uint64_t* keys;
  uint64_t mask;
  unsigned long long* count;
};

// Returns 1 if inserted, 0 if already present, -1 on a bounded-wait timeout
// or a full table (status set).
template <int KT>
__device__ int table_insert(const TableView& t, const uint64_t (&b)[KT],
                            uint64_t h, int* status) {
  const uint32_t fp = kTagReady | uint32_t(h >> 33);
  uint64_t slot = h & t.mask;
  for (uint64_t probe = 0; probe <= t.mask; ++probe) {
    uint32_t tag = ld_acquire_u32(t.tags + slot);
    if (tag == 0u) {
      uint32_t old = atomicCAS(t.tags + slot, 0u, kTagBusy);
      if (old == 0u) {
        uint64_t* dst = t.keys + slot * KT;
#pragma unroll
        for (int k = 0; k < KT; ++k) dst[k] = b[k];
        st_release_u32(t.tags + slot, fp);
        atomicAdd(t.count, 1ull);
        return 1;
      }
      tag = old;
    }
    if (tag == kTagBusy) {
      uint32_t spins = 0;
      do {
        __nanosleep(32);
        tag = ld_acquire_u32(t.tags + slot);
      } while (tag == kTagBusy && ++spins < kSlotSpinLimit);
      if (tag == kTagBusy) {
        set_status(status, ST_TIMEOUT);
        return -1;
      }
    }
    if (tag == fp) {
      const uint64_t* src = t.keys + slot * KT;
      bool same = true;
#pragma unroll
      for (int k = 0; k < KT; ++k) same &= (ld_relaxed_u64(src + k) == b[k]);
      if (same) return 0;
    }
    slot = (slot + 1) & t.mask;
  }
  set_status(status, ST_TABLE_FULL);
  return -1;
}

constexpr int kPairThreads = 256;

// Grid: x = column tile bj, y = row tile bi - row_lo.  Tiles with bj < bi
// lie below the diagonal and exit at once.  Shared rows use an odd stride of
// KT + 1 words so that lanes reading consecutive rows hit distinct banks.
template <int KT>
__global__ void __launch_bounds__(kPairThreads)
    pair_insert_kernel(const uint64_t* __restrict__ X, int64_t n, int64_t row_lo,
                       TableView t, int* status) {
  constexpr int T = kPairTile;
  constexpr int SKT = KT + 1;
  __shared__ uint64_t A[T * SKT];
  __shared__ uint64_t B[T * SKT];
  const int64_t bi = row_lo + blockIdx.y, bj = blockIdx.x;
  if (bj < bi) return;
  const int64_t i0 = bi * T, j0 = bj * T;
  for (int e = threadIdx.x; e < T * KT; e += kPairThreads) {
    int r = e / KT, k = e - r * KT;
    A[r * SKT + k] = (i0 + r < n) ? X[(i0 + r) * KT + k] : 0ull;
    B[r * SKT + k] = (j0 + r < n) ? X[(j0 + r) * KT + k] : 0ull;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31;
  for (int p = threadIdx.x; p < T * T; p += kPairThreads) {
    const int i = p / T, j = p - (p / T) * T;
    bool valid = (i0 + i < n) && (j0 + j < n) && (bi < bj || i <= j);
    uint64_t b[KT];
    uint64_t any = 0;
#pragma unroll
    for (int k = 0; k < KT; ++k) {
      b[k] = A[i * SKT + k] & B[j * SKT + k];
      any |= b[k];
    }
    bool has = valid && any != 0;
    unsigned active = __ballot_sync(0xffffffffu, has);
    if (!has) continue;
    uint64_t h = hash_key<KT>(b);
    // Lanes holding the same key insert it once: the lowest lane of each
    // group of equal hashes is its leader; a lane whose key equals its
    // leader's skips the insert.
    unsigned peers = __match_any_sync(active, h);
    int leader = __ffs(peers) - 1;
    bool same = true;
#pragma unroll
    for (int k = 0; k < KT; ++k) same &= (__shfl_sync(active, b[k], leader) == b[k]);
    if (leader != lane && same) continue;
    table_insert<KT>(t, b, h, status);
  }
}

template <int KT>
__global__ void rehash_kernel(TableView from, TableView to, int* status) {
  int64_t s = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (s > int64_t(from.mask)) return;
  uint32_t tag = from.tags[s];
  if (!(tag & kTagReady)) return;
  uint64_t b[KT];
#pragma unroll
  for (int k = 0; k < KT; ++k) b[k] = from.keys[s * KT + k];
  table_insert<KT>(to, b, hash_key<KT>(b), status);
}

// Warp-aggregated append of every published key.
template <int KT>
__global__ void compact_kernel(TableView t, uint64_t* __restrict__ out,
                               unsigned long long* out_count) {
  const int lane = threadIdx.x & 31;
  const int64_t cap = int64_t(t.mask) + 1;
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  for (int64_t base = int64_t(blockIdx.x) * blockDim.x + (threadIdx.x & ~31);
       base < cap; base += stride) {
    int64_t s = base + lane;
    bool ready = s < cap && (t.tags[s] & kTagReady);
    unsigned m = __ballot_sync(0xffffffffu, ready);
    if (m == 0) continue;
    unsigned long long pos0 = 0;
    if (lane == 0) pos0 = atomicAdd(out_count, (unsigned long long)__popc(m));
    pos0 = __shfl_sync(0xffffffffu, pos0, 0);
    if (ready) {
      uint64_t pos = pos0 + __popc(m & ((1u << lane) - 1u));
#pragma unroll
      for (int k = 0; k < KT; ++k) out[pos * KT + k] = t.keys[s * KT + k];
    }
  }
}

static TableView view(const HashTable& t) {
  return TableView{t.tags, t.keys, t.cap - 1, t.count};
}

cudaError_t launch_pair_insert(const uint64_t* X, int64_t n, int KT,
                               int64_t row_lo, int64_t row_hi, HashTable t,
                               int* status, cudaStream_t s) {
  int64_t nt = ceil_div(n, kPairTile);
  if (row_hi <= row_lo || nt == 0) return cudaSuccess;
  dim3 grid(unsigned(nt), unsigned(row_hi - row_lo));
  IG_DISPATCH_KT(KT, (pair_insert_kernel<KTC><<<grid, kPairThreads, 0, s>>>(
                         X, n, row_lo, view(t), status)));
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_rehash(HashTable from, HashTable to, int KT, int* status,
                          cudaStream_t s) {
  unsigned blocks = unsigned(ceil_div(int64_t(from.cap), 256));
  IG_DISPATCH_KT(KT, (rehash_kernel<KTC><<<blocks, 256, 0, s>>>(view(from), view(to), status)));
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_compact(HashTable t, int KT, uint64_t* out,
                           unsigned long long* out_count, cudaStream_t s) {
  int64_t blocks = ceil_div(int64_t(t.cap), 256);
  if (blocks > 4 * 1024) blocks = 4 * 1024;
  IG_DISPATCH_KT(KT, (compact_kernel<KTC><<<unsigned(blocks), 256, 0, s>>>(view(t), out, out_count)));
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace igk
