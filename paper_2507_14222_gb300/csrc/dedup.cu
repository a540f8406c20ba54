// Candidate generation and deduplication (Eq. 1; pairwise intersection as
// in Section 3.3).
//
// Every pair i <= j of one class's records is ANDed (i == j yields the record
// itself, the "union X^c" term of Eq. 1) and the non-empty results are
// inserted into an open-addressing hash set, so B^c is formed as a set on
// the device without materialising the O(n^2) intersections.
//
// A slot is one 64-bit word: 0 = empty, otherwise
//   bit 63 = 1 | 19 fingerprint bits (62..44) | i (43..22) | j (21..0),
// naming the pair whose intersection is the stored key.  The key itself is
// never stored: it is recomputed as X[i] AND X[j] from the class's records,
// which are read-only while the table is built.  A key is therefore claimed
// and published by a single 64-bit CAS -- there is no half-written state,
// no acquire/release protocol and no waiting on another thread's slot.
//
// Overflow cannot happen: before claiming an empty slot a thread takes a
// reservation (atomicAdd on `reserved`) and gives up if the table already
// holds `limit` keys (half its capacity), recording its tile band.  The host
// then doubles the table, rehashes it, and replays the bands from the first
// failed one (inserts are idempotent).
#include "common.cuh"
#include "internal.h"

namespace igk {

constexpr int kIdxBits = 22;
constexpr uint64_t kIdxMask = (1ull << kIdxBits) - 1;
constexpr uint64_t kFpMask = 0xfffff00000000000ull;  // bit 63 + 19 fingerprint bits

__device__ __forceinline__ uint64_t slot_value(uint64_t h, uint32_t i, uint32_t j) {
  return (1ull << 63) | ((h >> 45) << 44) | (uint64_t(i) << kIdxBits) | uint64_t(j);
}

template <int KT>
__device__ __forceinline__ void pair_key(const uint64_t* __restrict__ X, uint64_t v,
                                         uint64_t (&k)[KT]) {
  const uint64_t* a = X + ((v >> kIdxBits) & kIdxMask) * KT;
  const uint64_t* b = X + (v & kIdxMask) * KT;
#pragma unroll
  for (int w = 0; w < KT; ++w) k[w] = __ldg(a + w) & __ldg(b + w);
}

// Returns 1 if inserted, 0 if already present, -1 if no reservation was
// granted (the band is recorded for replay).
template <int KT>
__device__ int table_insert(const PairTable& t, const uint64_t* __restrict__ X,
                            const uint64_t (&b)[KT], uint64_t h, uint32_t i, uint32_t j,
                            int band, int* status) {
  const uint64_t val = slot_value(h, i, j);
  uint64_t slot = h & t.mask;
  bool reserved = false;
  for (uint64_t probe = 0; probe <= t.mask; ++probe) {
    unsigned long long cur = ld_relaxed_u64(t.slots + slot);
    if (cur == 0ull) {
      if (!reserved) {
        if (atomicAdd(t.reserved, 1ull) >= t.limit) {
          atomicMin(t.failed_band, band);
          return -1;
        }
        reserved = true;
      }
      cur = atomicCAS(reinterpret_cast<unsigned long long*>(t.slots + slot), 0ull,
                      (unsigned long long)val);
      if (cur == 0ull) {
        atomicAdd(t.count, 1ull);
        return 1;
      }
    }
    if ((cur & kFpMask) == (val & kFpMask)) {
      uint64_t k2[KT];
      pair_key<KT>(X, cur, k2);
      bool same = true;
#pragma unroll
      for (int w = 0; w < KT; ++w) same &= (k2[w] == b[w]);
      if (same) {
        if (reserved) atomicAdd(t.reserved, ~0ull);  // give the reservation back
        return 0;
      }
    }
    slot = (slot + 1) & t.mask;
  }
  set_status(status, ST_TABLE_FULL);
  return -1;
}

constexpr int kPairThreads = 256;

// Grid: x = column tile bj, y = row tile bi - band_lo.  Tiles with bj < bi
// lie below the diagonal and exit at once.  Shared rows use an odd stride of
// KT + 1 words so that lanes reading consecutive rows hit distinct banks.
template <int KT>
__global__ void __launch_bounds__(kPairThreads)
    pair_insert_kernel(const uint64_t* __restrict__ X, int64_t n, int64_t band_lo,
                       PairTable t, int* status) {
  constexpr int T = kPairTile;
  constexpr int SKT = KT + 1;
  __shared__ uint64_t A[T * SKT];
  __shared__ uint64_t B[T * SKT];
  const int64_t bi = band_lo + blockIdx.y, bj = blockIdx.x;
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
    table_insert<KT>(t, X, b, h, uint32_t(i0 + i), uint32_t(j0 + j), int(bi), status);
  }
}

template <int KT>
__global__ void rehash_kernel(const uint64_t* __restrict__ X, const uint64_t* __restrict__ from,
                              uint64_t from_cap, PairTable to, int* status) {
  int64_t s = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (s >= int64_t(from_cap)) return;
  const uint64_t v = from[s];
  if (v == 0ull) return;
  uint64_t b[KT];
  pair_key<KT>(X, v, b);
  table_insert<KT>(to, X, b, hash_key<KT>(b), uint32_t((v >> kIdxBits) & kIdxMask),
                   uint32_t(v & kIdxMask), 0, status);
}

// Warp-aggregated append of every stored key, recomputed from its pair.
template <int KT>
__global__ void compact_kernel(const uint64_t* __restrict__ X, const uint64_t* __restrict__ slots,
                               uint64_t cap, uint64_t* __restrict__ out,
                               unsigned long long* out_count) {
  const int lane = threadIdx.x & 31;
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  for (int64_t base = int64_t(blockIdx.x) * blockDim.x + (threadIdx.x & ~31);
       base < int64_t(cap); base += stride) {
    int64_t s = base + lane;
    const uint64_t v = s < int64_t(cap) ? slots[s] : 0ull;
    unsigned m = __ballot_sync(0xffffffffu, v != 0ull);
    if (m == 0) continue;
    unsigned long long pos0 = 0;
    if (lane == 0) pos0 = atomicAdd(out_count, (unsigned long long)__popc(m));
    pos0 = __shfl_sync(0xffffffffu, pos0, 0);
    if (v != 0ull) {
      uint64_t pos = pos0 + __popc(m & ((1u << lane) - 1u));
      uint64_t b[KT];
      pair_key<KT>(X, v, b);
#pragma unroll
      for (int k = 0; k < KT; ++k) out[pos * KT + k] = b[k];
    }
  }
}

cudaError_t launch_pair_insert(const uint64_t* X, int64_t n, int KT, int64_t band_lo,
                               PairTable t, int* status, cudaStream_t s) {
  int64_t nt = ceil_div(n, kPairTile);
  if (band_lo >= nt) return cudaSuccess;
  dim3 grid{unsigned(nt), unsigned(nt - band_lo), 1u};
  IG_DISPATCH_KT(KT, (pair_insert_kernel<KTC><<<grid, kPairThreads, 0, s>>>(X, n, band_lo, t,
                                                                             status)));
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_rehash(const uint64_t* X, const uint64_t* from, uint64_t from_cap,
                          PairTable to, int KT, int* status, cudaStream_t s) {
  unsigned blocks = unsigned(ceil_div(int64_t(from_cap), 256));
  IG_DISPATCH_KT(KT, (rehash_kernel<KTC><<<blocks, 256, 0, s>>>(X, from, from_cap, to, status)));
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_compact(const uint64_t* X, const uint64_t* slots, uint64_t cap, int KT,
                           uint64_t* out, unsigned long long* out_count, cudaStream_t s) {
  int64_t blocks = ceil_div(int64_t(cap), 256);
  if (blocks > 8 * 1024) blocks = 8 * 1024;
  IG_DISPATCH_KT(KT, (compact_kernel<KTC><<<unsigned(blocks), 256, 0, s>>>(X, slots, cap, out,
                                                                            out_count)));
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace igk
