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
// Overflow cannot happen and every insert ends: an insert probes at most
// `max_probe` slots, and a pair tile that starts when the table already holds
// `limit` keys (half its capacity) inserts nothing.  Either way the tile's
// band is recorded; the host then grows the table, rehashes it, and replays
// the bands from the first failed one (inserts are idempotent).  Bounding the
// probe keeps lookups exact: slots are written once and never cleared, so a
// stored key sits within `max_probe` slots of its home, before any empty one.
//
// Warps count the keys they add in registers and add them to the table's
// count every few hundred keys at most (and their CTA once when it ends): a
// per-key atomic on one global counter would serialise every new key in one
// L2 slice.
#include <algorithm>
#include <atomic>

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

// A key held in registers (pair tiles), or given as the AND of two rows of
// global memory and read word by word where it is needed (rehash).
template <int KT>
struct RegKey {
  const uint64_t (&w)[KT];
  __device__ __forceinline__ uint64_t operator()(int k) const { return w[k]; }
};
struct GlobalPairKey {
  const uint64_t* a;
  const uint64_t* b;
  __device__ __forceinline__ uint64_t operator()(int w) const {
    return __ldg(a + w) & __ldg(b + w);
  }
};

// Returns 1 if inserted, 0 if already present, -1 if no reservation was
// granted (the band is recorded for replay).
template <int KT, class Key>
__device__ int table_insert(const PairTable& t, const uint64_t* __restrict__ X, const Key& key,
                            uint64_t h, uint32_t i, uint32_t j, int band, int* status) {
  const uint64_t val = slot_value(h, i, j);
  uint64_t slot = h & t.mask;
  for (uint64_t probe = 0; probe < t.max_probe; ++probe) {
    unsigned long long cur = ld_relaxed_u64(t.slots + slot);
    if (cur == 0ull) {
      cur = atomicCAS(reinterpret_cast<unsigned long long*>(t.slots + slot), 0ull,
                      (unsigned long long)val);
      if (cur == 0ull) return 1;
    }
    if ((cur & kFpMask) == (val & kFpMask)) {
      const uint64_t* ca = X + ((cur >> kIdxBits) & kIdxMask) * KT;
      const uint64_t* cb = X + (cur & kIdxMask) * KT;
      bool same = true;
      if constexpr (KT >= 2) {
        // Rows of KT >= 2 words are 16-byte aligned: two words per load.
#pragma unroll
        for (int w = 0; w < KT; w += 2) {
          const ulonglong2 va = __ldg(reinterpret_cast<const ulonglong2*>(ca + w));
          const ulonglong2 vb = __ldg(reinterpret_cast<const ulonglong2*>(cb + w));
          same &= ((va.x & vb.x) == key(w)) & ((va.y & vb.y) == key(w + 1));
        }
      } else {
        same = (__ldg(ca) & __ldg(cb)) == key(0);
      }
      if (same) return 0;
    }
    slot = (slot + 1) & t.mask;
  }
  if (t.max_probe > t.mask) set_status(status, ST_TABLE_FULL);  // every slot taken
  atomicMin(t.failed_band, band);
  return -1;
}

constexpr int kPairThreads = 256;

// Grid: x = column tile bj, y = row tile bi - band_lo.  Tiles with bj < bi
// lie below the diagonal and exit at once.  Shared rows use an odd stride of
// KT + 1 words so that lanes reading consecutive rows hit distinct banks.
// Each thread forms its intersection once in registers (about 64 in all);
// more resident CTAs would not help anyway, since their shared memory comes
// out of the L1 that caches the class's records, which every key comparison
// reads.
//
// Overflow is watched during the tile, not only at its start: warps add
// their new keys to the table's count every `t.flush` keys, and a warp whose
// addition takes the count to the limit records its band and stops its
// whole tile (its band is replayed on the grown table).  Every warp that
// adds keys learns of the overflow at its next addition, so inserts stop
// within one flush interval; without the watch, tiles that started before
// the table filled kept inserting into an ever fuller table, every insert
// probing up to max_probe slots.  (Polling the count instead cost 0.1-0.4 ms
// per 148k fit: the poll's latency on that one hot line stalled its warp.)
template <int KT>
struct PairSmem {
  uint64_t A[kPairTile * (KT + 1)];
  uint64_t B[kPairTile * (KT + 1)];
  unsigned int n_new;
  int table_full;
  volatile int stop_tile;
};

// One pair tile (bi, bj), bj >= bi, of the records X[0, n): run by the whole
// CTA, which may run several in turn (the shared state is reset here).
template <int KT>
__device__ __forceinline__ void pair_tile(const uint64_t* __restrict__ X, int64_t n, int64_t bi,
                                          int64_t bj, const PairTable& t, int* status,
                                          PairSmem<KT>& sm) {
  constexpr int T = kPairTile;
  constexpr int SKT = KT + 1;
  uint64_t* const A = sm.A;
  uint64_t* const B = sm.B;
  __syncthreads();  // every thread is done with the previous tile's state
  if (threadIdx.x == 0) {
    sm.n_new = 0;
    sm.stop_tile = 0;
    sm.table_full = ld_relaxed_u64(reinterpret_cast<const uint64_t*>(t.count)) >= t.limit;
  }
  const int64_t i0 = bi * T, j0 = bj * T;
  for (int e = threadIdx.x; e < T * KT; e += kPairThreads) {
    int r = e / KT, k = e - r * KT;
    A[r * SKT + k] = (i0 + r < n) ? X[(i0 + r) * KT + k] : 0ull;
    B[r * SKT + k] = (j0 + r < n) ? X[(j0 + r) * KT + k] : 0ull;
  }
  __syncthreads();
  if (sm.table_full) {  // uniform: the whole tile waits for the grown table
    if (threadIdx.x == 0) atomicMin(t.failed_band, int(bi));
    return;
  }
  const int lane = threadIdx.x & 31;
  unsigned int wnew = 0;  // keys this warp added and has not yet counted (same in every lane)
  for (int p = threadIdx.x; p < T * T; p += kPairThreads) {
    const int i = p / T, j = p - (p / T) * T;
    const bool valid = (i0 + i < n) && (j0 + j < n) && (bi < bj || i <= j);
    uint64_t kw[KT];
    uint64_t any = 0;
    uint64_t h = hash_begin();
#pragma unroll
    for (int k = 0; k < KT; ++k) {
      kw[k] = A[i * SKT + k] & B[j * SKT + k];
      any |= kw[k];
      h = hash_word(h, kw[k]);
    }
    h = hash_end(h);
    bool pending = valid && any != 0;
    const unsigned active = __ballot_sync(0xffffffffu, pending);
    if (pending) {
      // Lanes holding the same key insert it once: the lowest lane of each
      // group of equal hashes is its leader; a lane whose key equals its
      // leader's skips the insert.  Most hashes are unique in the warp, and
      // those lanes skip the compare.
      const unsigned peers = __match_any_sync(active, h);
      if (__popc(peers) > 1) {
        const int leader = __ffs(peers) - 1;
        bool same = true;
#pragma unroll
        for (int k = 0; k < KT; ++k) same &= (__shfl_sync(peers, kw[k], leader) == kw[k]);
        if (leader != lane && same) pending = false;
      }
    }
    bool added = false;
    if (pending)
      added = table_insert<KT>(t, X, RegKey<KT>{kw}, h, uint32_t(i0 + i), uint32_t(j0 + j),
                               int(bi), status) == 1;
    wnew += unsigned(__popc(__ballot_sync(0xffffffffu, added)));
    if (t.flush && wnew >= t.flush) {
      if (lane == 0) {
        const unsigned long long before = atomicAdd(t.count, (unsigned long long)wnew);
        if (before + wnew >= t.limit) {
          atomicMin(t.failed_band, int(bi));
          sm.stop_tile = 1;
        }
      }
      wnew = 0;
    }
    if (__shfl_sync(0xffffffffu, lane == 0 ? sm.stop_tile : 0, 0)) break;
  }
  if (lane == 0 && wnew) atomicAdd(&sm.n_new, wnew);
  __syncthreads();
  if (threadIdx.x == 0 && sm.n_new != 0) atomicAdd(t.count, (unsigned long long)sm.n_new);
}

template <int KT>
__global__ void __launch_bounds__(kPairThreads)
    pair_insert_kernel(const uint64_t* __restrict__ X, int64_t n, int64_t band_lo,
                       PairTable t, int* status, const unsigned long long* __restrict__ n_dev) {
  __shared__ PairSmem<KT> sm;
  if (n_dev && int64_t(*n_dev) < n) n = int64_t(*n_dev);
  const int64_t bi = band_lo + blockIdx.y, bj = blockIdx.x;
  if (bj < bi || bj * kPairTile >= n) return;
  pair_tile<KT>(X, n, bi, bj, t, status, sm);
}

// Many tables in one launch (independent problems and classes, of any word
// count): a persistent grid takes pair tiles from one device-side queue,
// the tiles of job j numbered [tile_off[j], tile_off[j + 1]) band by band
// from the job's band_lo.  Each CTA draws its next tile with one atomic, so
// large and small jobs share the SMs without a launch per job; a tile runs
// the code of its job's word count in shared memory sized for the largest.
union PairSmemAny {
  PairSmem<1> k1;
  PairSmem<2> k2;
  PairSmem<4> k4;
  PairSmem<8> k8;
  PairSmem<16> k16;
};

__global__ void __launch_bounds__(kPairThreads, 4)
    pair_insert_multi_kernel(const PairJob* __restrict__ jobs, int n_jobs,
                             const int64_t* __restrict__ tile_off,
                             unsigned long long* next_tile, int* status) {
  __shared__ PairSmemAny sm;
  __shared__ int64_t tile[3];  // job, bi, bj
  __shared__ PairJob job;      // the current tile's job (read from here, not held in registers)
  const int64_t total = tile_off[n_jobs];
  for (;;) {
    if (threadIdx.x == 0) {
      const int64_t q = int64_t(atomicAdd(next_tile, 1ull));
      tile[0] = -1;
      if (q < total) {
        // The job holding tile q, then its band: band b of a job with nt
        // tile rows starts after sum_{x = band_lo}^{b - 1} (nt - x) tiles.
        int lo = 0, hi = n_jobs - 1;
        while (lo < hi) {
          const int mid = (lo + hi + 1) >> 1;
          if (tile_off[mid] <= q) lo = mid; else hi = mid - 1;
        }
        const PairJob& jb = jobs[lo];
        const int64_t nt = ceil_div(jb.n, kPairTile), b0 = jb.band_lo;
        const int64_t r = q - tile_off[lo];
        auto before = [&](int64_t b) {  // tiles of the bands [b0, b)
          return (b - b0) * nt - (b * (b - 1) / 2 - b0 * (b0 - 1) / 2);
        };
        int64_t blo = b0, bhi = nt - 1;
        while (blo < bhi) {
          const int64_t mid = (blo + bhi + 1) >> 1;
          if (before(mid) <= r) blo = mid; else bhi = mid - 1;
        }
        job = jb;
        tile[0] = lo;
        tile[1] = blo;
        tile[2] = blo + (r - before(blo));
      }
    }
    __syncthreads();
    const int64_t j = tile[0], bi = tile[1], bj = tile[2];
    if (j < 0) break;
    switch (job.KT) {  // uniform
      case 1: pair_tile<1>(job.X, job.n, bi, bj, job.t, status, sm.k1); break;
      case 2: pair_tile<2>(job.X, job.n, bi, bj, job.t, status, sm.k2); break;
      case 4: pair_tile<4>(job.X, job.n, bi, bj, job.t, status, sm.k4); break;
      case 8: pair_tile<8>(job.X, job.n, bi, bj, job.t, status, sm.k8); break;
      default: pair_tile<16>(job.X, job.n, bi, bj, job.t, status, sm.k16); break;
    }
  }
}

template <int KT>
__global__ void rehash_kernel(const uint64_t* __restrict__ X, const uint64_t* __restrict__ from,
                              uint64_t from_cap, PairTable to, int* status) {
  __shared__ unsigned int n_new;
  if (threadIdx.x == 0) n_new = 0;
  __syncthreads();
  const int64_t s = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  const uint64_t v = s < int64_t(from_cap) ? from[s] : 0ull;
  if (v != 0ull) {
    uint64_t b[KT];
    pair_key<KT>(X, v, b);
    const GlobalPairKey key{X + ((v >> kIdxBits) & kIdxMask) * KT, X + (v & kIdxMask) * KT};
    if (table_insert<KT>(to, X, key, hash_key<KT>(b), uint32_t((v >> kIdxBits) & kIdxMask),
                         uint32_t(v & kIdxMask), 0, status) == 1)
      atomicAdd(&n_new, 1u);
  }
  __syncthreads();
  if (threadIdx.x == 0 && n_new != 0) atomicAdd(to.count, (unsigned long long)n_new);
}

// Appends every stored key, recomputed from its pair.  Each block takes a
// contiguous range of slots: it first counts the stored keys there and
// reserves room for them with one atomic on the global count, then places
// them through a shared-memory cursor -- one global atomic per block rather
// than per warp, all on one address.  (The order of the output does not
// matter: it is sorted into canonical order later.)
constexpr int kCompactThreads = 256;
template <int KT>
__global__ void __launch_bounds__(kCompactThreads)
    compact_kernel(const uint64_t* __restrict__ X, const uint64_t* __restrict__ slots,
                   uint64_t cap, uint64_t* __restrict__ out, int64_t out_rows,
                   unsigned long long* out_count, int* status) {
  __shared__ unsigned int blk_count, blk_cursor;
  __shared__ unsigned long long blk_base;
  const int lane = threadIdx.x & 31;
  const int64_t per = ((int64_t(cap) + gridDim.x - 1) / gridDim.x + 31) & ~int64_t(31);
  const int64_t lo = int64_t(blockIdx.x) * per;
  const int64_t hi = lo + per < int64_t(cap) ? lo + per : int64_t(cap);
  if (threadIdx.x == 0) {
    blk_count = 0;
    blk_cursor = 0;
  }
  __syncthreads();
  unsigned int mine = 0;
  for (int64_t s = lo + threadIdx.x; s < hi; s += blockDim.x) mine += slots[s] != 0ull ? 1u : 0u;
#pragma unroll
  for (int o = 16; o; o >>= 1) mine += __shfl_xor_sync(0xffffffffu, mine, o);
  if (lane == 0 && mine) atomicAdd(&blk_count, mine);
  __syncthreads();
  if (threadIdx.x == 0) blk_base = blk_count ? atomicAdd(out_count, (unsigned long long)blk_count) : 0ull;
  __syncthreads();
  // The stored pairs of each 32-slot step are expanded by the whole warp,
  // 32 / KT keys per instruction with consecutive lanes on consecutive words.
  __shared__ uint64_t kept_v[kCompactThreads];
  uint64_t* my_kept = kept_v + (threadIdx.x & ~31);
  constexpr int kRowsPer = 32 / KT;
  const int sub = lane / KT, word = lane % KT;
  for (int64_t base = lo + (threadIdx.x & ~31); base < hi; base += blockDim.x) {
    const int64_t s = base + lane;
    const uint64_t v = s < hi ? slots[s] : 0ull;
    const unsigned m = __ballot_sync(0xffffffffu, v != 0ull);
    if (m == 0) continue;
    unsigned int p0 = 0;
    if (lane == 0) p0 = atomicAdd(&blk_cursor, unsigned(__popc(m)));
    p0 = __shfl_sync(0xffffffffu, p0, 0);
    if (v != 0ull) my_kept[__popc(m & ((1u << lane) - 1u))] = v;
    __syncwarp();
    const int nk = __popc(m);
    for (int b = sub; b < nk; b += kRowsPer) {
      const uint64_t pos = blk_base + p0 + unsigned(b);
      if (pos >= uint64_t(out_rows)) {
        set_status(status, ST_COUNT);
        continue;
      }
      const uint64_t kv = my_kept[b];
      out[pos * KT + word] = __ldg(X + ((kv >> kIdxBits) & kIdxMask) * KT + word) &
                             __ldg(X + (kv & kIdxMask) * KT + word);
    }
    __syncwarp();
  }
}

// Marks the repeated rows of X[0, n): rows are put in an open-addressing
// table of row indices (cap > n slots, all 0xffffffff) by content; the row
// that claims a content's slot represents it (flag 0) and every other row
// with that content is flagged 1.  The table is never full, so every probe
// ends within cap slots.
template <int KT>
__global__ void mark_repeats_kernel(const uint64_t* __restrict__ X, int64_t n,
                                    uint32_t* __restrict__ table, uint64_t mask,
                                    uint32_t* __restrict__ flag) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  uint64_t w[KT];
#pragma unroll
  for (int k = 0; k < KT; ++k) w[k] = X[i * KT + k];
  uint64_t slot = hash_key<KT>(w) & mask;
  for (uint64_t probe = 0; probe <= mask; ++probe) {
    uint32_t cur = table[slot];
    if (cur == 0xffffffffu) {
      cur = atomicCAS(table + slot, 0xffffffffu, uint32_t(i));
      if (cur == 0xffffffffu) {
        flag[i] = 0u;
        return;
      }
    }
    bool same = true;
#pragma unroll
    for (int k = 0; k < KT; ++k) same &= X[int64_t(cur) * KT + k] == w[k];
    if (same) {
      flag[i] = 1u;
      return;
    }
    slot = (slot + 1) & mask;
  }
}

cudaError_t launch_mark_repeats(const uint64_t* X, int64_t n, int KT, uint32_t* table,
                                uint64_t cap, uint32_t* flag, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  if (cap <= uint64_t(n) || (cap & (cap - 1)) != 0) return cudaErrorInvalidValue;
  IG_DISPATCH_KT(KT, (mark_repeats_kernel<KTC><<<unsigned(ceil_div(n, 256)), 256, 0, s>>>(
                         X, n, table, cap - 1, flag)));
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_pair_insert(const uint64_t* X, int64_t n, int KT, int64_t band_lo,
                               PairTable t, int* status, cudaStream_t s,
                               const unsigned long long* n_dev) {
  int64_t nt = ceil_div(n, kPairTile);
  if (band_lo >= nt) return cudaSuccess;
  dim3 grid{unsigned(nt), unsigned(nt - band_lo), 1u};
  // Warps count their new keys into the table every `flush` keys, often
  // enough that the count lags the table by at most about a quarter of the
  // limit over all warps in flight (at most 8 CTAs of 8 warps per SM).
  const int64_t tiles = (nt - band_lo) * (nt - band_lo + 1) / 2;
  const int64_t warps = std::min<int64_t>(tiles, int64_t(num_sms()) * 8) * (kPairThreads / 32);
  t.flush = uint32_t(std::max<int64_t>(1, std::min<int64_t>(256, int64_t(t.limit) / (4 * warps))));
  IG_DISPATCH_KT(KT, (pair_insert_kernel<KTC><<<grid, kPairThreads, 0, s>>>(X, n, band_lo, t,
                                                                             status, n_dev)));
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_pair_insert_multi(const PairJob* jobs, int n_jobs, const int64_t* tile_off,
                                     unsigned long long* next_tile, int* status, cudaStream_t s) {
  if (n_jobs <= 0) return cudaSuccess;
  pair_insert_multi_kernel<<<unsigned(pair_multi_grid_warps() / (kPairThreads / 32)),
                             kPairThreads, 0, s>>>(jobs, n_jobs, tile_off, next_tile, status);
  count_launches(1);
  return cudaGetLastError();
}

int pair_multi_grid_warps() {
  static std::atomic<int> per_sm{0};
  int v = per_sm.load(std::memory_order_relaxed);
  if (v == 0) {
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, pair_insert_multi_kernel, kPairThreads,
                                                      0) != cudaSuccess ||
        v < 1)
      v = 1;
    per_sm.store(v, std::memory_order_relaxed);
  }
  return v * num_sms() * (kPairThreads / 32);
}

cudaError_t launch_rehash(const uint64_t* X, const uint64_t* from, uint64_t from_cap,
                          PairTable to, int KT, int* status, cudaStream_t s) {
  unsigned blocks = unsigned(ceil_div(int64_t(from_cap), 256));
  IG_DISPATCH_KT(KT, (rehash_kernel<KTC><<<blocks, 256, 0, s>>>(X, from, from_cap, to, status)));
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_compact(const uint64_t* X, const uint64_t* slots, uint64_t cap, int KT,
                           uint64_t* out, int64_t out_rows, unsigned long long* out_count,
                           int* status, cudaStream_t s) {
  // Ranges of at least 4,096 slots, at most 16 blocks per SM.
  int64_t blocks = ceil_div(int64_t(cap), 4096);
  if (blocks > int64_t(num_sms()) * 16) blocks = int64_t(num_sms()) * 16;
  if (blocks < 1) blocks = 1;
  IG_DISPATCH_KT(KT, (compact_kernel<KTC><<<unsigned(blocks), kCompactThreads, 0, s>>>(
                         X, slots, cap, out, out_rows, out_count, status)));
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace igk
