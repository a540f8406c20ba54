// Subset tests with an item index (exact pruning of Eq. 3, Eq. 2 and Eq. 4).
//
// p is inside r only if r contains every item of p, in particular the item
// k(p) of p that the fewest records contain.  So instead of testing every
// (pattern, record) pair:
//   * the records ("multi" side) are filed under every item they contain:
//     group l holds a copy of each record with item l;
//   * the patterns ("keyed" side) are filed under their key item k(p), the
//     item of p with the smallest record count (lowest item on ties); a
//     pattern with an item no record contains is filed in the extra group L
//     and needs no test at all (it is inside no record);
//   * group l's patterns are tested only against group l's records, as dense
//     blocks of the integer-pipe kernel.
// Every (pattern, record) pair with p inside r is met exactly once (in group
// k(p)), and no pair outside a common group can have p inside r, so counts,
// flags and score sums are the same as from the full product.
//
// Work items are (group, own tile, stream range) blocks.  For the integer
// grouped kernel here the host builds the list from the group sizes (read
// back) and balances the stream ranges across the GPU; the tensor-core form
// builds its items on the device (subset_tc.cu).
#include <algorithm>
#include <vector>

#include "common.cuh"
#include "internal.h"

namespace igk {

// ---- building the groups ------------------------------------------------------

// freq[l] += number of rows containing item l.
__global__ void item_histogram_kernel(const uint64_t* __restrict__ rows, int64_t n, int stride,
                                      int K, int L, uint32_t* __restrict__ freq) {
  extern __shared__ uint32_t h[];
  for (int l = threadIdx.x; l < L; l += blockDim.x) h[l] = 0;
  __syncthreads();
  const int64_t step = int64_t(gridDim.x) * blockDim.x;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += step)
    for (int k = 0; k < K; ++k) {
      uint64_t w = rows[i * stride + k];
      while (w) {
        const int b = __ffsll(static_cast<long long>(w)) - 1;
        w &= w - 1;
        atomicAdd(&h[k * 64 + b], 1u);
      }
    }
  __syncthreads();
  for (int l = threadIdx.x; l < L; l += blockDim.x)
    if (h[l]) atomicAdd(freq + l, h[l]);
}

// Exclusive scan of cnt[0..len) into off[0..len] (off[len] = total), one block.
__global__ void small_scan_kernel(const uint32_t* __restrict__ cnt, int len,
                                  uint32_t* __restrict__ off) {
  __shared__ uint32_t part[1024];
  const int chunk = (len + 1023) / 1024;
  const int lo = threadIdx.x * chunk, hi = min(len, lo + chunk);
  uint32_t s = 0;
  for (int i = lo; i < hi; ++i) s += cnt[i];
  part[threadIdx.x] = s;
  __syncthreads();
  for (int d = 1; d < 1024; d <<= 1) {
    uint32_t v = threadIdx.x >= d ? part[threadIdx.x - d] : 0u;
    __syncthreads();
    part[threadIdx.x] += v;
    __syncthreads();
  }
  uint32_t run = part[threadIdx.x] - s;
  for (int i = lo; i < hi; ++i) {
    off[i] = run;
    run += cnt[i];
  }
  if (threadIdx.x == 1023) off[len] = part[1023];
}

// Writes the rows of one round of copies for a warp: lane j of the warp
// has a copy to place (has) at row pos of out, with the contents of its
// record, staged in shared memory at rec + (rec0 + j) * KT.  The warp writes
// 32 / KT rows per store, each row as KT consecutive 8-byte words, so a
// store covers whole rows instead of one word of 32 scattered rows.
__device__ __forceinline__ void warp_write_rows(const uint64_t* rec, int rec0, int KT,
                                                bool has, uint32_t pos,
                                                uint64_t* __restrict__ out) {
  const int lane = threadIdx.x & 31;
  const int per = 32 / KT;
  const int wr = lane / KT, ww = lane - wr * KT;
  for (int r0 = 0; r0 < 32; r0 += per) {
    const int src = r0 + wr;
    const uint32_t p = __shfl_sync(0xffffffffu, pos, src);
    const int h = __shfl_sync(0xffffffffu, has ? 1 : 0, src);
    if (h) out[int64_t(p) * KT + ww] = rec[(rec0 + src) * KT + ww];
  }
}

// Stages rows [i0, i0 + blockDim.x) (K words each, zero words up to KT) in
// shared memory.
__device__ __forceinline__ void stage_rows(const uint64_t* __restrict__ rows, int64_t n,
                                           int stride, int K, int KT, int64_t i0,
                                           uint64_t* rec) {
  const int nb = blockDim.x;
  for (int e = threadIdx.x; e < nb * KT; e += nb) {
    const int r = e / KT, q = e - r * KT;
    rec[e] = (i0 + r < n && q < K) ? rows[(i0 + r) * stride + q] : 0ull;
  }
}

// Copies row i into the group of every item it contains, one warp per row:
// the lanes test the row's item positions 32 at a time, each set position
// takes a slot in its group, and the warp writes the row to those slots as
// whole rows (32 / KT rows per store).  A block first counts its copies per
// item in shared memory and reserves one range per item in the group with a
// single global atomic, so the slots come from shared-memory atomics (the
// order inside a group does not matter).  Shared memory: one staged row per
// warp, then 2 * L counters.
__global__ void multi_scatter_kernel(const uint64_t* __restrict__ rows, int64_t n, int stride,
                                     int K, int KT, int L, const uint32_t* __restrict__ off,
                                     uint32_t* __restrict__ cursor, uint64_t* __restrict__ out,
                                     uint32_t* __restrict__ ids,
                                     const uint32_t* __restrict__ id_map) {
  extern __shared__ uint64_t shm[];
  const int warps = int(blockDim.x >> 5);
  const int warp = int(threadIdx.x >> 5), lane = int(threadIdx.x & 31);
  uint64_t* rec = shm;                                             // [warps][KT]
  uint32_t* cnt = reinterpret_cast<uint32_t*>(rec + warps * KT);  // [L]
  uint32_t* base = cnt + L;                                        // [L]
  const int64_t r0 = int64_t(blockIdx.x) * warps;
  for (int e = threadIdx.x; e < warps * KT; e += blockDim.x) {
    const int r = e / KT, q = e - r * KT;
    rec[e] = (r0 + r < n && q < K) ? rows[(r0 + r) * stride + q] : 0ull;
  }
  for (int l = threadIdx.x; l < L; l += blockDim.x) cnt[l] = 0;
  __syncthreads();
  const uint64_t* my = rec + warp * KT;
  for (int l = lane; l < L; l += 32)
    if ((my[l >> 6] >> (l & 63)) & 1ull) atomicAdd(&cnt[l], 1u);
  __syncthreads();
  for (int l = threadIdx.x; l < L; l += blockDim.x) {
    const uint32_t c = cnt[l];
    base[l] = c ? off[l] + atomicAdd(cursor + l, c) : 0u;
    cnt[l] = 0;
  }
  __syncthreads();
  const int64_t i = r0 + warp;
  const uint32_t my_id = i < n ? (id_map ? id_map[i] : uint32_t(i)) : 0u;
  const int per = 32 / KT;                   // rows per store
  const int g = lane / KT, ww = lane - g * KT;  // this lane writes word ww of the g-th row
  for (int l0 = 0; l0 < L; l0 += 32) {
    const int l = l0 + lane;
    const bool has = l < L && ((my[l >> 6] >> (l & 63)) & 1ull);
    uint32_t pos = 0;
    if (has) {
      pos = base[l] + atomicAdd(&cnt[l], 1u);
      ids[pos] = my_id;
    }
    unsigned m = __ballot_sync(0xffffffffu, has);
    while (m) {
      unsigned b = m;
      for (int k = 0; k < g && b; ++k) b &= b - 1u;  // the g-th set lane of m
      const int src = b ? __ffs(int(b)) - 1 : 0;
      const uint32_t p = __shfl_sync(0xffffffffu, pos, src);
      if (b) out[int64_t(p) * KT + ww] = my[ww];
      for (int k = 0; k < per && m; ++k) m &= m - 1u;
    }
  }
}

// key[i] = the item of row i with the smallest freq (lowest item on ties),
// or L when one of its items has freq 0 (or the row is empty); kcount[g]
// counts the rows keyed to g.  freq is read from a shared copy and the
// counts are aggregated per block: popular keys would otherwise take one
// global atomic per row on a few addresses.  Shared memory: 2 * L + 1
// counters.
__global__ void key_item_kernel(const uint64_t* __restrict__ rows, int64_t n, int stride, int K,
                                int L, const uint32_t* __restrict__ freq,
                                uint32_t* __restrict__ key, uint32_t* __restrict__ kcount,
                                const unsigned long long* __restrict__ n_dev) {
  extern __shared__ uint32_t shk[];
  if (n_dev && int64_t(*n_dev) < n) n = int64_t(*n_dev);
  uint32_t* f_s = shk;          // [L]
  uint32_t* c_s = shk + L;      // [L + 1]
  for (int l = threadIdx.x; l < L; l += blockDim.x) f_s[l] = freq[l];
  for (int l = threadIdx.x; l <= L; l += blockDim.x) c_s[l] = 0;
  __syncthreads();
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i < n) {
    uint32_t best = 0xffffffffu;
    int best_l = L;
    for (int k = 0; k < K; ++k) {
      uint64_t x = rows[i * stride + k];
      while (x) {
        const int b = __ffsll(static_cast<long long>(x)) - 1;
        x &= x - 1;
        const int l = k * 64 + b;
        const uint32_t f = f_s[l];
        if (f < best) {
          best = f;
          best_l = l;
        }
      }
    }
    if (best == 0u) best_l = L;
    key[i] = uint32_t(best_l);
    atomicAdd(&c_s[best_l], 1u);
  }
  __syncthreads();
  for (int l = threadIdx.x; l <= L; l += blockDim.x)
    if (c_s[l]) atomicAdd(kcount + l, c_s[l]);
}

// Files row i under its key (block-aggregated like multi_scatter_kernel;
// rows written whole by warp_write_rows).  Shared memory: blockDim.x * KT
// words of rows, then 2 * groups counters.
__global__ void keyed_scatter_kernel(const uint64_t* __restrict__ rows, int64_t n, int stride,
                                     int K, int KT, int groups, const uint32_t* __restrict__ key,
                                     const uint32_t* __restrict__ off,
                                     uint32_t* __restrict__ cursor, uint64_t* __restrict__ out,
                                     uint32_t* __restrict__ ids,
                                     const uint64_t* __restrict__ payload,
                                     uint64_t* __restrict__ payload_out,
                                     const unsigned long long* __restrict__ n_dev) {
  extern __shared__ uint64_t shm[];
  if (n_dev && int64_t(*n_dev) < n) n = int64_t(*n_dev);
  uint64_t* rec = shm;
  uint32_t* cnt = reinterpret_cast<uint32_t*>(rec + blockDim.x * KT);  // [groups]
  uint32_t* base = cnt + groups;                                       // [groups]
  const int64_t i0 = int64_t(blockIdx.x) * blockDim.x;
  stage_rows(rows, n, stride, K, KT, i0, rec);
  for (int l = threadIdx.x; l < groups; l += blockDim.x) cnt[l] = 0;
  __syncthreads();
  const int64_t i = i0 + threadIdx.x;
  const bool valid = i < n;
  const uint32_t l = valid ? key[i] : 0u;
  if (valid) atomicAdd(&cnt[l], 1u);
  __syncthreads();
  for (int g = threadIdx.x; g < groups; g += blockDim.x) {
    const uint32_t c = cnt[g];
    base[g] = c ? off[g] + atomicAdd(cursor + g, c) : 0u;
    cnt[g] = 0;
  }
  __syncthreads();
  uint32_t pos = 0;
  if (valid) {
    pos = base[l] + atomicAdd(&cnt[l], 1u);
    ids[pos] = uint32_t(i);
    if (payload) payload_out[pos] = payload[i];
  }
  warp_write_rows(rec, threadIdx.x & ~31, KT, valid, pos, out);
}

// Threads per block of the scatter kernels: small inputs use narrow blocks
// so that they still spread over the SMs.
static int scatter_threads(int64_t n) {
  return n >= int64_t(num_sms()) * 4 * 256 ? 256 : (n >= int64_t(num_sms()) * 4 * 64 ? 64 : 32);
}

// ---- the grouped subset kernel ------------------------------------------------

constexpr int kGThreads = 256;
constexpr int kGStages = 3;

template <int KT>
struct GShape {
  static constexpr int TR = (8192 / (KT * 8)) > 256 ? 256 : (8192 / (KT * 8));
  static constexpr int Q = KT >= 16 ? 2 : 4;
  static constexpr int H = 2 * KT;
};

struct GroupedParams {
  const WorkItem* items;
  const uint64_t* keyed;        // patterns, grouped by key (stride KT, padded)
  const uint32_t* keyed_ids;    // original pattern of each grouped row
  const uint64_t* keyed_score;  // MODE_SUM: S of each grouped pattern (padded)
  const uint64_t* multi;        // record copies, grouped by item (stride KT, padded)
  const uint32_t* multi_ids;    // original record of each copy
  uint32_t* out_u32;            // ANY / COUNT: per pattern
  unsigned long long* out_u64;  // SUM: per record
  int* status;
};

// One work item: the rows [own_begin, +own_count) of one side of a group sit
// in registers (Q per thread), the rows [str_begin, +str_count) of the other
// side stream through shared memory.  The side in registers is the larger
// one, so that the lanes are busy.  When it is the side the result belongs
// to (patterns for ANY / COUNT, records for SUM) the result accumulates in
// registers; otherwise every hit updates the streamed row's result directly
// (atomics: hits are few).
template <int KT, int MODE, int Q>
__device__ __forceinline__ void grouped_body(const GroupedParams& p, const WorkItem& wi,
                                             uint8_t* smem) {
  using S = GShape<KT>;
  constexpr int TR = S::TR, H = S::H;
  constexpr uint32_t kRowBytes = TR * KT * 8;
  uint64_t* rows_s = reinterpret_cast<uint64_t*>(smem);
  uint64_t* bars = rows_s + kGStages * TR * KT;

  const bool own_keyed = wi.own_keyed != 0;
  // Results stay in registers when the own side is the result side.
  const bool own_result = (MODE == MODE_SUM) ? !own_keyed : own_keyed;
  const uint64_t* own_rows = own_keyed ? p.keyed : p.multi;
  const uint64_t* str_rows = own_keyed ? p.multi : p.keyed;
  const uint32_t* str_ids = own_keyed ? p.multi_ids : p.keyed_ids;

  uint32_t own[Q][H];
  bool valid[Q];
  // warp_rows[q]: some lane of this warp holds own row q (warp-uniform; the
  // rows of a block fill q = 0 first, so these form a prefix).  A warp skips
  // the tests of a q that none of its lanes holds.
  bool warp_rows[Q];
  unsigned long long own_score[Q];
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    const int64_t r = int64_t(q) * kGThreads + threadIdx.x;
    valid[q] = r < wi.own_count;
    warp_rows[q] = int64_t(q) * kGThreads + (threadIdx.x & ~31u) < wi.own_count;
    const uint64_t* src = own_rows + (wi.own_begin + r) * KT;
#pragma unroll
    for (int k = 0; k < KT; ++k) {
      const uint64_t w = valid[q] ? src[k] : 0ull;
      own[q][2 * k] = uint32_t(w);
      own[q][2 * k + 1] = uint32_t(w >> 32);
    }
    own_score[q] = 0;
    if constexpr (MODE == MODE_SUM)
      if (valid[q] && own_keyed) own_score[q] = p.keyed_score[wi.own_begin + r];
  }
  // Stream tiles may start at any row: with KT >= 2 every row is 16-byte
  // aligned, as the bulk copy needs.
  const int64_t s_lo = wi.str_begin, s_hi = wi.str_begin + wi.str_count;
  const int64_t ntiles = ceil_div(s_hi - s_lo, TR);
  if (threadIdx.x == 0) {
    for (int st = 0; st < kGStages; ++st) mbar_init(bars + st, 1);
    fence_mbar_init();
  }
  __syncthreads();
  auto issue = [&](int64_t tile) {
    const int st = int(tile % kGStages);
    const int64_t r0 = s_lo + tile * TR;
    mbar_arrive_expect_tx(bars + st, kRowBytes);
    bulk_g2s(rows_s + st * TR * KT, str_rows + r0 * KT, kRowBytes, bars + st);
  };
  if (threadIdx.x == 0)
    for (int64_t t = 0; t < ntiles && t < kGStages; ++t) issue(t);

  bool cov[Q];
  uint32_t cnt[Q];
  unsigned long long sum[Q];
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    cov[q] = false;
    cnt[q] = 0;
    sum[q] = 0;
  }
  int64_t tile = 0;
  bool failed = false;
  for (; tile < ntiles; ++tile) {
    const int st = int(tile % kGStages);
    const bool ok = mbar_wait(bars + st, uint32_t((tile / kGStages) & 1), p.status);
    if (__syncthreads_or(!ok)) {
      failed = true;
      break;
    }
    const int64_t left = s_hi - (s_lo + tile * TR);
    const int nr = int(left < TR ? left : TR);
    const uint32_t* rs = reinterpret_cast<const uint32_t*>(rows_s + st * TR * KT);
    if (!warp_rows[0]) {
      // no own row in this warp: nothing to test
    } else if (own_keyed) {
      // pattern (own) inside record (streamed)?
#pragma unroll 2
      for (int r = 0; r < nr; ++r) {
        uint32_t rh[H];
#pragma unroll
        for (int v = 0; v < H / 4; ++v) {
          const uint4 x = reinterpret_cast<const uint4*>(rs + r * H)[v];
          rh[4 * v] = x.x;
          rh[4 * v + 1] = x.y;
          rh[4 * v + 2] = x.z;
          rh[4 * v + 3] = x.w;
        }
#pragma unroll
        for (int q = 0; q < Q; ++q) {
          if (!warp_rows[q]) break;
          uint32_t acc = 0;
#pragma unroll
          for (int h = 0; h < H; ++h) acc |= own[q][h] & ~rh[h];
          const bool hit = acc == 0u && valid[q];
          if constexpr (MODE == MODE_ANY) cov[q] |= hit;
          if constexpr (MODE == MODE_COUNT) cnt[q] += hit ? 1u : 0u;
          if constexpr (MODE == MODE_SUM) {
            if (hit) atomicAdd(p.out_u64 + str_ids[s_lo + tile * TR + r], own_score[q]);
          }
        }
      }
    } else {
      // pattern (streamed) inside record (own)?
#pragma unroll 2
      for (int r = 0; r < nr; ++r) {
        uint32_t rh[H];
#pragma unroll
        for (int v = 0; v < H / 4; ++v) {
          const uint4 x = reinterpret_cast<const uint4*>(rs + r * H)[v];
          rh[4 * v] = x.x;
          rh[4 * v + 1] = x.y;
          rh[4 * v + 2] = x.z;
          rh[4 * v + 3] = x.w;
        }
#pragma unroll
        for (int q = 0; q < Q; ++q) {
          if (!warp_rows[q]) break;
          uint32_t acc = 0;
#pragma unroll
          for (int h = 0; h < H; ++h) acc |= rh[h] & ~own[q][h];
          const bool hit = acc == 0u && valid[q];
          if constexpr (MODE == MODE_SUM) {
            if (hit) sum[q] += p.keyed_score[s_lo + tile * TR + r];
          } else {
            if (hit) {
              const uint32_t sid = str_ids[s_lo + tile * TR + r];
              if constexpr (MODE == MODE_ANY) p.out_u32[sid] = 1u;
              if constexpr (MODE == MODE_COUNT) atomicAdd(p.out_u32 + sid, 1u);
            }
          }
        }
      }
    }
    bool stop = false;
    if constexpr (MODE == MODE_ANY) {
      // Early exit once every pattern held in registers is covered.
      bool done = own_result;
#pragma unroll
      for (int q = 0; q < Q; ++q) done &= (cov[q] || !valid[q]);
      stop = __syncthreads_and(done) != 0;
    } else {
      __syncthreads();
    }
    if (stop) break;
    if (threadIdx.x == 0 && tile + kGStages < ntiles) issue(tile + kGStages);
  }
  if (threadIdx.x == 0 && tile < ntiles) {
    const int64_t first = failed ? tile : tile + 1;
    const int64_t end = (tile + kGStages < ntiles) ? tile + kGStages : ntiles;
    for (int64_t t = first; t < end; ++t)
      if (!mbar_wait(bars + int(t % kGStages), uint32_t((t / kGStages) & 1), p.status)) break;
  }
  if (!own_result) return;
  const uint32_t* own_ids = own_keyed ? p.keyed_ids : p.multi_ids;
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    if (!valid[q]) continue;
    const uint32_t id = own_ids[wi.own_begin + int64_t(q) * kGThreads + threadIdx.x];
    if constexpr (MODE == MODE_ANY) {
      if (cov[q]) p.out_u32[id] = 1u;
    }
    if constexpr (MODE == MODE_COUNT) {
      if (cnt[q]) atomicAdd(p.out_u32 + id, cnt[q]);
    }
    if constexpr (MODE == MODE_SUM) {
      if (sum[q]) atomicAdd(p.out_u64 + id, sum[q]);
    }
  }
}

// Each block holds 256 * q own rows, q = 1, 2 or 4 chosen per work item
// from the size of its group (q never exceeds GShape<KT>::Q).
template <int KT, int MODE>
__global__ void __launch_bounds__(kGThreads) grouped_subset_kernel(GroupedParams p) {
  extern __shared__ __align__(128) uint8_t smem[];
  const WorkItem wi = p.items[blockIdx.x];
  if (wi.q <= 1)
    grouped_body<KT, MODE, 1>(p, wi, smem);
  else if (wi.q == 2 || GShape<KT>::Q == 2)
    grouped_body<KT, MODE, 2>(p, wi, smem);
  else
    grouped_body<KT, MODE, (GShape<KT>::Q >= 4 ? 4 : 2)>(p, wi, smem);
}

// ---- host side ----------------------------------------------------------------

cudaError_t launch_item_histogram(const uint64_t* rows, int64_t n, int stride, int K, int L,
                                  uint32_t* freq, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  int64_t blocks = ceil_div(n, 256);
  if (blocks > int64_t(num_sms()) * 4) blocks = int64_t(num_sms()) * 4;
  item_histogram_kernel<<<unsigned(blocks), 256, size_t(L) * 4, s>>>(rows, n, stride, K, L, freq);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_small_scan(const uint32_t* cnt, int len, uint32_t* off, cudaStream_t s) {
  small_scan_kernel<<<1, 1024, 0, s>>>(cnt, len, off);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_multi_scatter(const uint64_t* rows, int64_t n, int stride, int K, int KT,
                                 int L, const uint32_t* off, uint32_t* cursor, uint64_t* out,
                                 uint32_t* ids, const uint32_t* id_map, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  // One warp per row; large inputs take wide blocks, so that popular items
  // get few global reservations.
  const int warps = n >= int64_t(num_sms()) * 32 * 4 ? 32 : 8;
  const size_t smem = size_t(warps) * KT * 8 + size_t(2) * L * 4;
  multi_scatter_kernel<<<unsigned(ceil_div(n, warps)), warps * 32, smem, s>>>(
      rows, n, stride, K, KT, L, off, cursor, out, ids, id_map);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_key_item(const uint64_t* rows, int64_t n, int stride, int K, int L,
                            const uint32_t* freq, uint32_t* key, uint32_t* kcount,
                            const unsigned long long* n_dev, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  key_item_kernel<<<unsigned(ceil_div(n, 256)), 256, size_t(2 * L + 1) * 4, s>>>(
      rows, n, stride, K, L, freq, key, kcount, n_dev);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_keyed_scatter(const uint64_t* rows, int64_t n, int stride, int K, int KT,
                                 int groups, const uint32_t* key, const uint32_t* off,
                                 uint32_t* cursor, uint64_t* out, uint32_t* ids,
                                 const uint64_t* payload, uint64_t* payload_out,
                                 const unsigned long long* n_dev, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  const int nb = scatter_threads(n);
  const size_t smem = size_t(nb) * KT * 8 + size_t(2) * groups * 4;
  keyed_scatter_kernel<<<unsigned(ceil_div(n, nb)), nb, smem, s>>>(
      rows, n, stride, K, KT, groups, key, off, cursor, out, ids, payload, payload_out, n_dev);
  count_launches(1);
  return cudaGetLastError();
}

int grouped_rows_per_tile(int KT) {
  switch (KT) {
    case 2: return GShape<2>::TR;
    case 4: return GShape<4>::TR;
    case 8: return GShape<8>::TR;
    case 16: return GShape<16>::TR;
  }
  return 256;
}

int grouped_own_per_cta(int KT) { return kGThreads * (KT >= 16 ? 2 : 4); }

template <int KT, int MODE>
static cudaError_t grouped_t(const GroupedArgs& a, cudaStream_t s) {
  using S = GShape<KT>;
  GroupedParams p{a.items, a.keyed, a.keyed_ids, a.keyed_score, a.multi, a.multi_ids,
                  a.out_u32, a.out_u64, a.status};
  const size_t smem = size_t(kGStages) * S::TR * KT * 8 + kGStages * sizeof(uint64_t);
  grouped_subset_kernel<KT, MODE><<<unsigned(a.n_items), kGThreads, smem, s>>>(p);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_grouped_subset(const GroupedArgs& a, cudaStream_t s) {
  if (a.n_items == 0) return cudaSuccess;
#define IG_G_CASE(KTV)                                          \
  case KTV:                                                     \
    switch (a.mode) {                                           \
      case MODE_ANY: return grouped_t<KTV, MODE_ANY>(a, s);     \
      case MODE_COUNT: return grouped_t<KTV, MODE_COUNT>(a, s); \
      case MODE_SUM: return grouped_t<KTV, MODE_SUM>(a, s);     \
    }                                                           \
    break;
  switch (a.KT) {
    IG_G_CASE(2)
    IG_G_CASE(4)
    IG_G_CASE(8)
    IG_G_CASE(16)
  }
#undef IG_G_CASE
  return cudaErrorInvalidValue;
}

// Blocks (group, own tile, stream range) with about `target` tests each;
// in every group the larger side goes to registers (own).
void build_work_items(const uint32_t* keyed_off, const uint32_t* multi_off, int groups,
                      int own_tile, int str_tile, int64_t n_blocks_goal, bool mode_sum,
                      int max_q_param, int flip, std::vector<WorkItem>* items, int64_t* tests) {
  const int max_q = std::max(1, std::min(own_tile / 256, max_q_param));
  items->clear();
  *tests = 0;
  // The result side stays in registers unless the other side is at least
  // twice as large (then per-hit atomics are the cheaper way to fill lanes).
  auto orient = [&](int64_t nk, int64_t nm) {
    return mode_sum ? (nk >= int64_t(flip) * nm) : (int64_t(flip) * nk >= nm);
  };
  // A block's cost is the lane-tests it executes: every stream row meets
  // 32 * ceil(own rows / 32) lanes (warps without an own row skip the tests).
  // Stream ranges are cut so that every block costs about the same, and
  // there are about n_blocks_goal of them.
  auto lanes = [](int64_t oc) { return ((oc + 31) / 32) * 32; };
  int64_t total = 0;
  for (int l = 0; l < groups; ++l) {
    const int64_t nk = int64_t(keyed_off[l + 1]) - keyed_off[l];
    const int64_t nm = int64_t(multi_off[l + 1]) - multi_off[l];
    if (nk == 0 || nm == 0) continue;
    const bool ok = orient(nk, nm);
    total += lanes(ok ? nk : nm) * (ok ? nm : nk);
  }
  const int64_t target = std::max<int64_t>(total / std::max<int64_t>(1, n_blocks_goal), 1 << 16);
  for (int l = 0; l < groups; ++l) {
    const int64_t nk = int64_t(keyed_off[l + 1]) - keyed_off[l];
    const int64_t nm = int64_t(multi_off[l + 1]) - multi_off[l];
    if (nk == 0 || nm == 0) continue;
    *tests += nk * nm;
    const bool own_keyed = orient(nk, nm);
    const int64_t no = own_keyed ? nk : nm, ns = own_keyed ? nm : nk;
    const int64_t o0 = own_keyed ? keyed_off[l] : multi_off[l];
    const int64_t s0 = own_keyed ? multi_off[l] : keyed_off[l];
    // Rows per thread from the group's size: small groups use narrow blocks.
    int q = 1;
    while (q < max_q && 256 * q < no) q *= 2;
    const int64_t tile = std::min<int64_t>(own_tile, 256 * q);
    for (int64_t o = 0; o < no; o += tile) {
      const int64_t oc = std::min<int64_t>(tile, no - o);
      int64_t per = std::max<int64_t>(str_tile, target / lanes(oc));
      per = ((per + str_tile - 1) / str_tile) * str_tile;
      for (int64_t r = 0; r < ns; r += per) {
        WorkItem w;
        w.own_begin = o0 + o;
        w.own_count = oc;
        w.str_begin = s0 + r;
        w.str_count = std::min<int64_t>(per, ns - r);
        w.own_keyed = own_keyed ? 1 : 0;
        w.q = q;
        items->push_back(w);
      }
    }
  }
}

// ---- record index -------------------------------------------------------------

void release_record_index(RecordIndex* idx, cudaStream_t s) {
  for (void* p : {static_cast<void*>(idx->rows), static_cast<void*>(idx->ids),
                  static_cast<void*>(idx->small)})
    if (p) cudaFreeAsync(p, s);
  idx->rows = nullptr;
  idx->ids = nullptr;
  idx->small = nullptr;
  idx->usable = false;
}

cudaError_t build_record_index(const uint64_t* rows, int64_t n, int stride, int K, int KT,
                               double max_fill, RecordIndex* idx, cudaStream_t s,
                               const uint32_t* id_map) {
  *idx = RecordIndex();
  idx->K = K;
  idx->KT = KT;
  idx->L = 64 * K;
  idx->n_rows = n;
  const int L = idx->L;
  cudaError_t e;
#define IG_I_TRY(x)                  \
  if ((e = (x)) != cudaSuccess) {     \
    release_record_index(idx, s);    \
    return e;                        \
  }
  // freq[L], off[L+1], cursor[L] in one allocation.
  IG_I_TRY(cudaMallocAsync(reinterpret_cast<void**>(&idx->small), size_t(3 * L + 1) * 4, s));
  idx->freq = idx->small;
  idx->off = idx->freq + L;
  uint32_t* cursor = idx->off + (L + 1);
  IG_I_TRY(cudaMemsetAsync(idx->small, 0, size_t(3 * L + 1) * 4, s));
  if (n > 0) {
    void* tok = prof_begin(kStageIndexBuild, s);
    IG_I_TRY(launch_item_histogram(rows, n, stride, K, L, idx->freq, s));
    IG_I_TRY(launch_small_scan(idx->freq, L, idx->off, s));
    prof_end(tok);
  }
  idx->h_off.assign(L + 1, 0u);
  IG_I_TRY(cudaMemcpyAsync(idx->h_off.data(), idx->off, (L + 1) * 4, cudaMemcpyDeviceToHost, s));
  IG_I_TRY(cudaStreamSynchronize(s));
  idx->n_copies = idx->h_off[L];
  idx->usable = n > 0 && double(idx->n_copies) <= max_fill * double(n) * double(L);
  if (!idx->usable) return cudaSuccess;
  // Grouped copies, padded by one stream tile so whole-tile copies stay in bounds.
  IG_I_TRY(cudaMallocAsync(reinterpret_cast<void**>(&idx->rows),
                           size_t(idx->n_copies + 256) * KT * 8, s));
  IG_I_TRY(cudaMallocAsync(reinterpret_cast<void**>(&idx->ids), size_t(idx->n_copies) * 4, s));
  void* tok = prof_begin(kStageIndexBuild, s);
  IG_I_TRY(launch_multi_scatter(rows, n, stride, K, KT, L, idx->off, cursor, idx->rows, idx->ids,
                                id_map, s));
  prof_end(tok);
#undef IG_I_TRY
  return cudaSuccess;
}

namespace {
// Pinned staging for work lists: reused once the copy out of it (recorded
// by `done`) has finished.
struct Staging {
  WorkItem* buf = nullptr;
  size_t cap = 0;
  cudaEvent_t done = nullptr;
};
thread_local Staging g_staging;
}  // namespace

void release_keyed_index(KeyedIndex* k, cudaStream_t s) {
  for (void* p : {static_cast<void*>(k->rows), static_cast<void*>(k->ids),
                  static_cast<void*>(k->score), static_cast<void*>(k->off)})
    if (p) cudaFreeAsync(p, s);
  k->rows = nullptr;
  k->ids = nullptr;
  k->score = nullptr;
  k->off = nullptr;
  k->n = 0;
}

cudaError_t build_keyed_index(const uint64_t* keyed, int64_t n, int stride, int K, int KT,
                              const uint32_t* freq, const uint64_t* score, KeyedIndex* out,
                              cudaStream_t s, const unsigned long long* n_dev, bool host_offsets) {
  *out = KeyedIndex();
  out->K = K;
  out->KT = KT;
  out->L = 64 * K;
  out->n = n;
  const int L = out->L, groups = L + 1;
  cudaError_t e;
  uint32_t *kcount = nullptr, *key = nullptr;
#define IG_K_TRY(x)                            \
  if ((e = (x)) != cudaSuccess) {               \
    if (kcount) cudaFreeAsync(kcount, s);      \
    if (key) cudaFreeAsync(key, s);            \
    release_keyed_index(out, s);               \
    return e;                                  \
  }
  // kcount[groups] and cursor[groups] scratch; off[groups+1] kept.
  IG_K_TRY(cudaMallocAsync(reinterpret_cast<void**>(&kcount), size_t(2 * groups) * 4, s));
  IG_K_TRY(cudaMallocAsync(reinterpret_cast<void**>(&out->off), size_t(groups + 1) * 4, s));
  IG_K_TRY(cudaMallocAsync(reinterpret_cast<void**>(&key), size_t(std::max<int64_t>(1, n)) * 4, s));
  IG_K_TRY(cudaMemsetAsync(kcount, 0, size_t(2 * groups) * 4, s));
  IG_K_TRY(cudaMallocAsync(reinterpret_cast<void**>(&out->rows), size_t(n + 256) * KT * 8, s));
  IG_K_TRY(cudaMallocAsync(reinterpret_cast<void**>(&out->ids), size_t(std::max<int64_t>(1, n)) * 4, s));
  if (score)
    IG_K_TRY(cudaMallocAsync(reinterpret_cast<void**>(&out->score), size_t(n + 256) * 8, s));
  void* tok = prof_begin(kStageIndexBuild, s);
  IG_K_TRY(launch_key_item(keyed, n, stride, K, L, freq, key, kcount, n_dev, s));
  IG_K_TRY(launch_small_scan(kcount, groups, out->off, s));
  IG_K_TRY(launch_keyed_scatter(keyed, n, stride, K, KT, groups, key, out->off, kcount + groups,
                                out->rows, out->ids, score, out->score, n_dev, s));
  prof_end(tok);
  if (host_offsets) {
    out->h_off.assign(groups + 1, 0u);
    IG_K_TRY(cudaMemcpyAsync(out->h_off.data(), out->off, (groups + 1) * 4, cudaMemcpyDeviceToHost, s));
    IG_K_TRY(cudaStreamSynchronize(s));
    out->n = int64_t(out->h_off[groups]);  // the rows filed: n, or *n_dev when given
  }
  cudaFreeAsync(kcount, s);
  cudaFreeAsync(key, s);
#undef IG_K_TRY
  return cudaSuccess;
}

cudaError_t indexed_subset_prebuilt(int mode, const RecordIndex& idx, const KeyedIndex& kx,
                                    uint32_t* out_u32, unsigned long long* out_u64, int* status,
                                    int64_t* tests_out, int prof_stage, int max_q,
                                    int flip_factor, int tc, cudaStream_t s,
                                    uint64_t score_max) {
  *tests_out = 0;
  if (kx.n == 0 || idx.n_rows == 0) return cudaSuccess;
  const int L = idx.L, KT = idx.KT;
  if (tc && tc_supported(KT))  // work items built on the device; *tests_out written later
    return indexed_subset_tc(mode, idx, kx, out_u32, out_u64, status, tests_out, prof_stage,
                             score_max, s);
  std::vector<WorkItem> items;
  int64_t tests = 0;
  build_work_items(kx.h_off.data(), idx.h_off.data(), L, grouped_own_per_cta(KT),
                   grouped_rows_per_tile(KT), int64_t(num_sms()) * 8, mode == MODE_SUM, max_q,
                   std::max(1, flip_factor), &items, &tests);
  *tests_out = tests;
  if (items.empty()) return cudaSuccess;
  cudaError_t e;
  Staging& st = g_staging;
  if (st.done && (e = cudaEventSynchronize(st.done)) != cudaSuccess) return e;
  if (st.cap < items.size()) {
    if (st.buf) cudaFreeHost(st.buf);
    st.buf = nullptr;
    st.cap = 0;
    if ((e = cudaMallocHost(reinterpret_cast<void**>(&st.buf), items.size() * 2 * sizeof(WorkItem))) !=
        cudaSuccess)
      return e;
    st.cap = items.size() * 2;
  }
  if (!st.done && (e = cudaEventCreateWithFlags(&st.done, cudaEventDisableTiming)) != cudaSuccess)
    return e;
  std::copy(items.begin(), items.end(), st.buf);
  WorkItem* d_items = nullptr;
  if ((e = cudaMallocAsync(reinterpret_cast<void**>(&d_items), items.size() * sizeof(WorkItem), s)) !=
      cudaSuccess)
    return e;
  e = cudaMemcpyAsync(d_items, st.buf, items.size() * sizeof(WorkItem), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaEventRecord(st.done, s);
  if (e == cudaSuccess) {
    GroupedArgs g{mode,    KT,       d_items, int64_t(items.size()), kx.rows, kx.ids,
                  kx.score, idx.rows, idx.ids, out_u32,               out_u64, status};
    void* tok = prof_stage >= 0 ? prof_begin(prof_stage, s) : nullptr;
    e = launch_grouped_subset(g, s);
    prof_end(tok);
  }
  cudaFreeAsync(d_items, s);
  return e;
}

cudaError_t indexed_subset(const IndexedArgs& a, cudaStream_t s) {
  *a.tests_out = 0;
  const RecordIndex& idx = *a.index;
  if (a.n_keyed == 0 || idx.n_rows == 0) return cudaSuccess;
  KeyedIndex kx;
  // The tensor-core form builds its work items on the device: no read-back.
  const bool device_items = a.tc && tc_supported(idx.KT);
  cudaError_t e = build_keyed_index(a.keyed, a.n_keyed, a.keyed_stride, idx.K, idx.KT, idx.freq,
                                    a.mode == MODE_SUM ? a.keyed_score : nullptr, &kx, s,
                                    a.n_keyed_dev, !device_items);
  if (e != cudaSuccess) return e;
  if (kx.n == 0) {  // no keyed rows left on the device: nothing to test
    release_keyed_index(&kx, s);
    return cudaSuccess;
  }
  e = indexed_subset_prebuilt(a.mode, idx, kx, a.out_u32, a.out_u64, a.status, a.tests_out,
                              a.prof_stage, a.max_q, a.flip_factor, a.tc, s, a.score_max);
  release_keyed_index(&kx, s);
  return e;
}

}  // namespace igk
