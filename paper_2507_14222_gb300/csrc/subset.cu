// Subset tests on the integer pipe (Eq. 6, Eq. 3, Eq. 2, Eq. 4).
//
// One kernel serves the three uses of the subset test:
//   MODE_ANY   coherence (Eq. 3): is candidate b inside ANY opposite record?
//   MODE_COUNT support (Eq. 2):   how many same-class records contain b?
//   MODE_SUM   evidence (Eq. 4):  sum of S(b) over patterns b inside record x.
//
// Each thread keeps Q "own" rows in registers as 32-bit halves; the CTA
// streams the other operand through shared memory in tiles of TR rows,
// fetched by one thread with 1-D TMA bulk copies into a kStages-deep ring of
// buffers, each completing on its own mbarrier.  Every lane of a warp reads
// the same streamed row (a shared-memory broadcast), and the test of one
// (pattern p, record r) pair is 2*KT instances of acc |= p & ~r, each a
// single LOP3, followed by acc == 0: p is inside r iff no item of p is
// missing from r, which is Eq. 6's conjunction of (p AND r) == p over words.
//
// The grid is (own blocks) x (stream splits); partial results of the splits
// are combined with atomics (OR-like store, integer adds), so the result is
// independent of the split count and of scheduling.
#include "common.cuh"
#include "internal.h"

namespace igk {

constexpr int kSubThreads = 256;
constexpr int kStages = 4;

template <int KT>
struct SubsetShape {
  // 8 KiB of rows per stage, between 64 and 256 rows (divides kRowPad).
  static constexpr int TR = (8192 / (KT * 8)) > 256 ? 256 : (8192 / (KT * 8));
  static constexpr int Q = KT >= 16 ? 2 : 4;  // own rows per thread
  static constexpr int H = 2 * KT;            // 32-bit halves per row
};

struct SubsetParams {
  const uint64_t* own;
  int64_t n_own;
  int own_stride;
  const uint64_t* stream;
  const uint64_t* stream_score;
  int64_t n_stream;
  int64_t per_split;  // stream rows per grid.y split, a multiple of TR
  uint32_t* out_u32;
  unsigned long long* out_u64;
  int* status;
  const unsigned long long* n_own_dev;
};

template <int H>
__device__ __forceinline__ void load_halves(const uint32_t* src, uint32_t (&d)[H]) {
  if constexpr (H >= 4) {
#pragma unroll
    for (int v = 0; v < H / 4; ++v) {
      uint4 x = reinterpret_cast<const uint4*>(src)[v];
      d[4 * v] = x.x;
      d[4 * v + 1] = x.y;
      d[4 * v + 2] = x.z;
      d[4 * v + 3] = x.w;
    }
  } else {
    uint2 x = *reinterpret_cast<const uint2*>(src);
    d[0] = x.x;
    d[1] = x.y;
  }
}

template <int KT, int MODE>
__global__ void __launch_bounds__(kSubThreads)
    subset_kernel(SubsetParams p) {
  using S = SubsetShape<KT>;
  constexpr int TR = S::TR, Q = S::Q, H = S::H;
  constexpr uint32_t kRowBytes = TR * KT * 8;
  constexpr uint32_t kScoreBytes = MODE == MODE_SUM ? TR * 8 : 0;

  extern __shared__ __align__(128) uint8_t smem[];
  uint64_t* rows_s = reinterpret_cast<uint64_t*>(smem);
  uint64_t* score_s = rows_s + kStages * TR * KT;
  uint64_t* bars = score_s + (MODE == MODE_SUM ? kStages * TR : 0);

  // CTAs past the own rows (when their count is read on the device) exit
  // before touching any barrier or copy.
  const int64_t n_own = p.n_own_dev ? int64_t(*p.n_own_dev) : p.n_own;
  const int64_t own_base = int64_t(blockIdx.x) * (kSubThreads * Q);
  if (own_base >= n_own) return;

  // Own rows -> registers (words beyond own_stride read as zero).
  uint32_t own[Q][H];
  bool valid[Q];
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    int64_t row = own_base + q * kSubThreads + threadIdx.x;
    valid[q] = row < n_own;
#pragma unroll
    for (int k = 0; k < KT; ++k) {
      uint64_t w = (valid[q] && k < p.own_stride) ? p.own[row * p.own_stride + k] : 0ull;
      own[q][2 * k] = uint32_t(w);
      own[q][2 * k + 1] = uint32_t(w >> 32);
    }
  }

  const int64_t s_lo = int64_t(blockIdx.y) * p.per_split;
  int64_t s_hi = s_lo + p.per_split;
  if (s_hi > p.n_stream) s_hi = p.n_stream;
  const int64_t ntiles = s_hi > s_lo ? ceil_div(s_hi - s_lo, TR) : 0;

  if (threadIdx.x == 0) {
    for (int st = 0; st < kStages; ++st) mbar_init(bars + st, 1);
    fence_mbar_init();
  }
  __syncthreads();

  auto issue = [&](int64_t tile) {
    const int st = int(tile % kStages);
    const int64_t r0 = s_lo + tile * TR;
    mbar_arrive_expect_tx(bars + st, kRowBytes + kScoreBytes);
    bulk_g2s(rows_s + st * TR * KT, p.stream + r0 * KT, kRowBytes, bars + st);
    if constexpr (MODE == MODE_SUM)
      bulk_g2s(score_s + st * TR, p.stream_score + r0, kScoreBytes, bars + st);
  };
  if (threadIdx.x == 0)
    for (int64_t t = 0; t < ntiles && t < kStages; ++t) issue(t);

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
    const int st = int(tile % kStages);
    const uint32_t parity = uint32_t((tile / kStages) & 1);
    // Every thread waits on the stage's barrier; the decision to give up is
    // made CTA-wide so that no thread is left waiting at a later barrier.
    const bool ok = mbar_wait(bars + st, parity, p.status);
    if (__syncthreads_or(!ok)) {
      failed = true;
      break;
    }
    int nr = int((s_hi - (s_lo + tile * TR)) < TR ? (s_hi - (s_lo + tile * TR)) : TR);
    const uint32_t* rs = reinterpret_cast<const uint32_t*>(rows_s + st * TR * KT);
#pragma unroll 2
    for (int r = 0; r < nr; ++r) {
      uint32_t rh[H];
      load_halves<H>(rs + r * H, rh);
      unsigned long long sc = 0;
      if constexpr (MODE == MODE_SUM) sc = score_s[st * TR + r];
#pragma unroll
      for (int q = 0; q < Q; ++q) {
        uint32_t acc = 0;
#pragma unroll
        for (int h = 0; h < H; ++h) {
          if constexpr (MODE == MODE_SUM)
            acc |= rh[h] & ~own[q][h];   // streamed pattern inside own record?
          else
            acc |= own[q][h] & ~rh[h];   // own pattern inside streamed record?
        }
        const bool hit = acc == 0u;
        if constexpr (MODE == MODE_ANY) cov[q] |= hit;
        if constexpr (MODE == MODE_COUNT) cnt[q] += hit ? 1u : 0u;
        if constexpr (MODE == MODE_SUM) sum[q] += hit ? sc : 0ull;
      }
    }
    bool stop = false;
    if constexpr (MODE == MODE_ANY) {
      bool done = true;
#pragma unroll
      for (int q = 0; q < Q; ++q) done &= (cov[q] || !valid[q]);
      stop = __syncthreads_and(done) != 0;  // also frees this stage
    } else {
      __syncthreads();
    }
    if (stop) break;
    if (threadIdx.x == 0 && tile + kStages < ntiles) issue(tile + kStages);
  }
  // Tiles issued but not consumed must land before the CTA exits: after an
  // early stop at `tile` they are tile+1 .. tile+kStages-1; after a failed
  // wait, tile .. tile+kStages-1 (clipped to ntiles).
  if (threadIdx.x == 0 && tile < ntiles) {
    const int64_t first = failed ? tile : tile + 1;
    const int64_t end = (tile + kStages < ntiles) ? tile + kStages : ntiles;
    for (int64_t t = first; t < end; ++t)
      if (!mbar_wait(bars + int(t % kStages), uint32_t((t / kStages) & 1), p.status)) break;
  }

#pragma unroll
  for (int q = 0; q < Q; ++q) {
    if (!valid[q]) continue;
    int64_t row = own_base + q * kSubThreads + threadIdx.x;
    if constexpr (MODE == MODE_ANY) {
      if (cov[q]) p.out_u32[row] = 1u;
    }
    if constexpr (MODE == MODE_COUNT) {
      if (cnt[q]) atomicAdd(p.out_u32 + row, cnt[q]);
    }
    if constexpr (MODE == MODE_SUM) {
      if (sum[q]) atomicAdd(p.out_u64 + row, sum[q]);
    }
  }
}

template <int KT, int MODE>
static cudaError_t launch_subset_t(const SubsetArgs& a, cudaStream_t s) {
  using S = SubsetShape<KT>;
  if (a.n_own == 0 || a.n_stream == 0) return cudaSuccess;
  const int64_t own_per_cta = int64_t(kSubThreads) * S::Q;
  const int64_t gx = ceil_div(a.n_own, own_per_cta);
  const int64_t stream_tiles = ceil_div(a.n_stream, S::TR);
  // Enough CTAs for every SM to hold several; each split covers whole tiles.
  const int64_t target = int64_t(num_sms()) * 4;
  int64_t splits = ceil_div(target, gx);
  if (splits > stream_tiles) splits = stream_tiles;
  if (splits > 65535) splits = 65535;
  if (splits < 1) splits = 1;
  const int64_t per_split = ceil_div(stream_tiles, splits) * S::TR;
  splits = ceil_div(a.n_stream, per_split);
  SubsetParams p{a.own,     a.n_own,   a.own_stride, a.stream,  a.stream_score, a.n_stream,
                 per_split, a.out_u32, a.out_u64,    a.status, a.n_own_dev};
  const size_t smem = size_t(kStages) * (S::TR * KT * 8 + (MODE == MODE_SUM ? S::TR * 8 : 0)) +
                      kStages * sizeof(uint64_t);
  if (gx > 0x7fffffff) return cudaErrorInvalidValue;
  dim3 grid{unsigned(gx), unsigned(splits), 1u};
  subset_kernel<KT, MODE><<<grid, kSubThreads, smem, s>>>(p);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_subset(const SubsetArgs& a, cudaStream_t s) {
  switch (a.mode) {
    case MODE_ANY: { IG_DISPATCH_KT(a.KT, return (launch_subset_t<KTC, MODE_ANY>(a, s))); }
    case MODE_COUNT: { IG_DISPATCH_KT(a.KT, return (launch_subset_t<KTC, MODE_COUNT>(a, s))); }
    case MODE_SUM: { IG_DISPATCH_KT(a.KT, return (launch_subset_t<KTC, MODE_SUM>(a, s))); }
  }
  return cudaErrorInvalidValue;
}

// Warp-aggregated append of the rows whose flag is zero.
constexpr int kSelectThreads = 256;
template <int KT>
__global__ void __launch_bounds__(kSelectThreads)
    select_unflagged_kernel(const uint64_t* __restrict__ rows, int64_t n,
                            const uint32_t* __restrict__ flag, uint64_t* __restrict__ out,
                            unsigned long long* out_count, const unsigned long long* n_dev) {
  // Each block takes a contiguous range of rows: it counts the unflagged
  // ones, reserves room for them with one atomic on the global count, and
  // places them through a shared-memory cursor (one global atomic per block).
  __shared__ unsigned int blk_count, blk_cursor;
  __shared__ unsigned long long blk_base;
  if (n_dev) n = int64_t(*n_dev);
  const int lane = threadIdx.x & 31;
  const int64_t per = ((n + gridDim.x - 1) / gridDim.x + 31) & ~int64_t(31);
  const int64_t lo = int64_t(blockIdx.x) * per;
  const int64_t hi = lo + per < n ? lo + per : n;
  if (threadIdx.x == 0) {
    blk_count = 0;
    blk_cursor = 0;
  }
  __syncthreads();
  unsigned int mine = 0;
  for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) mine += flag[i] == 0u ? 1u : 0u;
#pragma unroll
  for (int o = 16; o; o >>= 1) mine += __shfl_xor_sync(0xffffffffu, mine, o);
  if (lane == 0 && mine) atomicAdd(&blk_count, mine);
  __syncthreads();
  if (threadIdx.x == 0) blk_base = blk_count ? atomicAdd(out_count, (unsigned long long)blk_count) : 0ull;
  __syncthreads();
  // The kept rows of each 32-row step are copied by the whole warp, 32 / KT
  // rows per instruction with consecutive lanes on consecutive words.
  __shared__ int64_t kept_row[kSelectThreads];
  int64_t* my_kept = kept_row + (threadIdx.x & ~31);
  constexpr int kRowsPer = 32 / KT;
  const int sub = lane / KT, word = lane % KT;
  for (int64_t base = lo + (threadIdx.x & ~31); base < hi; base += blockDim.x) {
    const int64_t i = base + lane;
    const bool keep = i < hi && flag[i] == 0u;
    const unsigned m = __ballot_sync(0xffffffffu, keep);
    if (m == 0) continue;
    unsigned int p0 = 0;
    if (lane == 0) p0 = atomicAdd(&blk_cursor, unsigned(__popc(m)));
    p0 = __shfl_sync(0xffffffffu, p0, 0);
    if (keep) my_kept[__popc(m & ((1u << lane) - 1u))] = i;
    __syncwarp();
    const int nk = __popc(m);
    for (int b = sub; b < nk; b += kRowsPer) {
      const uint64_t pos = blk_base + p0 + unsigned(b);
      out[pos * KT + word] = rows[my_kept[b] * KT + word];
    }
    __syncwarp();
  }
}

cudaError_t launch_select_unflagged(const uint64_t* rows, int64_t n, int KT,
                                    const uint32_t* flag, uint64_t* out,
                                    unsigned long long* out_count, cudaStream_t s,
                                    const unsigned long long* n_dev) {
  if (n == 0) return cudaSuccess;
  // Ranges of at least 2,048 rows, at most 16 blocks per SM (n is an upper
  // bound when the count is on the device).
  int64_t blocks = ceil_div(n, 2048);
  if (blocks > int64_t(num_sms()) * 16) blocks = int64_t(num_sms()) * 16;
  if (blocks < 1) blocks = 1;
  IG_DISPATCH_KT(KT, (select_unflagged_kernel<KTC><<<unsigned(blocks), kSelectThreads, 0, s>>>(
                         rows, n, flag, out, out_count, n_dev)));
  count_launches(1);
  return cudaGetLastError();
}

// Eq. 2: S = f * |b|^2, |b| the number of items of b.
__global__ void pattern_score_kernel(const uint64_t* __restrict__ rows, int64_t n,
                                     int KT, const uint32_t* __restrict__ f,
                                     uint64_t* __restrict__ S,
                                     unsigned long long* __restrict__ smax) {
  int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  unsigned long long v = 0;
  if (i < n) {
    uint64_t items = 0;
    for (int k = 0; k < KT; ++k) items += __popcll(rows[i * KT + k]);
    v = uint64_t(f[i]) * items * items;
    S[i] = v;
  }
  if (smax) {
    // Largest score of the warp, then one atomic per warp.
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
      const unsigned long long o = __shfl_xor_sync(0xffffffffu, v, d);
      v = o > v ? o : v;
    }
    if ((threadIdx.x & 31) == 0 && v) atomicMax(smax, v);
  }
}

cudaError_t launch_pattern_score(const uint64_t* rows, int64_t n, int KT,
                                 const uint32_t* f, uint64_t* S, cudaStream_t s,
                                 unsigned long long* smax) {
  if (n == 0) return cudaSuccess;
  pattern_score_kernel<<<unsigned(ceil_div(n, 256)), 256, 0, s>>>(rows, n, KT, f, S, smax);
  count_launches(1);
  return cudaGetLastError();
}

// Regulations 1-3 of Section 3.1, in the paper's order.
__global__ void labels_kernel(const unsigned long long* __restrict__ A,
                              const unsigned long long* __restrict__ N, int64_t m,
                              int reg3, double threshold, uint8_t* __restrict__ out) {
  int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t >= m) return;
  const long long a = (long long)A[t], nn = (long long)N[t];
  uint8_t label = a >= nn ? 1 : 0;                          // Regulation 1
  if (a == 0 && nn == 0) label = 1;                         // Regulation 2
  if (reg3 && label == 0 && double(nn) < threshold) label = 1;  // Regulation 3
  out[t] = label;
}

cudaError_t launch_labels(const unsigned long long* A, const unsigned long long* N,
                          int64_t m, int reg3, double threshold, uint8_t* out,
                          cudaStream_t s) {
  if (m == 0) return cudaSuccess;
  labels_kernel<<<unsigned(ceil_div(m, 256)), 256, 0, s>>>(A, N, m, reg3, threshold, out);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace igk
