// Subset tests on the tensor cores: a 0/1 GEMM with tcgen05 (sm_100 family).
//
// Eq. 6 tests every word of p against r.  Counted instead over items l,
//   D[p, r] = sum_l p_l * (1 - r_l)
// is the number of items of p missing from r, so p is inside r iff D == 0.
// That sum is a matrix product of 0/1 matrices: pattern bits against
// complemented record bits.  The operands are expanded to one FP8 (E4M3)
// byte per item (1.0 = 0x38) and multiplied by tcgen05.mma kind::f8f6f4 into
// FP32 accumulators in tensor memory; the counts are at most 64*KT <= 512,
// exact in FP32, and D == 0 is read straight from the accumulator bits.
//
// One CTA owns 128 "own" rows (the A operand, M = 128, resident in shared
// memory) and streams tiles of N = 128 rows of the other operand (B) through
// a ring of shared-memory stages filled by 1-D TMA bulk copies.  Warp roles:
//   warp 0   lane 0 issues the bulk copies (A once, then the B tiles);
//   warp 1   allocates tensor memory; lane 0 issues the MMAs and commits;
//   warps 2-5 read the accumulators (tcgen05.ld, one 32-lane quarter each)
//            and reduce them: any / count / score-weighted sum (Eq. 3, 2, 4).
// Two accumulator buffers let the epilogue of tile t overlap the MMAs of
// tile t+1.  Every wait is bounded; on a timeout the CTA records it in the
// status word, stops issuing work, waits (bounded) for what is in flight and
// frees its tensor memory.
//
// The operands live in global memory already in the shared-memory image the
// MMA reads (K-major, 128-byte swizzle: 8-row x 128-byte atoms, the 16-byte
// chunk c of row r stored at chunk c ^ (r mod 8)), so every tile is one
// contiguous bulk copy.  expand_kernel writes these images from packed rows.
#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "common.cuh"
#include "internal.h"

namespace igk {

constexpr int kTcM = 128;          // own rows per CTA (MMA M)
constexpr int kTcN = 128;          // stream rows per tile (MMA N)
constexpr int kTcThreads = 192;    // 6 warps
constexpr uint32_t kTmemCols = 2 * kTcN;

template <int KT>
struct TcShape {
  static constexpr int kBytesPerRow = KT * 64;             // one byte per item
  static constexpr int kKSteps = KT * 64 / 32;             // MMA K = 32 for 8-bit inputs
  static constexpr uint32_t kABytes = kTcM * kBytesPerRow;
  static constexpr uint32_t kBBytes = kTcN * kBytesPerRow;
  static constexpr int kStages = (200 * 1024 - int(kABytes)) / int(kBBytes) > 6
                                     ? 6
                                     : (200 * 1024 - int(kABytes)) / int(kBBytes);
  static constexpr size_t kSmem = 1024 + kABytes + size_t(kStages) * kBBytes + 256;
};

// ---- operand images ---------------------------------------------------------

// img tile t holds rows [t*R, t*R + R): byte offset of item k of tile row r is
//   (k / 128) * (R * 128) + r * 128 + (((k % 128) / 16) ^ (r % 8)) * 16 + k % 16.
// One thread writes one 16-byte chunk.  Rows >= n are zero.
template <int KT, int R>
__global__ void expand_kernel(const uint64_t* __restrict__ rows, int64_t n, int stride,
                              int complement, int64_t ntiles, uint8_t* __restrict__ img) {
  constexpr int64_t chunks_per_tile = int64_t(R) * KT * 4;
  const int64_t id = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (id >= ntiles * chunks_per_tile) return;
  const int64_t tile = id / chunks_per_tile;
  const int64_t rem = id - tile * chunks_per_tile;
  const int katom = int(rem / (R * 8));
  const int rem2 = int(rem - int64_t(katom) * R * 8);
  const int r = rem2 >> 3, pos = rem2 & 7;
  const int c = pos ^ (r & 7);
  const int k0 = katom * 128 + c * 16;
  const int64_t g = tile * R + r;
  uint32_t bits = 0;
  if (g < n) {
    const int word = k0 >> 6;
    uint64_t w = word < stride ? rows[g * stride + word] : 0ull;
    if (complement) w = ~w;
    bits = uint32_t((w >> (k0 & 63)) & 0xffffu);
  }
  uint32_t v[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    uint32_t x = 0;
#pragma unroll
    for (int b = 0; b < 4; ++b) x |= ((bits >> (4 * q + b)) & 1u) ? (0x38u << (8 * b)) : 0u;
    v[q] = x;
  }
  *reinterpret_cast<uint4*>(img + tile * (int64_t(R) * KT * 64) + int64_t(katom) * R * 128 +
                            r * 128 + pos * 16) = make_uint4(v[0], v[1], v[2], v[3]);
}

// ---- tcgen05 wrappers ---------------------------------------------------------

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, atoms of
// 8 rows x 128 bytes stacked 1024 bytes apart (SBO); descriptor version 1.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= uint64_t((saddr & 0x3ffffu) >> 4);       // start address
  d |= uint64_t(1) << 16;                        // leading byte offset (unused here)
  d |= uint64_t(1024 >> 4) << 32;                // stride byte offset
  d |= uint64_t(1) << 46;                        // version
  d |= uint64_t(2) << 61;                        // 128-byte swizzle
  return d;
}

// Instruction descriptor, kind::f8f6f4: D F32, A and B E4M3, both K-major,
// N = kTcN, M = kTcM.
constexpr uint32_t kTcIdesc = (1u << 4) | (0u << 7) | (0u << 10) | (uint32_t(kTcN >> 3) << 17) |
                              (uint32_t(kTcM >> 4) << 24);

__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                       uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(kTcIdesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void tc_mma_desc(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                            uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void tc_commit(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.release.cta.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

// 32 consecutive accumulator columns of this thread's lane.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&v)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
        "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]),
        "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]),
        "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]),
        "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]),
        "=r"(v[31])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// 32 consecutive accumulator columns of this thread's lane, with their
// minimum as unsigned words (tcgen05.ld.red.min): the accumulators hold
// non-negative FP32 counts, so the minimum word is 0 exactly when one of the
// 32 counts is 0.
__device__ __forceinline__ void tmem_ld32_min(uint32_t taddr, uint32_t (&v)[32], uint32_t& mn) {
  asm volatile(
      "tcgen05.ld.red.sync.aligned.32x32b.x32.min.u32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, %32, [%33];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
        "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]),
        "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]),
        "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]),
        "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]),
        "=r"(v[31]), "=r"(mn)
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// This thread's lane, 32 consecutive columns from registers.  Completion is
// awaited with tmem_wait_st.
__device__ __forceinline__ void tmem_st32(uint32_t taddr, const uint32_t (&v)[32]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], "
      "{%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,"
      "%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32};" ::"r"(taddr),
      "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]),
      "r"(v[8]), "r"(v[9]), "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]),
      "r"(v[15]), "r"(v[16]), "r"(v[17]), "r"(v[18]), "r"(v[19]), "r"(v[20]), "r"(v[21]),
      "r"(v[22]), "r"(v[23]), "r"(v[24]), "r"(v[25]), "r"(v[26]), "r"(v[27]), "r"(v[28]),
      "r"(v[29]), "r"(v[30]), "r"(v[31])
      : "memory");
}

__device__ __forceinline__ void tmem_wait_st() {
  asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

// D (+)= A * B^T with A (M = 128 rows, one per lane, 4 E4M3 items per
// column in item order) in tensor memory and B described in shared memory.
__device__ __forceinline__ void tc_mma_tmem_a(uint32_t d_tmem, uint32_t a_tmem, uint64_t bdesc,
                                              uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], [%1], %2, %3, p;\n\t}" ::"r"(d_tmem),
      "r"(a_tmem), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

// ---- the kernel -------------------------------------------------------------

struct TcParams {
  const uint8_t* a_img;                 // own rows, tiles of kTcM
  int64_t n_own;
  const unsigned long long* n_own_dev;  // optional device-side own count
  const uint8_t* b_img;                 // stream rows, tiles of kTcN
  int64_t b_tile0;                      // first stream tile of this launch
  int64_t n_stream;                     // stream rows from tile b_tile0 on
  int64_t tiles_per_split;
  const uint64_t* score;                // MODE_SUM: S of stream row j (from b_tile0 * kTcN)
  uint32_t* out_u32;
  unsigned long long* out_u64;
  int* status;
};

template <int KT, int MODE>
__global__ void __launch_bounds__(kTcThreads, 1) subset_tc_kernel(TcParams p) {
  using S = TcShape<KT>;
  constexpr int STAGES = S::kStages;
  extern __shared__ uint8_t smem_raw[];
  const int64_t n_own = p.n_own_dev ? int64_t(*p.n_own_dev) : p.n_own;
  const int64_t own0 = int64_t(blockIdx.x) * kTcM;
  if (own0 >= n_own) return;
  const int64_t t_lo = int64_t(blockIdx.y) * p.tiles_per_split;
  const int64_t total_tiles = ceil_div(p.n_stream, kTcN);
  const int64_t t_hi = (t_lo + p.tiles_per_split < total_tiles) ? t_lo + p.tiles_per_split
                                                                 : total_tiles;
  const int ntiles = int(t_hi > t_lo ? t_hi - t_lo : 0);
  const int own_valid = int(n_own - own0 < kTcM ? n_own - own0 : kTcM);
  const int64_t str_first = t_lo * kTcN;            // stream rows of this CTA's tiles
  const int64_t str_count = p.n_stream - str_first;

  // 1024-byte aligned carve-up of dynamic shared memory.
  const uint32_t raw = smem_u32(smem_raw);
  uint8_t* base = smem_raw + ((1024u - (raw & 1023u)) & 1023u);
  uint8_t* A_s = base;
  uint8_t* B_s = A_s + S::kABytes;
  uint64_t* bars = reinterpret_cast<uint64_t*>(B_s + size_t(STAGES) * S::kBBytes);
  uint64_t* a_full = bars;
  uint64_t* full = bars + 1;
  uint64_t* empty = full + STAGES;
  uint64_t* acc_full = empty + STAGES;
  uint64_t* acc_empty = acc_full + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(acc_empty + 2);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    mbar_init(a_full, 1);
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(full + s, 1);
      mbar_init(empty + s, 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(acc_full + b, 1);
      mbar_init(acc_empty + b, 4);
    }
    *abort_flag = 0;
    fence_mbar_init();
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      // Producer: A once, then the B tiles through the ring.
      mbar_arrive_expect_tx(a_full, S::kABytes);
      bulk_g2s(A_s, p.a_img + size_t(blockIdx.x) * S::kABytes, S::kABytes, a_full);
      int issued = 0;
      for (int t = 0; t < ntiles; ++t) {
        const int s = t % STAGES;
        if (!mbar_wait(empty + s, uint32_t(((t / STAGES) & 1) ^ 1), p.status) || *abort_flag) {
          *abort_flag = 1;
          break;
        }
        mbar_arrive_expect_tx(full + s, S::kBBytes);
        bulk_g2s(B_s + size_t(s) * S::kBBytes,
                 p.b_img + size_t(p.b_tile0 + t_lo + t) * S::kBBytes, S::kBBytes, full + s);
        issued = t + 1;
      }
      // Copies must have landed before the CTA may finish.
      mbar_wait(a_full, 0, p.status);
      for (int t = (issued > STAGES ? issued - STAGES : 0); t < issued; ++t)
        if (*abort_flag) mbar_wait(full + (t % STAGES), uint32_t((t / STAGES) & 1), p.status);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // MMA issuer.
      bool ok = mbar_wait(a_full, 0, p.status);
      int last = -1;
      const uint32_t a_base = smem_u32(A_s);
      for (int t = 0; t < ntiles && ok; ++t) {
        const int s = t % STAGES, b = t & 1;
        if (!mbar_wait(full + s, uint32_t((t / STAGES) & 1), p.status) ||
            !mbar_wait(acc_empty + b, uint32_t(((t >> 1) & 1) ^ 1), p.status) || *abort_flag) {
          *abort_flag = 1;
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t b_base = smem_u32(B_s + size_t(s) * S::kBBytes);
        const uint32_t d = tmem + uint32_t(b * kTcN);
#pragma unroll 4
        for (int k = 0; k < S::kKSteps; ++k) {
          const uint32_t koff = uint32_t(k >> 2) * (kTcM * 128) + uint32_t(k & 3) * 32;
          const uint32_t kboff = uint32_t(k >> 2) * (kTcN * 128) + uint32_t(k & 3) * 32;
          tc_mma(d, sw128_desc(a_base + koff), sw128_desc(b_base + kboff), k > 0 ? 1u : 0u);
        }
        tc_commit(empty + s);     // stage reusable once these MMAs are done
        tc_commit(acc_full + b);  // accumulator b ready for the epilogue
        last = t;
      }
      // MMAs complete in order: once the last commit has arrived, no MMA of
      // this CTA is still writing tensor memory.
      if (last >= 0) mbar_wait(acc_full + (last & 1), uint32_t((last >> 1) & 1), p.status);
    }
  } else {
    // Epilogue: warp w reads accumulator lanes 32*(w % 4) .. +32.
    const int quarter = warp & 3;
    const int tile_row = quarter * 32 + lane;
    const bool valid = tile_row < own_valid;
    bool cov = false;
    uint32_t cnt = 0;
    unsigned long long sum = 0;
    for (int t = 0; t < ntiles; ++t) {
      const int b = t & 1;
      bool ok = mbar_wait(acc_full + b, uint32_t((t >> 1) & 1), p.status);
      if (!__all_sync(0xffffffffu, ok) || *abort_flag) {
        *abort_flag = 1;
        break;
      }
      tc_fence_after();
      const int64_t j0 = str_first + int64_t(t) * kTcN;  // first stream row of this tile
      const int64_t left = str_count - int64_t(t) * kTcN;
      const int nvalid = int(left < kTcN ? left : kTcN);
#pragma unroll 1
      for (int c = 0; c < kTcN; c += 32) {
        uint32_t v[32];
        tmem_ld32(tmem + (uint32_t(quarter * 32) << 16) + uint32_t(b * kTcN + c), v);
#pragma unroll
        for (int i = 0; i < 32; ++i) {
          const bool hit = v[i] == 0u && (c + i) < nvalid;
          if constexpr (MODE == MODE_ANY) cov |= hit;
          if constexpr (MODE == MODE_COUNT) cnt += hit ? 1u : 0u;
          if constexpr (MODE == MODE_SUM) {
            if (hit) sum += p.score[j0 + c + i];
          }
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(acc_empty + b);
    }
    if (valid) {
      const int64_t row = own0 + tile_row;
      if constexpr (MODE == MODE_ANY) {
        if (cov) p.out_u32[row] = 1u;
      }
      if constexpr (MODE == MODE_COUNT) {
        if (cnt) atomicAdd(p.out_u32 + row, cnt);
      }
      if constexpr (MODE == MODE_SUM) {
        if (sum) atomicAdd(p.out_u64 + row, sum);
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(kTmemCols)
                 : "memory");
  }
}

// ---- host side --------------------------------------------------------------

template <int KT>
static cudaError_t expand(const uint64_t* rows, int64_t n, int stride, int complement, int R,
                          uint8_t* img, cudaStream_t s) {
  static_assert(kTcM == kTcN, "one tile height for both operands");
  if (R != kTcM) return cudaErrorInvalidValue;
  const int64_t ntiles = ceil_div(n, kTcM);
  const int64_t chunks = ntiles * int64_t(kTcM) * KT * 4;
  if (chunks == 0) return cudaSuccess;
  expand_kernel<KT, kTcM><<<unsigned(ceil_div(chunks, 256)), 256, 0, s>>>(
      rows, n, stride, complement, ntiles, img);
  count_launches(1);
  return cudaGetLastError();
}

template <int KT, int MODE>
static cudaError_t run_tc(const TcArgs& a, cudaStream_t s) {
  using S = TcShape<KT>;
  const int64_t gx = ceil_div(a.n_own, kTcM);
  const int64_t stream_tiles = ceil_div(a.n_stream, kTcN);
  const int64_t target = int64_t(num_sms()) * 2;
  int64_t splits = ceil_div(target, gx);
  if (splits > stream_tiles) splits = stream_tiles;
  if (splits > 65535) splits = 65535;
  if (splits < 1) splits = 1;
  const int64_t per = ceil_div(stream_tiles, splits);
  splits = ceil_div(stream_tiles, per);
  TcParams p{a.a_img, a.n_own, a.n_own_dev, a.b_img,   a.b_tile0, a.n_stream, per,
             a.score, a.out_u32, a.out_u64,   a.status};
  cudaError_t e = cudaFuncSetAttribute(subset_tc_kernel<KT, MODE>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, int(S::kSmem));
  if (e != cudaSuccess) return e;
  dim3 grid{unsigned(gx), unsigned(splits), 1u};
  subset_tc_kernel<KT, MODE><<<grid, kTcThreads, S::kSmem, s>>>(p);
  count_launches(1);
  return cudaGetLastError();
}

bool tc_supported(int KT) { return KT == 2 || KT == 4 || KT == 8; }

size_t tc_image_bytes(int64_t n, int KT, bool own_side) {
  const int R = own_side ? kTcM : kTcN;
  return size_t(ceil_div(n, R)) * R * KT * 64;
}

cudaError_t launch_expand(const uint64_t* rows, int64_t n, int stride, int KT, bool complement,
                          bool own_side, uint8_t* img, cudaStream_t s) {
  const int R = own_side ? kTcM : kTcN;
  switch (KT) {
    case 2: return expand<2>(rows, n, stride, complement ? 1 : 0, R, img, s);
    case 4: return expand<4>(rows, n, stride, complement ? 1 : 0, R, img, s);
    case 8: return expand<8>(rows, n, stride, complement ? 1 : 0, R, img, s);
  }
  return cudaErrorInvalidValue;
}

// ---- item-index blocks on the tensor cores ----------------------------------
//
// subset_tc_fused_kernel: the same 0/1 GEMM on the item index's blocks, with
// no operand images in global memory.  Packed 64*KT-bit rows are copied by
// TMA into shared staging.  The resident rows of a work item (one item
// group's patterns, in every mode) are expanded to E4M3 bytes (0x08 = 2^-6
// per set bit, which takes one multiply fewer to spread than 1.0) and
// written into tensor memory, where the MMA reads its A operand; the
// streamed rows (the other class's records for coherence, the own class's
// records for support, the scored records for evidence) are expanded into
// swizzled shared-memory tiles of 128 rows (the B operand).  Evidence keeps
// two 128-row halves of patterns per item, so each expanded stream tile
// serves two MMA chains.  Each chain (a "unit": one tile, one half)
// accumulates into one of the 128-column slots of tensor memory, taken in
// turn, so the epilogue of one unit overlaps the MMAs of the next.  The grid
// is persistent: CTA b runs the items [cta_off[b], cta_off[b + 1]), lists
// balanced by the host, with its tensor memory allocated once; an item's
// class (its pad field) picks the resident rows, scores and outputs, so one
// launch scores records against both classes.  Warp roles:
//   warp 0     lane 0 issues the bulk copies of packed rows;
//   warp 1     allocates tensor memory; lane 0 issues the MMAs and commits;
//   warps 2-5  epilogue (and 6-9 for evidence, a second group; the groups
//              split every unit's columns): lanes of TMEM quarter w % 4;
//              per 32 columns one load that also returns their minimum,
//              then hit masks, the slot handed back, and the reduction: an
//              "any" for coherence, a count of zeros for support, and for
//              evidence a warp sum of the patterns' scores per hit record;
//   the rest   expand packed tiles into operand tiles.
// Every wait is bounded; a timeout sets the status and an abort flag that
// every role checks.

constexpr int kFusedThreads = 704;  // 22 warps
// Resident halves and stream-tile rows per work item, by mode: evidence
// keeps two 128-row halves of patterns, so that each expanded stream tile
// serves two MMA chains.
constexpr int fused_halves(int mode) { return mode == MODE_SUM ? 2 : 1; }
constexpr int fused_n(int mode) { return 128; }

template <int KT, int MODE>
struct FusedShape {
  static constexpr int kHalves = fused_halves(MODE);
  // Epilogue warps (4 per group, one per 32-lane quarter of tensor memory;
  // evidence has two groups, which split every unit's columns) and expander
  // warps (the rest of the 22 after the producer and the MMA issuer).
  static constexpr int kEpiWarps = 4 * kHalves;
  static constexpr int kExpWarps = kFusedThreads / 32 - 2 - kEpiWarps;
  static constexpr int kN = fused_n(MODE);                          // stream rows per tile
  static constexpr int kOwn = 128 * kHalves;                        // resident rows per item
  static constexpr uint32_t kImgB = uint32_t(kN) * KT * 64;        // one expanded stream tile
  static constexpr uint32_t kPkA = uint32_t(kOwn) * KT * 8;        // packed resident rows
  static constexpr uint32_t kPkB = uint32_t(kN) * KT * 8;          // one packed stream tile
  // MODE_SUM: each epilogue warp stages the record ids of its columns of
  // the current stream tile.
  static constexpr size_t kScores =
      MODE == MODE_SUM ? size_t(kEpiWarps) * (kN / (kEpiWarps / 4)) * 4 : 0;
  // Tensor memory (512 columns): accumulator buffers of 128 columns, then
  // the resident operand, 16*KT columns (4 items each) per half, twice where
  // it fits, so that the next item's rows can be written while the MMAs
  // still read the current ones.
  // Three accumulator buffers where they fit beside two resident buffers
  // (each buffer more gives the epilogue a whole unit of MMA time before
  // the issuer needs its slot back; a second resident buffer lets the next
  // item's rows be written while the MMAs still read the current ones,
  // which matters more where items are short), else two; then the second
  // resident buffer where the rest allows.
  static constexpr int kACols = 16 * KT;
  static constexpr int kAccBufs = 3 * 128 + 2 * kHalves * kACols <= 512 ? 3 : 2;
  static constexpr int kAccCols = 128 * kAccBufs;
  static constexpr int kABufs = kAccCols + 2 * kHalves * kACols <= 512 ? 2 : 1;
  static_assert(kAccCols + kABufs * kHalves * kACols <= 512, "tensor memory overflow");
  // Alignment slack, barriers, scores and the packed resident rows; the
  // rest of 227 KB goes to the rings of expanded (up to 4) and packed (up to
  // 8) stream tiles.  Packed tiles are small, so their ring runs deeper and
  // keeps more bulk copies in flight than the expanded ring.
  static constexpr int kFixed = 1024 + 512 + int(kScores) + int(kPkA);
  static constexpr int kBudget = 227 * 1024;
  static constexpr int kXFit = (kBudget - kFixed - 2 * int(kPkB)) / int(kImgB);
  static constexpr int kXStages = kXFit > 4 ? 4 : kXFit;
  static constexpr int kPkFit = (kBudget - kFixed - kXStages * int(kImgB)) / int(kPkB);
  static constexpr int kPkStages = kPkFit > 8 ? 8 : kPkFit;
  static_assert(kXStages >= 2 && kPkStages >= 2, "shared memory too small for two stages");
  // At least 120 KB, so that no two CTAs (which each take all 512 tensor
  // memory columns) share an SM.
  static constexpr size_t kUsed =
      size_t(kFixed) + size_t(kXStages) * kImgB + size_t(kPkStages) * kPkB;
  static constexpr size_t kSmem = kUsed > 120 * 1024 ? kUsed : 120 * 1024;
  static constexpr uint32_t kIdesc = (1u << 4) | (0u << 7) | (0u << 10) |
                                     (uint32_t(kN >> 3) << 17) | (uint32_t(128 >> 4) << 24);
};

constexpr uint32_t kFusedTmemCols = 512;

struct FusedParams {
  const TcItem* items;        // grouped by CTA: CTA b runs items [cta_off[b], cta_off[b + 1])
  int64_t n_items;
  const int64_t* cta_off;     // gridDim.x + 1 entries
  // Per class of resident rows (an item's class is its `pad` field: one
  // launch can score the records against both classes' patterns):
  const uint64_t* own_rows0;  // grouped rows of the resident side (stride KT)
  const uint64_t* own_rows1;
  const uint32_t* own_ids0;   // original id of each grouped resident row
  const uint32_t* own_ids1;
  const uint64_t* score0;     // MODE_SUM: S of each grouped resident row (pattern)
  const uint64_t* score1;
  unsigned long long* sum0;   // MODE_SUM: per-record sums (Eq. 4: A or N)
  unsigned long long* sum1;
  // MODE_SUM: 1 when every score of the class is below 2^27, so that the
  // sum of one column's hits over a warp's 32 patterns fits in 32 bits; 0:
  // every hit goes to its record by its own 64-bit atomic.
  int narrow0, narrow1;
  const uint64_t* str_rows;  // grouped rows of the streamed side (stride KT)
  int own_complement;        // 1: the resident side is the record side
  const uint32_t* str_ids;   // MODE_SUM: original id of each grouped streamed row (record)
  // Polls a wait for a full stage, a free stage or an accumulator may take
  // (0: kMbarPollLimit); the waits for copies and MMAs in flight before the
  // CTA ends always take the full limit.  And, for tests of the timeout
  // path, the unit before whose MMAs the issuer waits on a barrier that
  // never completes (-1: none).
  uint32_t poll_limit;
  int64_t stall_unit;
  uint32_t* out_u32;          // MODE_ANY / MODE_COUNT (one class)
  int* status;
};

// One E4M3 byte per bit of a 4-bit group (n < 16): 0x08 (2^-6) for a set
// bit, 0 otherwise.  The multiply places bit b of n at bit 8b + 3 (the four
// shifted copies of n, at bits 3-6, 10-13, 17-20 and 24-27, do not overlap)
// and the mask keeps those bits.  A product of two such bytes is 2^-12 and a
// row's at most 512 of them add up exactly in FP32, so D == 0 still means
// "no item in common".
__device__ __forceinline__ uint32_t spread_nibble(uint32_t n) {
  return (n * 0x01020408u) & 0x08080808u;
}

// Expands `count` packed rows (the rest zero) into one R-row operand tile in
// the swizzled K-major layout of expand_kernel (atoms of R rows x 128 bytes;
// chunk `pos` of row r in every atom holds the 16 items of logical chunk
// pos ^ (r mod 8)).  Thread e of n handles the (row, chunk) pairs e, e + n,
// ... of the R x 8 grid, in every atom: the source half-word and its shift
// are the same for all atoms of a pair, and the atoms' items sit 128 bits
// apart in the packed row.  Consecutive threads write consecutive chunks.
template <int KT, int R>
__device__ __forceinline__ void expand_tile_smem(const uint64_t* pk, int count, bool complement,
                                                 uint8_t* dst, int e, int n) {
  const uint32_t flip = complement ? 0xffffffffu : 0u;
#pragma unroll 1
  for (int id = e; id < R * 8; id += n) {
    const int r = id >> 3, pos = id & 7;
    const int sw = pos ^ (r & 7);
    const uint32_t* src = reinterpret_cast<const uint32_t*>(pk + r * KT) + (sw >> 1);
    const int sh = (sw & 1) * 16;
    uint8_t* d = dst + r * 128 + pos * 16;
    const bool live = r < count;
#pragma unroll
    for (int a = 0; a < KT / 2; ++a) {
      const uint32_t bits = live ? ((src[4 * a] ^ flip) >> sh) : 0u;
      *reinterpret_cast<uint4*>(d + a * (R * 128)) =
          make_uint4(spread_nibble(bits & 15u), spread_nibble((bits >> 4) & 15u),
                     spread_nibble((bits >> 8) & 15u), spread_nibble((bits >> 12) & 15u));
    }
  }
}

__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}


template <int KT, int MODE>
__global__ void __launch_bounds__(kFusedThreads, 1) subset_tc_fused_kernel(FusedParams p) {
  using S = FusedShape<KT, MODE>;
  constexpr int XS = S::kXStages, PKS = S::kPkStages;
  constexpr int kN = S::kN, kOwn = S::kOwn;
  constexpr int PKB = kN * KT;  // words of one packed stream tile
  constexpr int NX = S::kExpWarps, NE = S::kEpiWarps;
  constexpr int kFirstExp = 2 + NE;  // first expander warp
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  uint8_t* base = smem_raw + ((1024u - (raw & 1023u)) & 1023u);
  uint8_t* B_x = base;                          // XS tiles of kImgB
  uint64_t* A_pk = reinterpret_cast<uint64_t*>(B_x + size_t(XS) * S::kImgB);
  uint64_t* B_pk = A_pk + kOwn * KT;
  uint64_t* bars = B_pk + size_t(PKS) * PKB;
  uint64_t* a_pk_full = bars;
  uint64_t* a_pk_empty = bars + 1;
  uint64_t* a_x_full = bars + 2;   // [kABufs]
  uint64_t* a_x_empty = bars + 4;  // [kABufs]
  uint64_t* b_pk_full = bars + 6;
  uint64_t* b_pk_empty = b_pk_full + PKS;
  uint64_t* b_x_full = b_pk_empty + PKS;
  uint64_t* b_x_empty = b_x_full + XS;
  uint64_t* acc_full = b_x_empty + XS;
  uint64_t* acc_empty = acc_full + S::kAccBufs;
  uint64_t* never = acc_empty + S::kAccBufs;  // no thread ever arrives on it
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(never + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t it_lo = p.cta_off[blockIdx.x], it_hi = p.cta_off[blockIdx.x + 1];
  const uint32_t lim = p.poll_limit ? p.poll_limit : kMbarPollLimit;
  // MODE_SUM: this warp's record ids for its columns of the current stream
  // tile (after the barriers' 512 bytes).
  constexpr int NG = NE / 4;      // epilogue groups; each takes kCols columns of every unit
  constexpr int kCols = kN / NG;
  uint32_t* sid = reinterpret_cast<uint32_t*>(bars + 64) + (warp >= 2 ? warp - 2 : 0) % NE * kCols;
  if (threadIdx.x == 0) {
    mbar_init(a_pk_full, 1);
    mbar_init(a_pk_empty, NX);
    for (int b = 0; b < S::kABufs; ++b) {
      mbar_init(a_x_full + b, NX);
      mbar_init(a_x_empty + b, 1);
    }
    for (int s = 0; s < PKS; ++s) {
      mbar_init(b_pk_full + s, 1);
      mbar_init(b_pk_empty + s, NX);
    }
    for (int s = 0; s < XS; ++s) {
      mbar_init(b_x_full + s, NX);
      mbar_init(b_x_empty + s, 1);
    }
    for (int b = 0; b < S::kAccBufs; ++b) {
      mbar_init(acc_full + b, 1);
      mbar_init(acc_empty + b, NE);  // every epilogue warp reads every unit
    }
    mbar_init(never, 1);
    *abort_flag = 0;
    fence_mbar_init();
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(kFusedTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      // Producer of packed tiles.
      int64_t tt = 0, ii = 0, issued_b = 0, issued_a = 0;
      auto tile_src = [&](const TcItem& w, int t) {
        return p.str_rows + (w.str_first + int64_t(t) * kN) * KT;
      };
      auto tile_bytes = [&](const TcItem& w, int t) {
        const int64_t left = int64_t(w.str_count) - int64_t(t) * kN;
        return uint32_t(left < kN ? left : kN) * KT * 8;
      };
      for (int64_t it = it_lo; it < it_hi && !*abort_flag; ++it, ++ii) {
        const TcItem w = p.items[it];
        if (!mbar_wait(a_pk_empty, uint32_t((ii & 1) ^ 1), p.status, lim)) {
          *abort_flag = 1;
          break;
        }
        const uint32_t abytes = uint32_t(w.own_count) * KT * 8;
        mbar_arrive_expect_tx(a_pk_full, abytes);
        bulk_g2s(A_pk, (w.pad ? p.own_rows1 : p.own_rows0) + w.own_first * KT, abytes,
                 a_pk_full);
        ++issued_a;
        for (int t = 0; t < w.b_tiles; ++t, ++tt) {
          const int s = int(tt % PKS);
          if (!mbar_wait(b_pk_empty + s, uint32_t(((tt / PKS) & 1) ^ 1), p.status, lim) ||
              *abort_flag) {
            *abort_flag = 1;
            break;
          }
          const uint32_t bytes = tile_bytes(w, t);
          mbar_arrive_expect_tx(b_pk_full + s, bytes);
          bulk_g2s(B_pk + size_t(s) * PKB, tile_src(w, t), bytes, b_pk_full + s);
          issued_b = tt + 1;
        }
      }
      if (*abort_flag) {
        // Copies in flight must land before the CTA may finish: the last
        // resident copy (the k-th completes phase k of a_pk_full) and the
        // stream copies of the last PKS tiles (earlier ones have been
        // consumed, or their stage could not have been reused).
        if (issued_a) mbar_wait(a_pk_full, uint32_t((issued_a - 1) & 1), p.status);
        for (int64_t t = (issued_b > PKS ? issued_b - PKS : 0); t < issued_b; ++t)
          mbar_wait(b_pk_full + (t % PKS), uint32_t((t / PKS) & 1), p.status);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // MMA issuer: per stream tile, one MMA chain per resident half (a
      // "unit"), the resident operand read from tensor memory.  Units take
      // the accumulator slots in turn, so the epilogue of one unit overlaps
      // the MMAs of the next.
      int64_t tt = 0, ii = 0, uu = 0;
      int64_t bx_last = -1, ax_last = -1;  // last tile / item whose stage / rows were released
      bool ok = true;
      for (int64_t it = it_lo; it < it_hi && ok; ++it, ++ii) {
        const TcItem w = p.items[it];
        const int halves = w.own_count > 128 ? 2 : 1;
        const int ab = S::kABufs == 2 ? int(ii & 1) : 0;
        const uint32_t aph = uint32_t((S::kABufs == 2 ? (ii >> 1) : ii) & 1);
        if (!mbar_wait(a_x_full + ab, aph, p.status, lim) || *abort_flag) {
          *abort_flag = 1;
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t a_tm = tmem + uint32_t(S::kAccCols + ab * S::kHalves * S::kACols);
        for (int t = 0; t < w.b_tiles && ok; ++t, ++tt) {
          const int s = int(tt % XS);
          // (The abort flag is read only at item boundaries: on an abort the
          // other roles stop, so this issuer's own bounded waits end too.)
          if (!mbar_wait(b_x_full + s, uint32_t((tt / XS) & 1), p.status, lim)) {
            *abort_flag = 1;
            ok = false;
            break;
          }
          // The descriptor's start address field is the byte address / 16, so
          // a K step's offset is added to it directly.
          const uint64_t bdesc = sw128_desc(smem_u32(B_x + size_t(s) * S::kImgB));
          for (int h = 0; h < halves; ++h, ++uu) {
            const int b = int(uu % S::kAccBufs);
            if ((uu == p.stall_unit && !mbar_wait(never, 0, p.status, lim)) ||
                !mbar_wait(acc_empty + b, uint32_t(((uu / S::kAccBufs) & 1) ^ 1), p.status, lim)) {
              *abort_flag = 1;
              ok = false;
              break;
            }
            tc_fence_after();
            const uint32_t d = tmem + uint32_t(b * 128);
            const uint32_t ah = a_tm + uint32_t(h * S::kACols);
#pragma unroll
            for (int k = 0; k < KT * 2; ++k) {
              // K step k: items 32k .. 32k + 31, resident columns 8k .. 8k + 7.
              const uint32_t boff = uint32_t(k >> 2) * (kN * 128) + uint32_t(k & 3) * 32;
              tc_mma_tmem_a(d, ah + uint32_t(8 * k), bdesc + uint64_t(boff >> 4), S::kIdesc,
                            k > 0 ? 1u : 0u);
            }
            tc_commit(acc_full + b);
          }
          if (!ok) break;
          tc_commit(b_x_empty + s);
          bx_last = tt;
        }
        if (!ok) break;
        tc_commit(a_x_empty + ab);  // the resident rows are free once this item's MMAs are done
        ax_last = ii;
      }
      // Before the CTA may finish, every MMA must be done (the last commit
      // to an accumulator) and every commit's arrival must have landed on
      // its barrier (the last stage and resident releases).
      if (uu > 0)
        mbar_wait(acc_full + ((uu - 1) % S::kAccBufs), uint32_t(((uu - 1) / S::kAccBufs) & 1),
                  p.status);
      if (bx_last >= 0)
        mbar_wait(b_x_empty + (bx_last % XS), uint32_t((bx_last / XS) & 1), p.status);
      if (ax_last >= 0)
        mbar_wait(a_x_empty + (S::kABufs == 2 ? int(ax_last & 1) : 0),
                  uint32_t((S::kABufs == 2 ? (ax_last >> 1) : ax_last) & 1), p.status);
    }
  } else if (warp < kFirstExp) {
    // Epilogue: warp w reads accumulator lanes 32*(w % 4) .. +32 (resident
    // rows quarter*32 + lane of the unit's half).  The NG groups of four
    // warps split every unit's columns -- group g reads columns [g*kCols,
    // (g+1)*kCols) -- so that each warp holds an accumulator slot for fewer
    // loads and the slot returns to the MMA issuer sooner.
    const int quarter = warp & 3;
    const int tile_row = quarter * 32 + lane;
    const int grp = (warp - 2) >> 2;
    const int col0 = grp * kCols;
    int64_t uu = 0;
    bool ok = true;
    for (int64_t it = it_lo; it < it_hi && ok; ++it) {
      const TcItem w = p.items[it];
      const int halves = w.own_count > 128 ? 2 : 1;
      const bool narrow = w.pad ? p.narrow1 != 0 : p.narrow0 != 0;
      unsigned long long* const out_sum = w.pad ? p.sum1 : p.sum0;
      // This lane's resident row in each half; rows past the item's are zero
      // operands (D = 0 against everything) and take no part.
      bool live[2];
      unsigned long long own_s[2] = {0ull, 0ull};
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        live[h] = h < halves && h * 128 + tile_row < w.own_count;
        if constexpr (MODE == MODE_SUM)
          if (live[h]) own_s[h] = (w.pad ? p.score1 : p.score0)[w.own_first + h * 128 + tile_row];
      }
      bool cov0 = false, cov1 = false;
      uint32_t cnt0 = 0, cnt1 = 0;
      for (int t = 0; t < w.b_tiles && ok; ++t) {
        const int64_t left = int64_t(w.str_count) - int64_t(t) * kN;
        const int nvalid = int(left < kN ? left : kN);
        // MODE_SUM: record ids of this warp's columns of the tile, lane i
        // holding those of columns col0 + i + 32q (which it adds to when the
        // warp sums a column's hits): loads issued before the wait for the
        // accumulator and first needed only by a hit, so their latency hides
        // behind the wait.  With wide sums (scores beyond 2^27) any lane may
        // need any column's id: those are staged in shared memory (once
        // every lane is done with the last tile's).
        uint32_t rid[kCols / 32];
        if constexpr (MODE == MODE_SUM) {
          const int64_t j0 = w.str_first + int64_t(t) * kN + col0;
#pragma unroll
          for (int q = 0; q < kCols / 32; ++q) {
            const int j = lane + 32 * q;
            rid[q] = col0 + j < nvalid ? p.str_ids[j0 + j] : 0u;
          }
          if (!narrow) {
            __syncwarp();
#pragma unroll
            for (int q = 0; q < kCols / 32; ++q) sid[lane + 32 * q] = rid[q];
            __syncwarp();
          }
        }
        for (int h = 0; h < halves; ++h, ++uu) {
          const int b = int(uu % S::kAccBufs);
          const bool got =
              mbar_wait(acc_full + b, uint32_t((uu / S::kAccBufs) & 1), p.status, lim);
          if (!__all_sync(0xffffffffu, got) || *abort_flag) {
            *abort_flag = 1;
            ok = false;
            break;
          }
          tc_fence_after();
          // Two phases.  While the unit holds its accumulator slot: per 32
          // columns one load with the columns' minimum and, where a lane's
          // chunk holds a hit, that lane's 32-bit hit mask -- a chunk whose
          // minimum is non-zero holds no hit (no count is 0), and columns
          // past the tile's rows (zero rows give D = 0) are not hits.  The
          // slot goes back to the MMA issuer after this warp's last load;
          // the masks are reduced after that, so that the sums and atomics
          // of the hits (about one test in 600 at NSL-KDD shape) do not
          // hold the slot.
          constexpr int NQ = kCols / 32;
          uint32_t hm[NQ];
#pragma unroll
          for (int q = 0; q < NQ; ++q) {
            const int c = col0 + 32 * q;
            uint32_t v[32], mn;
            __syncwarp();  // the lanes that built a mask rejoin before the load
            tmem_ld32_min(tmem + (uint32_t(quarter * 32) << 16) + uint32_t(b * 128 + c), v, mn);
            if (q == NQ - 1) {
              tc_fence_before();
              __syncwarp();
              if (lane == 0) mbar_arrive(acc_empty + b);
            }
            const bool tail = c + 32 > nvalid;
            uint32_t m = 0;
            if (live[h] && (mn == 0u || tail)) {
              if (MODE == MODE_ANY && !tail) {
                m = 1u;  // a hit somewhere: all that coherence needs
              } else {
#pragma unroll
                for (int i = 0; i < 32; ++i) m |= (v[i] == 0u ? 1u : 0u) << i;
                if (tail) {
                  const int r = nvalid - c;
                  m &= r <= 0 ? 0u : (1u << r) - 1u;
                }
              }
            }
            hm[q] = m;
          }
          __syncwarp();
          bool cov = false;
          uint32_t cnt = 0;
#pragma unroll
          for (int q = 0; q < NQ; ++q) {
            const uint32_t m = hm[q];
            if constexpr (MODE == MODE_ANY) cov |= m != 0u;
            if constexpr (MODE == MODE_COUNT) cnt += uint32_t(__popc(m));
            if constexpr (MODE == MODE_SUM) {
              // Eq. 4: every record holding a pattern gains its score.
              if (!__any_sync(0xffffffffu, m != 0u)) continue;
              const int c = col0 + 32 * q;
              const unsigned long long sv = own_s[h];
              if (narrow) {
                // Per column that any lane hit, the warp sums its patterns'
                // scores, and lane i adds column i's total to its record:
                // one atomic per (record, chunk) instead of one per hit, so
                // that the patterns of a record do not queue on its address.
                // Four columns per round: their warp sums are independent and
                // overlap.
                uint32_t cols = __reduce_or_sync(0xffffffffu, m);
                uint32_t mine = 0;
                while (cols) {
                  int i[4];
#pragma unroll
                  for (int k = 0; k < 4; ++k) {
                    i[k] = cols ? __ffs(cols) - 1 : 32;
                    cols &= cols - 1u;
                  }
                  uint32_t tot[4];
#pragma unroll
                  for (int k = 0; k < 4; ++k)
                    tot[k] = __reduce_add_sync(
                        0xffffffffu, (i[k] < 32 && ((m >> i[k]) & 1u)) ? uint32_t(sv) : 0u);
#pragma unroll
                  for (int k = 0; k < 4; ++k) mine = lane == i[k] ? tot[k] : mine;
                }
                if (mine) atomicAdd(out_sum + rid[q], (unsigned long long)mine);
              } else {
                // Straight to the records, four hits per round so that their
                // id loads and atomics overlap.
                const uint32_t* ids = sid + (c - col0);
                uint32_t mm = m;
                while (mm) {
                  int i[4];
#pragma unroll
                  for (int k = 0; k < 4; ++k) {
                    i[k] = mm ? __ffs(mm) - 1 : -1;
                    mm &= mm - 1u;
                  }
                  uint32_t r[4];
#pragma unroll
                  for (int k = 0; k < 4; ++k) r[k] = i[k] >= 0 ? ids[i[k]] : 0u;
#pragma unroll
                  for (int k = 0; k < 4; ++k)
                    if (i[k] >= 0) atomicAdd(out_sum + r[k], sv);
                }
              }
            }
          }
          if (h == 0) {
            cov0 |= cov;
            cnt0 += cnt;
          } else {
            cov1 |= cov;
            cnt1 += cnt;
          }
        }
      }
      if (!ok) break;
      if constexpr (MODE != MODE_SUM) {
        for (int h = 0; h < halves; ++h) {
          if (!live[h]) continue;
          const int64_t row =
              int64_t((w.pad ? p.own_ids1 : p.own_ids0)[w.own_first + h * 128 + tile_row]);
          if constexpr (MODE == MODE_ANY) {
            if (h == 0 ? cov0 : cov1) p.out_u32[row] = 1u;
          }
          if constexpr (MODE == MODE_COUNT) {
            const uint32_t c = h == 0 ? cnt0 : cnt1;
            if (c) atomicAdd(p.out_u32 + row, c);
          }
        }
      }
    }
  } else {
    // Expanders.
    const int e = threadIdx.x - kFirstExp * 32;
    int64_t tt = 0, ii = 0;
    bool ok = true;
    for (int64_t it = it_lo; it < it_hi && ok; ++it, ++ii) {
      const TcItem w = p.items[it];
      const int ab = S::kABufs == 2 ? int(ii & 1) : 0;
      const uint32_t aph = uint32_t((S::kABufs == 2 ? (ii >> 1) : ii) & 1);
      bool got = mbar_wait(a_pk_full, uint32_t(ii & 1), p.status, lim) &&
                 mbar_wait(a_x_empty + ab, aph ^ 1u, p.status, lim);
      if (!__all_sync(0xffffffffu, got) || *abort_flag) {
        *abort_flag = 1;
        break;
      }
      tc_fence_after();
      // Resident rows into tensor memory: warp w writes lanes 32*(w % 4)
      // .. +32 (the rows of that quarter of each half), one 32-column block
      // (128 items) at a time; the four warps of a quarter share its blocks.
      {
        const int quarter = warp & 3, wq = (warp - kFirstExp) >> 2;
        constexpr int kBlocksPerHalf = KT / 2;
        const uint32_t flip = p.own_complement ? 0xffffffffu : 0u;
        for (int blk = wq; blk < S::kHalves * kBlocksPerHalf; blk += NX / 4) {
          const int h = blk / kBlocksPerHalf, cb = blk % kBlocksPerHalf;
          const int r = h * 128 + quarter * 32 + lane;
          uint32_t x[4] = {0u, 0u, 0u, 0u};
          if (r < w.own_count) {
            const uint4 q4 = *reinterpret_cast<const uint4*>(A_pk + r * KT + 2 * cb);
            x[0] = q4.x ^ flip;
            x[1] = q4.y ^ flip;
            x[2] = q4.z ^ flip;
            x[3] = q4.w ^ flip;
          }
          uint32_t v[32];
#pragma unroll
          for (int j = 0; j < 32; ++j) v[j] = spread_nibble((x[j >> 3] >> (4 * (j & 7))) & 15u);
          tmem_st32(tmem + (uint32_t(quarter * 32) << 16) +
                        uint32_t(S::kAccCols + (ab * S::kHalves + h) * S::kACols + cb * 32),
                    v);
        }
        tmem_wait_st();
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) {
        mbar_arrive(a_pk_empty);
        mbar_arrive(a_x_full + ab);
      }
      for (int t = 0; t < w.b_tiles; ++t, ++tt) {
        const int sp = int(tt % PKS), sx = int(tt % XS);
        got = mbar_wait(b_pk_full + sp, uint32_t((tt / PKS) & 1), p.status, lim) &&
              mbar_wait(b_x_empty + sx, uint32_t(((tt / XS) & 1) ^ 1), p.status, lim);
        if (!__all_sync(0xffffffffu, got) || *abort_flag) {
          *abort_flag = 1;
          ok = false;
          break;
        }
        const int64_t left = int64_t(w.str_count) - int64_t(t) * kN;
        expand_tile_smem<KT, kN>(B_pk + size_t(sp) * PKB, int(left < kN ? left : kN),
                                 p.own_complement == 0, B_x + size_t(sx) * S::kImgB, e,
                                 NX * 32);
        fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0) {
          mbar_arrive(b_pk_empty + sp);
          mbar_arrive(b_x_full + sx);
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(kFusedTmemCols)
                 : "memory");
  }
}

template <int KT, int MODE>
static cudaError_t run_fused(const FusedParams& p, cudaStream_t s) {
  using S = FusedShape<KT, MODE>;
  cudaError_t e = cudaFuncSetAttribute(subset_tc_fused_kernel<KT, MODE>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, int(S::kSmem));
  if (e != cudaSuccess) return e;
  // One CTA per SM: the items' CTA lists (cta_off) are made for that many.
  subset_tc_fused_kernel<KT, MODE><<<unsigned(num_sms()), kFusedThreads, S::kSmem, s>>>(p);
  count_launches(1);
  return cudaGetLastError();
}

namespace {
// Test hook: IG_EVIDENCE_WIDE_SUMS=1 in the environment makes the evidence
// kernel add every hit to its record with a 64-bit atomic even where the
// scores would allow 32-bit warp sums per record, so that tests can check
// that path on ordinary data (both give the same sums).
bool force_wide_sums() {
  const char* v = std::getenv("IG_EVIDENCE_WIDE_SUMS");
  return v && v[0] == '1';
}

// Test hook for the timeout path: IG_TEST_STALL_UNIT=u makes every CTA of
// the fused kernel wait, before the MMAs of its u-th unit, on a barrier that
// never completes, with the stage and accumulator waits limited to a few
// polls, so that the kernel reports ST_TIMEOUT, drains the copies and MMAs
// it has in flight and ends.  Unset (the default): no stall.
void test_stall(uint32_t* poll_limit, int64_t* stall_unit) {
  *poll_limit = 0;
  *stall_unit = -1;
  const char* v = std::getenv("IG_TEST_STALL_UNIT");
  if (!v || !*v) return;
  *stall_unit = std::strtoll(v, nullptr, 10);
  *poll_limit = 64;
}

}  // namespace

// ---- work items, built on the device --------------------------------------
//
// The fused kernel's work items are (class, item group, resident tile of
// own_rows patterns, range of `per` stream tiles of 128 records), `per` set
// so that there are about eight items per SM.  Two kernels build them from
// the indexes' group offsets on the device -- no read-back, no host work,
// no copy: one CTA plans (sizes, offsets, cost classes, CTA lists), then one
// thread per item places it.  Items are dealt to the CTAs of the persistent
// grid: sorted by cost
// (stream tiles x halves + 2, in kCostBuckets classes, largest first), in
// snake order (CTAs 0 .. G-1, then G-1 .. 0, ...), so that every CTA runs a
// contiguous list, largest items first, with about equal totals.  The order
// of the items does not change any result (flags, counts and sums are
// order-independent integers).
constexpr int kItemThreads = 1024;
constexpr int kItemMaxL = 1024;   // items per index (64 K, K <= 16)
constexpr int kItemMaxGrid = 1024;
constexpr int kCostBuckets = 64;

struct ItemBuild {
  const uint32_t* own_off[2];  // keyed (pattern) group offsets per class
  const uint32_t* str_off;     // record group offsets
  int n_cls, L, own_rows, grid;
  int64_t max_items;
  TcItem* items;               // [max_items]
  int64_t* cta_off;            // [grid + 1]
  unsigned long long* tests;   // [n_cls]: (pattern, record) pairs met, per class
  int* status;
  // Passed from the plan kernel to the placement kernel:
  int64_t* goff;               // [2 L + 1] first item of each (class, group)
  uint32_t* boff;              // [kCostBuckets] first sorted position of each cost class
  uint32_t* bcnt;              // [kCostBuckets] positions taken so far
  int64_t* meta;               // [2]: item count, stream tiles per range (per)
};

// Cost class of an item (stream tiles x halves + 2, largest first).
__device__ __forceinline__ int cost_bucket(int64_t b_tiles, int64_t own_count, int64_t per) {
  const int64_t cmax = 2 * per + 2;
  const int64_t cost = b_tiles * (own_count > 128 ? 2 : 1) + 2;
  return int((cmax - cost) * kCostBuckets / (cmax + 1));
}

__device__ __forceinline__ int64_t div_up(int64_t a, int64_t b) { return (a + b - 1) / b; }

// Exclusive scan of v[0, n) in place (v[n] = total), by one block of at
// most 1,024 threads: a chunk of consecutive entries per thread, the chunk
// sums scanned by warp shuffles and then across the warps (part: 32 words).
template <class V>
__device__ void block_exclusive_scan(V* v, int n, V* part) {
  const int T = blockDim.x, t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int chunk = (n + T - 1) / T;
  const int lo = t * chunk, hi = lo + chunk < n ? lo + chunk : n;
  V sum = 0;
  for (int i = lo; i < hi; ++i) sum += v[i];
  V inc = sum;  // inclusive scan of the chunk sums within the warp
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const V x = __shfl_up_sync(0xffffffffu, inc, d);
    if (lane >= d) inc += x;
  }
  if (lane == 31) part[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    const int nw = (T + 31) >> 5;
    V w = lane < nw ? part[lane] : V(0);
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const V x = __shfl_up_sync(0xffffffffu, w, d);
      if (lane >= d) w += x;
    }
    if (lane < nw) part[lane] = w;  // inclusive over the warps
  }
  __syncthreads();
  V run = (warp ? part[warp - 1] : V(0)) + inc - sum;
  for (int i = lo; i < hi; ++i) {
    const V x = v[i];
    v[i] = run;
    run += x;
  }
  if (t == T - 1) v[n] = part[((T + 31) >> 5) - 1];
  __syncthreads();
}

// The plan, by one CTA: sizes, the items of each (class, group) and their
// offsets, the cost classes' sizes (per group in closed form: only a
// group's last resident tile and last stream range differ from the others)
// and offsets, and the CTA lists' offsets.
__global__ void __launch_bounds__(kItemThreads) tc_items_plan_kernel(ItemBuild b) {
  __shared__ uint32_t s_ob[2][kItemMaxL + 1];
  __shared__ uint32_t s_sb[kItemMaxL + 1];
  __shared__ int64_t s_off[2 * kItemMaxL + 1];
  __shared__ int64_t s_cta[kItemMaxGrid + 1];
  __shared__ int64_t s_part[32];
  __shared__ uint32_t s_hist[kCostBuckets];
  __shared__ unsigned long long s_tiles, s_tests[2];
  const int L = b.L, G = b.grid, t = threadIdx.x, T = blockDim.x;
  const int own_rows = b.own_rows, ng = b.n_cls * L;
  if (t == 0) {
    s_tiles = 0;
    s_tests[0] = s_tests[1] = 0;
  }
  for (int i = t; i < kCostBuckets; i += T) {
    s_hist[i] = 0;
    b.bcnt[i] = 0;
  }
  for (int l = t; l <= L; l += T) {
    s_sb[l] = b.str_off[l];
    for (int c = 0; c < b.n_cls; ++c) s_ob[c][l] = b.own_off[c][l];
  }
  __syncthreads();
  unsigned long long tiles = 0, tests[2] = {0, 0};
  for (int l = t; l < L; l += T) {
    const uint32_t ns = s_sb[l + 1] - s_sb[l];
    for (int c = 0; c < b.n_cls; ++c) {
      const uint32_t no = s_ob[c][l + 1] - s_ob[c][l];
      if (no && ns) {
        tiles += uint64_t(div_up(no, own_rows)) * uint64_t(div_up(ns, 128));
        tests[c] += uint64_t(no) * ns;
      }
    }
  }
  if (tiles) atomicAdd(&s_tiles, tiles);
  if (tests[0]) atomicAdd(&s_tests[0], tests[0]);
  if (tests[1]) atomicAdd(&s_tests[1], tests[1]);
  __syncthreads();
  const int64_t per_raw = int64_t(s_tiles) / (int64_t(G) * 8);
  const int64_t per = per_raw > 1 ? per_raw : 1;
  for (int g = t; g < ng; g += T) {
    const int c = g / L, l = g - c * L;
    const int64_t no = s_ob[c][l + 1] - s_ob[c][l], ns = s_sb[l + 1] - s_sb[l];
    int64_t items = 0;
    if (no && ns) {
      const int64_t A = div_up(no, own_rows), nb = div_up(ns, 128), nbp = div_up(nb, per);
      items = A * nbp;
      const int64_t rem_o = no - (A - 1) * own_rows, rem_b = nb - (nbp - 1) * per;
      if (A > 1 && nbp > 1)
        atomicAdd(&s_hist[cost_bucket(per, own_rows, per)], uint32_t((A - 1) * (nbp - 1)));
      if (A > 1) atomicAdd(&s_hist[cost_bucket(rem_b, own_rows, per)], uint32_t(A - 1));
      if (nbp > 1) atomicAdd(&s_hist[cost_bucket(per, rem_o, per)], uint32_t(nbp - 1));
      atomicAdd(&s_hist[cost_bucket(rem_b, rem_o, per)], 1u);
    }
    s_off[g] = items;
  }
  __syncthreads();
  block_exclusive_scan(s_off, ng, s_part);
  const int64_t n_items = s_off[ng];
  const bool fits = n_items <= b.max_items;  // always, with the host's bound
  if (t < 32) {  // exclusive scan of the cost classes' sizes by one warp
    const uint32_t a0 = s_hist[2 * t], a1 = s_hist[2 * t + 1];
    uint32_t inc = a0 + a1;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const uint32_t x = __shfl_up_sync(0xffffffffu, inc, d);
      if (t >= d) inc += x;
    }
    const uint32_t ex = inc - a0 - a1;
    b.boff[2 * t] = ex;
    b.boff[2 * t + 1] = ex + a0;
  }
  // CTA lists: the sorted item s goes to round s / G, CTA s % G in even
  // rounds and G - 1 - s % G in odd ones; a CTA's list holds one item per
  // round it takes part in.
  const int64_t R = fits ? n_items / G : 0, rem = fits ? n_items - R * G : 0;
  for (int g = t; g < G; g += T)
    s_cta[g] = R + (((R & 1) == 0) ? (g < rem ? 1 : 0) : (g >= G - rem ? 1 : 0));
  __syncthreads();
  block_exclusive_scan(s_cta, G, s_part);
  for (int i = t; i <= G; i += T) b.cta_off[i] = s_cta[i];
  for (int i = t; i <= ng; i += T) b.goff[i] = s_off[i];
  if (t < b.n_cls) b.tests[t] = s_tests[t];
  if (t == 0) {
    if (!fits) set_status(b.status, ST_COUNT);
    b.meta[0] = fits ? n_items : 0;  // nothing is placed past the bound
    b.meta[1] = per;
  }
}

// The placement, one thread per item: item k of its (class, group), its
// position among the items sorted by cost class, and its place in its CTA's
// list.
__global__ void tc_items_place_kernel(ItemBuild b) {
  const int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  const int64_t n_items = b.meta[0];
  if (k >= n_items) return;
  const int64_t per = b.meta[1];
  const int L = b.L, G = b.grid, own_rows = b.own_rows, ng = b.n_cls * L;
  int lo = 0, hi = ng - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (b.goff[mid] <= k) lo = mid; else hi = mid - 1;
  }
  const int c = lo / L, l = lo - c * L;
  const int64_t o0 = b.own_off[c][l], s0 = b.str_off[l];
  const int64_t no = int64_t(b.own_off[c][l + 1]) - o0, ns = int64_t(b.str_off[l + 1]) - s0;
  const int64_t nb = div_up(ns, 128), nbp = div_up(nb, per), j = k - b.goff[lo];
  const int64_t a = j / nbp, bs = (j - a * nbp) * per;
  TcItem it;
  it.own_first = o0 + a * own_rows;
  it.str_first = s0 + bs * 128;
  it.own_count = int32_t(min(int64_t(own_rows), no - a * own_rows));
  it.b_tiles = int32_t(min(per, nb - bs));
  it.str_count = int32_t(min(per * 128, ns - bs * 128));
  it.pad = c;
  const int bk = cost_bucket(it.b_tiles, it.own_count, per);
  const int64_t sp = int64_t(b.boff[bk]) + atomicAdd(b.bcnt + bk, 1u);
  const int64_t round = sp / G, kk = sp - round * G;
  const int64_t cta = (round & 1) ? G - 1 - kk : kk;
  b.items[b.cta_off[cta] + round] = it;
}

cudaError_t indexed_subset_tc_classes(int mode, const RecordIndex& idx, const KeyedIndex* const* kx,
                                      int n_cls, uint32_t* out_u32,
                                      unsigned long long* const* out_sum, int* status,
                                      int64_t* tests_out, int prof_stage,
                                      const uint64_t* score_max, cudaStream_t s) {
  const int L = idx.L, KT = idx.KT;
  if (n_cls < 1 || n_cls > 2 || (n_cls == 2 && mode != MODE_SUM)) return cudaErrorInvalidValue;
  if (idx.n_rows == 0 || !tc_supported(KT) || L > kItemMaxL) return cudaErrorInvalidValue;
  // Patterns (keyed) are resident and records (multi, complemented) stream,
  // in every mode: an item group holds far fewer patterns than records, so
  // items are long (about 90 stream tiles at NSL-KDD shape, against 6-9 with
  // the records resident) and the resident rows are expanded 10-15x less
  // often.  ANY / COUNT results stay per resident row; SUM adds each
  // pattern's score to the records containing it.  With two classes (SUM),
  // both classes' items share one launch, one schedule and one tail.
  const int G = num_sms();
  if (G > kItemMaxGrid) return cudaErrorInvalidValue;
  const int64_t own_rows = 128 * fused_halves(mode);
  // At most 16 G items beyond one per (class, group, resident tile).
  int64_t max_items = 16 * int64_t(G);
  for (int c = 0; c < n_cls; ++c) max_items += ceil_div(kx[c]->n, own_rows) + L + 1;
  const size_t item_bytes = size_t(max_items) * sizeof(TcItem);
  const size_t bytes = item_bytes + size_t(G + 1) * 8 + size_t(n_cls) * 8 +
                       size_t(2 * L + 1) * 8 + 2 * 8 + 2 * size_t(kCostBuckets) * 4;
  uint8_t* blk = nullptr;
  cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&blk), bytes, s);
  if (e != cudaSuccess) return e;
  TcItem* d_items = reinterpret_cast<TcItem*>(blk);
  int64_t* d_cta = reinterpret_cast<int64_t*>(blk + item_bytes);
  unsigned long long* d_tests = reinterpret_cast<unsigned long long*>(d_cta + G + 1);
  int64_t* d_goff = reinterpret_cast<int64_t*>(d_tests + n_cls);
  int64_t* d_meta = d_goff + (2 * L + 1);
  uint32_t* d_boff = reinterpret_cast<uint32_t*>(d_meta + 2);
  ItemBuild ib;
  ib.own_off[0] = kx[0]->off;
  ib.own_off[1] = kx[n_cls - 1]->off;
  ib.str_off = idx.off;
  ib.n_cls = n_cls;
  ib.L = L;
  ib.own_rows = int(own_rows);
  ib.grid = G;
  ib.max_items = max_items;
  ib.items = d_items;
  ib.cta_off = d_cta;
  ib.tests = d_tests;
  ib.status = status;
  ib.goff = d_goff;
  ib.meta = d_meta;
  ib.boff = d_boff;
  ib.bcnt = d_boff + kCostBuckets;
  tc_items_plan_kernel<<<1, kItemThreads, 0, s>>>(ib);
  tc_items_place_kernel<<<unsigned(ceil_div(max_items, 256)), 256, 0, s>>>(ib);
  count_launches(2);
  e = cudaGetLastError();
  if (e == cudaSuccess) {
    const KeyedIndex& k0 = *kx[0];
    const KeyedIndex& k1 = *kx[n_cls - 1];
    auto narrow = [&](int c) {
      return mode == MODE_SUM && score_max[c] < (uint64_t(1) << 27) && !force_wide_sums() ? 1 : 0;
    };
    FusedParams p{d_items,
                  max_items,
                  d_cta,
                  k0.rows,
                  k1.rows,
                  k0.ids,
                  k1.ids,
                  mode == MODE_SUM ? k0.score : nullptr,
                  mode == MODE_SUM ? k1.score : nullptr,
                  mode == MODE_SUM ? out_sum[0] : nullptr,
                  mode == MODE_SUM ? out_sum[n_cls - 1] : nullptr,
                  narrow(0),
                  narrow(n_cls - 1),
                  idx.rows,
                  0,
                  idx.ids,
                  0u,
                  -1,
                  out_u32,
                  status};
    test_stall(&p.poll_limit, &p.stall_unit);
    void* tok = prof_stage >= 0 ? prof_begin(prof_stage, s) : nullptr;
#define IG_TCF_CASE(KTV)                                                   \
  case KTV:                                                                \
    e = mode == MODE_ANY     ? run_fused<KTV, MODE_ANY>(p, s)              \
        : mode == MODE_COUNT ? run_fused<KTV, MODE_COUNT>(p, s)            \
                             : run_fused<KTV, MODE_SUM>(p, s);             \
    break;
    switch (KT) {
      IG_TCF_CASE(2)
      IG_TCF_CASE(4)
      IG_TCF_CASE(8)
    }
#undef IG_TCF_CASE
    prof_end(tok);
  }
  // The tests, into the caller's pinned words when the stream gets here.
  if (e == cudaSuccess && tests_out)
    e = cudaMemcpyAsync(tests_out, d_tests, size_t(n_cls) * 8, cudaMemcpyDeviceToHost, s);
  cudaFreeAsync(blk, s);
  return e;
}

cudaError_t indexed_subset_tc(int mode, const RecordIndex& idx, const KeyedIndex& kx,
                              uint32_t* out_u32, unsigned long long* out_u64, int* status,
                              int64_t* tests_out, int prof_stage, uint64_t score_max,
                              cudaStream_t s) {
  if (idx.n_rows == 0 || !tc_supported(idx.KT)) return cudaErrorInvalidValue;
  const KeyedIndex* kxs[1] = {&kx};
  unsigned long long* sums[1] = {out_u64};
  return indexed_subset_tc_classes(mode, idx, kxs, 1, out_u32, sums, status, tests_out,
                                   prof_stage, &score_max, s);
}

cudaError_t launch_subset_tc(const TcArgs& a, cudaStream_t s) {
  if (a.n_own == 0 || a.n_stream == 0) return cudaSuccess;
#define IG_TC_CASE(KTV)                                                        \
  case KTV:                                                                    \
    switch (a.mode) {                                                          \
      case MODE_ANY: return run_tc<KTV, MODE_ANY>(a, s);                       \
      case MODE_COUNT: return run_tc<KTV, MODE_COUNT>(a, s);                   \
      case MODE_SUM: return run_tc<KTV, MODE_SUM>(a, s);                       \
    }                                                                          \
    break;
  switch (a.KT) {
    IG_TC_CASE(2)
    IG_TC_CASE(4)
    IG_TC_CASE(8)
  }
#undef IG_TC_CASE
  return cudaErrorInvalidValue;
}

}  // namespace igk
