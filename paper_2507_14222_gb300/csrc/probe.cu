// Throughput probes: measured rates of the units the IG kernels are bound
// by, used as roofline denominators (ig_probe in include/ig.h).  None of
// this is part of the method; it measures the hardware the method runs on.
//
//  * LOP3: eight independent lop3.b32 chains per thread, all SMs.  The
//    integer-pipe subset test (Eq. 6 as acc |= p & ~r) is one LOP3 per
//    32-bit half word.
//  * L2 read: coalesced 16-byte loads over a buffer small enough to stay in
//    L2, after one pass that brings it there.
//  * L2 random: 16-byte loads at hashed 16-byte offsets of such a buffer
//    (the access pattern of the dedup table's key compares).
//  * MMA: back-to-back tcgen05.mma kind::f8f6f4 chains (E4M3 operands, FP32
//    accumulators in tensor memory), M = 128, N = 64 / 128 / 256, 16 MMAs of
//    K = 32 per chain (one 512-item row pair, as in the subset GEMM), with A
//    read from shared memory or from tensor memory.  One thread per CTA
//    issues; the chains are committed to an mbarrier whose wait is bounded.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "../../include/ig.h"
#include "common.cuh"
#include "internal.h"

namespace igk {
namespace {

// ---- integer pipe ---------------------------------------------------------------

__global__ void __launch_bounds__(256) lop3_probe_kernel(uint32_t seed, int iters,
                                                         uint32_t* __restrict__ sink) {
  uint32_t a[8], b[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    a[j] = seed ^ (threadIdx.x * 0x9e3779b9u) ^ (j * 0x85ebca6bu);
    b[j] = ~a[j] * 3u + j;
  }
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int r = 0; r < 16; ++r) {
#pragma unroll
      for (int j = 0; j < 8; ++j)
        // a = a | (b & ~a') with a' the next chain: the subset test's shape.
        asm("lop3.b32 %0, %0, %1, %2, 0xF4;" : "+r"(a[j]) : "r"(b[j]), "r"(a[(j + 1) & 7]));
    }
  }
  uint32_t x = 0;
#pragma unroll
  for (int j = 0; j < 8; ++j) x ^= a[j];
  if (x == 0x12345678u) sink[blockIdx.x] = x;  // keeps the chains live
}

// ---- L2 ---------------------------------------------------------------------------

__global__ void __launch_bounds__(512) l2_read_kernel(const uint4* __restrict__ buf, int64_t n16,
                                                      int passes, uint32_t* __restrict__ sink) {
  uint32_t acc = 0;
  const int64_t step = int64_t(gridDim.x) * blockDim.x;
  for (int p = 0; p < passes; ++p)
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n16; i += step) {
      const uint4 v = __ldcg(buf + i);
      acc ^= v.x ^ v.y ^ v.z ^ v.w;
    }
  if (acc == 0x9e3779b9u) sink[blockIdx.x] = acc;
}

__global__ void __launch_bounds__(512) l2_random_kernel(const uint4* __restrict__ buf,
                                                        uint64_t mask16, int per_thread,
                                                        uint32_t* __restrict__ sink) {
  uint32_t acc = 0;
  const uint64_t t = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x;
#pragma unroll 8
  for (int i = 0; i < per_thread; ++i) {
    const uint64_t h = mix64(t * 0x100000001b3ull + uint64_t(i)) & mask16;
    const uint4 v = __ldcg(buf + h);
    acc ^= v.x ^ v.w;
  }
  if (acc == 0x9e3779b9u) sink[blockIdx.x] = acc;
}

__global__ void fill_kernel(uint4* buf, int64_t n16) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i < n16) {
    const uint64_t h = mix64(uint64_t(i));
    buf[i] = make_uint4(uint32_t(h), uint32_t(h >> 32), uint32_t(i), uint32_t(h >> 17));
  }
}

// ---- tensor cores -------------------------------------------------------------------

__device__ __forceinline__ uint64_t probe_sw128_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= uint64_t((saddr & 0x3ffffu) >> 4);
  d |= uint64_t(1) << 16;
  d |= uint64_t(1024 >> 4) << 32;
  d |= uint64_t(1) << 46;
  d |= uint64_t(2) << 61;
  return d;
}

template <int N>
__host__ __device__ constexpr uint32_t probe_idesc() {
  return (1u << 4) | (uint32_t(N >> 3) << 17) | (uint32_t(128 >> 4) << 24);
}

constexpr int kProbeKBytes = 512;  // items per row (one byte each): 16 K steps of 32

template <int N>
struct ProbeShape {
  static constexpr uint32_t kA = 128 * kProbeKBytes;
  static constexpr uint32_t kB = uint32_t(N) * kProbeKBytes;
  // At least 120 KB, so that no two CTAs (each taking all 512 tensor
  // memory columns) share an SM.
  static constexpr size_t kUsed = 1024 + size_t(kA) + kB + 64;
  static constexpr size_t kSmem = kUsed > 120 * 1024 ? kUsed : 120 * 1024;
};

// One CTA per SM; thread 0 issues `chains` chains of 16 MMAs.  With A_TMEM
// the A operand (128 rows x 512 items) is first written into tensor memory
// columns [2N, 2N + 128).  flags: kProbeCommitEach -- a tcgen05.commit after
// every chain; kProbeTwoSlots -- chains alternate between two accumulators
// of N columns and chain c is issued only once chain c - 2 (the same
// accumulator) has completed, the hand-over pattern of the fused kernel.
constexpr int kProbeCommitEach = 1, kProbeTwoSlots = 2;
template <int N, bool A_TMEM>
__global__ void __launch_bounds__(128, 1) mma_probe_kernel(int chains, int flags, int* status,
                                                           unsigned long long* cycles) {
  using S = ProbeShape<N>;
  static_assert(!A_TMEM || 2 * N + 128 <= 512, "tensor memory columns");
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  uint8_t* base = smem_raw + ((1024u - (raw & 1023u)) & 1023u);
  uint8_t* A = base;
  uint8_t* B = A + S::kA;
  uint64_t* bar = reinterpret_cast<uint64_t*>(B + S::kB);  // [3]: final, slot 0, slot 1
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bar + 3);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // 0/1 operands (0x08 per set item), about half the items set.
  for (uint32_t i = threadIdx.x; i < (S::kA + S::kB) / 4; i += blockDim.x) {
    const uint32_t h = uint32_t(mix64(i + 77u * blockIdx.x));
    reinterpret_cast<uint32_t*>(A)[i] = h & 0x08080808u;
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  if (threadIdx.x == 0) {
    for (int i = 0; i < 3; ++i) mbar_init(bar + i, 1);
    fence_mbar_init();
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(512)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;
  if constexpr (A_TMEM) {
    // Each warp writes its 32 lanes of the 128 A columns.
    for (int c0 = 0; c0 < 128; c0 += 8) {
      uint32_t v[8];
#pragma unroll
      for (int j = 0; j < 8; ++j)
        v[j] = uint32_t(mix64(uint64_t(warp * 32 + lane) * 131u + c0 + j)) & 0x08080808u;
      asm volatile(
          "tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"r"(
              tmem + (uint32_t(warp * 32) << 16) + uint32_t(2 * N + c0)),
          "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]),
          "r"(v[7])
          : "memory");
    }
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (threadIdx.x == 0) {
    const uint64_t t0 = clock64();
    const uint32_t a_base = smem_u32(A), b_base = smem_u32(B);
    const bool two = (flags & kProbeTwoSlots) != 0;
    bool ok = true;
    for (int c = 0; c < chains && ok; ++c) {
      const uint32_t d = two ? tmem + uint32_t((c & 1) * N) : tmem;
      if (two && c >= 2) ok = mbar_wait(bar + 1 + (c & 1), uint32_t(((c - 2) >> 1) & 1), status);
#pragma unroll
      for (int k = 0; k < kProbeKBytes / 32; ++k) {
        const uint32_t aoff = uint32_t(k >> 2) * (128 * 128) + uint32_t(k & 3) * 32;
        const uint32_t boff = uint32_t(k >> 2) * (N * 128) + uint32_t(k & 3) * 32;
        const uint32_t acc = k > 0 ? 1u : 0u;
        if constexpr (A_TMEM) {
          asm volatile(
              "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
              "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], [%1], %2, %3, p;\n\t}" ::"r"(d),
              "r"(tmem + uint32_t(2 * N + 8 * k)), "l"(probe_sw128_desc(b_base + boff)),
              "r"(probe_idesc<N>()), "r"(acc)
              : "memory");
        } else {
          asm volatile(
              "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
              "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
              "l"(probe_sw128_desc(a_base + aoff)), "l"(probe_sw128_desc(b_base + boff)),
              "r"(probe_idesc<N>()), "r"(acc)
              : "memory");
        }
      }
      if (two || (flags & kProbeCommitEach))
        asm volatile(
            "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                smem_u32(bar + 1 + (two ? (c & 1) : 0)))
            : "memory");
    }
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_u32(bar))
        : "memory");
    mbar_wait(bar, 0, status);
    cycles[blockIdx.x] = clock64() - t0;
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512)
                 : "memory");
  }
}

template <int N, bool A_TMEM>
cudaError_t run_mma_probe(int chains, int flags, int* status, unsigned long long* cycles,
                          cudaStream_t s) {
  using S = ProbeShape<N>;
  cudaError_t e = cudaFuncSetAttribute(mma_probe_kernel<N, A_TMEM>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, int(S::kSmem));
  if (e != cudaSuccess) return e;
  mma_probe_kernel<N, A_TMEM><<<unsigned(num_sms()), 128, S::kSmem, s>>>(chains, flags, status,
                                                                        cycles);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace

// Runs one probe twice (a warm-up launch, then the timed one) and returns
// its rate per second and the timed launch's device time.
int probe_run(int probe, int arg, double* rate, double* ms, double* cycles_out) {
  cudaError_t e = cudaSuccess;
  cudaStream_t s = nullptr;
  cudaEvent_t ev[2] = {nullptr, nullptr};
  void* buf = nullptr;
  int* status = nullptr;
  unsigned long long* cyc = nullptr;
  uint32_t* sink = nullptr;
  const int sms = num_sms();
  double work = 0.0;  // units of the rate per timed launch
  int rc = IG_OK;
#define IG_P_TRY(x)            \
  if ((e = (x)) != cudaSuccess) \
    goto done;
  IG_P_TRY(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
  IG_P_TRY(cudaEventCreate(&ev[0]));
  IG_P_TRY(cudaEventCreate(&ev[1]));
  IG_P_TRY(cudaMalloc(&status, sizeof(int)));
  IG_P_TRY(cudaMemset(status, 0, sizeof(int)));
  IG_P_TRY(cudaMalloc(&cyc, sizeof(unsigned long long) * sms));
  IG_P_TRY(cudaMemset(cyc, 0, sizeof(unsigned long long) * sms));
  IG_P_TRY(cudaMalloc(&sink, sizeof(uint32_t) * 4096));
  for (int rep = 0; rep < 2; ++rep) {
    if (rep == 1) IG_P_TRY(cudaEventRecord(ev[0], s));
    switch (probe) {
      case IG_PROBE_LOP3: {
        const int blocks = sms * 8, iters = 4096;
        lop3_probe_kernel<<<blocks, 256, 0, s>>>(0x1234u + rep, iters, sink);
        count_launches(1);
        work = double(blocks) * 256 * iters * 16 * 8;
        break;
      }
      case IG_PROBE_L2_READ:
      case IG_PROBE_L2_RANDOM: {
        const int64_t mib = arg > 0 ? arg : 48;
        const int64_t n16 = (mib << 20) / 16;
        if (!buf) {
          IG_P_TRY(cudaMalloc(&buf, size_t(n16) * 16));
          fill_kernel<<<unsigned(ceil_div(n16, 256)), 256, 0, s>>>(static_cast<uint4*>(buf), n16);
          count_launches(1);
          // Bring the buffer into L2.
          l2_read_kernel<<<sms * 4, 512, 0, s>>>(static_cast<const uint4*>(buf), n16, 1, sink);
          count_launches(1);
        }
        if (probe == IG_PROBE_L2_READ) {
          const int passes = 20;
          l2_read_kernel<<<sms * 4, 512, 0, s>>>(static_cast<const uint4*>(buf), n16, passes,
                                                  sink);
          work = double(n16) * 16 * passes;
        } else {
          uint64_t p2 = 1;
          while (p2 * 2 <= uint64_t(n16)) p2 *= 2;
          const int per = 256;
          l2_random_kernel<<<sms * 8, 512, 0, s>>>(static_cast<const uint4*>(buf), p2 - 1, per,
                                                   sink);
          work = double(sms) * 8 * 512 * per * 16;
        }
        count_launches(1);
        break;
      }
      case IG_PROBE_MMA_F8_SMEM:
      case IG_PROBE_MMA_F8_TMEM: {
        const int N = (arg & 0xfff) > 0 ? (arg & 0xfff) : 128;
        const int flags = (arg >> 12) & 3;
        const bool tm = probe == IG_PROBE_MMA_F8_TMEM;
        const int chains = 2048;
        if (N == 64) e = tm ? run_mma_probe<64, true>(chains, flags, status, cyc, s)
                            : run_mma_probe<64, false>(chains, flags, status, cyc, s);
        else if (N == 128) e = tm ? run_mma_probe<128, true>(chains, flags, status, cyc, s)
                                  : run_mma_probe<128, false>(chains, flags, status, cyc, s);
        else if (N == 256 && !tm) e = run_mma_probe<256, false>(chains, flags, status, cyc, s);
        else {
          rc = report_error(IG_E_INVAL, "ig_probe: MMA probe N must be 64, 128 or 256 "
                                        "(64 or 128 with A in tensor memory)");
          goto done;
        }
        IG_P_TRY(e);
        work = double(sms) * chains * 2.0 * 128 * N * kProbeKBytes;
        break;
      }
      default:
        rc = report_error(IG_E_INVAL, "ig_probe: unknown probe");
        goto done;
    }
    IG_P_TRY(cudaGetLastError());
    if (rep == 1) IG_P_TRY(cudaEventRecord(ev[1], s));
  }
  IG_P_TRY(cudaStreamSynchronize(s));
  {
    float t = 0.f;
    IG_P_TRY(cudaEventElapsedTime(&t, ev[0], ev[1]));
    int st = 0;
    IG_P_TRY(cudaMemcpy(&st, status, sizeof(int), cudaMemcpyDeviceToHost));
    if (st & ST_TIMEOUT) {
      rc = report_error(IG_E_TIMEOUT, "ig_probe: a bounded device wait ran out");
      goto done;
    }
    if (ms) *ms = double(t);
    if (rate) *rate = t > 0.f ? work / (double(t) * 1e-3) : 0.0;
    if (cycles_out) {
      double mx = 0.0;
      if (probe == IG_PROBE_MMA_F8_SMEM || probe == IG_PROBE_MMA_F8_TMEM) {
        std::vector<unsigned long long> h(sms);
        IG_P_TRY(cudaMemcpy(h.data(), cyc, sizeof(unsigned long long) * sms,
                            cudaMemcpyDeviceToHost));
        for (int i = 0; i < sms; ++i) mx = std::max(mx, double(h[i]));
      }
      *cycles_out = mx;
    }
  }
done:
#undef IG_P_TRY
  if (e != cudaSuccess && rc == IG_OK) {
    rc = report_error(e == cudaErrorMemoryAllocation ? IG_E_NOMEM : IG_E_CUDA,
                      cudaGetErrorString(e));
  }
  if (buf) cudaFree(buf);
  if (status) cudaFree(status);
  if (cyc) cudaFree(cyc);
  if (sink) cudaFree(sink);
  for (cudaEvent_t x : ev)
    if (x) cudaEventDestroy(x);
  if (s) cudaStreamDestroy(s);
  return rc;
}

}  // namespace igk

extern "C" int ig_probe(int32_t probe, int32_t arg, double* rate, double* ms, double* cycles) {
  return igk::probe_run(probe, arg, rate, ms, cycles);
}
