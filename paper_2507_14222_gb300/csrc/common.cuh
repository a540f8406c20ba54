// Device-side helpers shared by the IG kernels (sm_103a).
//
// * a device status word that kernels OR error bits into instead of trapping;
// * bounded mbarrier waits and 1-D TMA bulk copies (cp.async.bulk) for
//   staging row tiles into shared memory;
// * the 64-bit key hash used by the candidate hash table.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#define IG_MAX_KT_WORDS 16

namespace igk {

// Bits of the per-call device status word.
enum : int {
  ST_TIMEOUT = 1,     // a bounded wait (mbarrier or hash slot) ran out
  ST_TABLE_FULL = 2,  // a hash probe sequence visited every slot
  ST_BAD_INPUT = 4,   // input value out of range (code >= card, label > 1)
  ST_COUNT = 8,       // a table held more keys than its count (nothing written past it)
};

// Upper bounds on spin loops.  Each mbarrier poll is a try_wait that
// suspends the thread until the phase completes or about kMbarSuspendNs
// nanoseconds pass, so the bound below is about two seconds of waiting.  The
// suspension keeps waiting warps (the tensor-core kernels' producer,
// expander and epilogue roles spend much of their time waiting) from
// spending issue slots that the working warps of the SM need.
constexpr uint32_t kMbarSuspendNs = 2000;
constexpr uint32_t kMbarPollLimit = 1u << 20;
constexpr uint32_t kSlotSpinLimit = 1u << 22;

__device__ __forceinline__ void set_status(int* status, int bits) {
  atomicOr(status, bits);
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(count)
               : "memory");
}

// Make mbarrier initialisation visible to the async (TMA) proxy.
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar,
                                                      uint32_t bytes) {
  asm volatile(
      "mbarrier.arrive.expect_tx.release.cta.shared::cta.b64 _, [%0], %1;" ::"r"(
          smem_u32(bar)),
      "r"(bytes)
      : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.acquire.cta.shared::cta.b64 p, [%1], %2, %3;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity), "n"(kMbarSuspendNs)
      : "memory");
  return ok != 0;
}

// Waits for the given phase parity; false (and ST_TIMEOUT set) if the poll
// limit (kMbarPollLimit unless given) is reached first.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity,
                                          int* status, uint32_t limit = kMbarPollLimit) {
  for (uint32_t it = 0; it < limit; ++it)
    if (mbar_try_wait(bar, parity)) return true;
  set_status(status, ST_TIMEOUT);
  return false;
}

// 1-D TMA bulk copy global -> shared, completing on `bar` with `bytes`
// transaction bytes.  dst, src and bytes must be multiples of 16.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src,
                                         uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cta.global.mbarrier::complete_tx::bytes "
      "[%0], [%1], %2, [%3];" ::"r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ uint32_t ld_acquire_u32(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_release_u32(uint32_t* p, uint32_t v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ uint64_t ld_relaxed_u64(const uint64_t* p) {
  uint64_t v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

// 64-bit mixing function (the finaliser of the splitmix64 generator,
// Steele, Lea and Flood, "Fast splittable pseudorandom number generators",
// OOPSLA 2014).
__device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}

// Hash of a KT-word key: one multiply-xorshift round per word (so the word
// position matters), then the full mixing function so that keys differing
// in a single sparse bit land far apart.
// The same hash taken one word at a time (hash_begin, hash_word per word in
// order, hash_end), for callers that do not hold the key in registers.
__device__ __forceinline__ uint64_t hash_begin() { return 0x243f6a8885a308d3ull; }
__device__ __forceinline__ uint64_t hash_word(uint64_t h, uint64_t w) {
  h = (h ^ w) * 0x9e3779b97f4a7c15ull;
  return h ^ (h >> 32);
}
__device__ __forceinline__ uint64_t hash_end(uint64_t h) { return mix64(h); }

template <int KT>
__device__ __forceinline__ uint64_t hash_key(const uint64_t (&w)[KT]) {
  uint64_t h = hash_begin();
#pragma unroll
  for (int k = 0; k < KT; ++k) h = hash_word(h, w[k]);
  return hash_end(h);
}

__host__ __device__ constexpr int64_t ceil_div(int64_t a, int64_t b) {
  return (a + b - 1) / b;
}


// Calls __VA_ARGS__ with the compile-time constant KTC equal to the runtime
// padded word count KT_VAR (1, 2, 4, 8 or 16); other values return
// cudaErrorInvalidValue from the enclosing function.
#define IG_DISPATCH_KT(KT_VAR, ...)                        \
  switch (KT_VAR) {                                        \
    case 1: { constexpr int KTC = 1; __VA_ARGS__; break; } \
    case 2: { constexpr int KTC = 2; __VA_ARGS__; break; } \
    case 4: { constexpr int KTC = 4; __VA_ARGS__; break; } \
    case 8: { constexpr int KTC = 8; __VA_ARGS__; break; } \
    case 16: { constexpr int KTC = 16; __VA_ARGS__; break; } \
    default: return cudaErrorInvalidValue;                 \
  }

}  // namespace igk
