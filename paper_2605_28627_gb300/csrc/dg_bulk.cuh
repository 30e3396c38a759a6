// Staging of a contiguous global range of doubles into shared memory with the
// bulk-copy engine (cp.async.bulk, TMA without a tensor map), completion
// tracked by an mbarrier's transaction count.
//
// A bulk copy wants a 16-byte aligned source and destination and a size that
// is a multiple of 16 bytes.  A range of doubles starts on an 8-byte boundary
// (element blocks of an odd number of nodes, or a caller's view at an odd
// offset), so the 16-byte aligned middle of the range goes through the bulk
// copy into a destination with the same address modulo 16, and the at most
// one double before and one after it are copied with plain loads by the
// issuing thread.  Nothing outside the range is read.
//
// Use (one phase per initialisation):
//   one thread: bulk_bar_init(&bar); bulk_expect(&bar, middle bytes of its ranges);
//               bulk_stage_range(...) for each range
//   __syncthreads();                 // barrier initialised, head/tail doubles stored
//   bulk_wait(&bar, 0);              // the bulk copies have landed
//   __syncthreads(); that thread: bulk_bar_inval(&bar)   // before the memory is initialised again
// The wait is bounded: after kBulkWaitLimit polls it records the failure in
// this translation unit's bulk-wait word (read by the entry points of checked
// builds) and returns, so a lost completion cannot hang the GPU.
#pragma once

#include <cstdint>

#include "dg_check.cuh"

namespace dg {

constexpr long kBulkWaitLimit = 1L << 26;

static __device__ unsigned dg_bulk_wait_failed;   // one per translation unit

__device__ __forceinline__ unsigned smem_addr(const void* p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void bulk_bar_init(uint64_t* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(bar)) : "memory");
  // make the initialised barrier visible to the asynchronous (bulk-copy) proxy
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Invalidate a barrier whose phase every waiter has seen complete, so that its
// memory may be initialised again (a persistent kernel's next tile).
__device__ __forceinline__ void bulk_bar_inval(uint64_t* bar) {
  asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_addr(bar)) : "memory");
}

// The issuing thread's arrival, expecting `bytes` of bulk-copy transactions.
__device__ __forceinline__ void bulk_expect(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

// Bytes of the 16-byte aligned middle of the range [src, src + count).
__device__ __forceinline__ unsigned bulk_middle_bytes(const double* src, int count) {
  const uintptr_t s0 = reinterpret_cast<uintptr_t>(src), s1 = s0 + 8 * (uintptr_t)count;
  const uintptr_t a0 = (s0 + 15) & ~uintptr_t(15), a1 = s1 & ~uintptr_t(15);
  return a1 > a0 ? static_cast<unsigned>(a1 - a0) : 0u;
}

// Where the staged copy of src[0..count) lives inside a shared-memory region
// (which needs count * 8 + 24 bytes): 16-byte aligned up, then offset so that
// it has src's address modulo 16.
__device__ __forceinline__ double* bulk_stage_ptr(void* region, const double* src) {
  const uintptr_t r = (reinterpret_cast<uintptr_t>(region) + 15) & ~uintptr_t(15);
  return reinterpret_cast<double*>(r + (reinterpret_cast<uintptr_t>(src) & 15));
}

// Issue the copy of src[0..count) to dst (from bulk_stage_ptr): the aligned
// middle by the bulk engine, the head and tail doubles by plain loads.  The
// middle's bytes must already be expected on bar.
__device__ __forceinline__ void bulk_stage_range(double* dst, const double* src, int count, uint64_t* bar) {
  const uintptr_t s0 = reinterpret_cast<uintptr_t>(src), s1 = s0 + 8 * (uintptr_t)count;
  const uintptr_t a0 = (s0 + 15) & ~uintptr_t(15), a1 = s1 & ~uintptr_t(15);
  if (a1 > a0) {
    const long off = (long)(a0 - s0) / 8;
    bulk_copy_g2s(dst + off, src + off, static_cast<unsigned>(a1 - a0), bar);
    if (off) dst[0] = src[0];
    const long tail = (long)(s1 - a1) / 8;
    if (tail) dst[count - 1] = src[count - 1];
  } else {
    for (int i = 0; i < count; ++i) dst[i] = src[i];
  }
}

// Bounded wait for the phase `phase` of bar; false (and the failure recorded)
// if it did not complete within kBulkWaitLimit polls.
__device__ __forceinline__ bool bulk_wait(uint64_t* bar, unsigned phase) {
  const unsigned addr = smem_addr(bar);
  for (long it = 0; it < kBulkWaitLimit; ++it) {
    unsigned done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(addr), "r"(phase)
        : "memory");
    if (done) return true;
  }
  atomicExch(&dg_bulk_wait_failed, 1u);
  return false;
}

// Host reader of this translation unit's bulk-wait word: returns it and clears it.
#define DG_BULK_READER(name)                                                     \
  unsigned name() {                                                              \
    unsigned w = 0, z = 0;                                                       \
    if (cudaMemcpyFromSymbol(&w, dg_bulk_wait_failed, sizeof w) != cudaSuccess)   \
      return 0;                                                                  \
    if (w) cudaMemcpyToSymbol(dg_bulk_wait_failed, &z, sizeof z);                \
    return w;                                                                    \
  }

}  // namespace dg
