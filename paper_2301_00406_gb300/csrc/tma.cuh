// Tensor-memory-access (TMA) tile copies between global and shared memory,
// with the mbarrier that signals a load's completion, for sm_100-class GPUs.
//
// A tile is described on the host by a CUtensorMap (cuTensorMapEncodeTiled,
// fetched from the driver at run time, so the library does not link libcuda)
// and moved by one thread with cp.async.bulk.tensor; loads complete on an
// mbarrier by transaction bytes, stores are tracked by bulk groups.  Every
// wait on an mbarrier is bounded in time: after one second the wait gives up,
// records the failure (a shared flag and, when given, a status word in global
// memory) and later waits of the CTA return at once, so the kernel runs to
// its end and the host reads the status.
#pragma once

#include <cuda.h>
#include <stdint.h>

#include "common.cuh"

namespace nlos {

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Rounds a dynamic shared-memory pointer up to 1024 bytes (the period of the
// 128-byte swizzle, which the tile base must keep).
__device__ __forceinline__ unsigned char* align1024(unsigned char* p) {
  const uint32_t a = smem_u32(p);
  return p + ((1024u - (a & 1023u)) & 1023u);
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ uint64_t tma_global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Waits for the phase of `bar` with the given parity, for at most limit_ns
// (one second by default).  On giving up: *fail = 1 and, if status is given,
// *status = NLOS_ERR_TIMEOUT (when it still holds NLOS_OK).  Returns
// immediately once *fail is set.
__device__ __forceinline__ void mbar_wait_bounded(uint32_t bar, uint32_t parity, volatile int* fail,
                                                  int32_t* status, uint64_t limit_ns = 1000000000ull) {
  if (*fail) return;
  const uint64_t t0 = tma_global_ns();
  for (;;) {
    uint32_t done;
    asm volatile(
        "{\n.reg .pred P;\nmbarrier.try_wait.parity.shared::cta.b64 P, [%1], %2;\nselp.b32 %0, 1, 0, P;\n}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return;
    if (tma_global_ns() - t0 > limit_ns) {
      *fail = 1;
      if (status) atomicCAS(reinterpret_cast<int*>(status), NLOS_OK, NLOS_ERR_TIMEOUT);
      return;
    }
  }
}

// 2-D tile load: box at element coordinates (x, y) of the map into shared
// memory at dst, completing `bar` by its byte count.
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
      "[%4];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
      : "memory");
}

// 3-D tile load: box at (x, y, z).
__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* map, int x, int y, int z, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
      "[%5];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(bar)
      : "memory");
}

// 2-D tile store from shared memory at src to the box at (x, y); part of the
// thread's current bulk group.
__device__ __forceinline__ void tma_store_2d(const CUtensorMap* map, int x, int y, uint32_t src) {
  asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.tile.bulk_group [%0, {%1, %2}], [%3];" ::"l"(
                   reinterpret_cast<uint64_t>(map)),
               "r"(x), "r"(y), "r"(src)
               : "memory");
}
__device__ __forceinline__ void tma_store_3d(const CUtensorMap* map, int x, int y, int z, uint32_t src) {
  asm volatile("cp.async.bulk.tensor.3d.global.shared::cta.tile.bulk_group [%0, {%1, %2, %3}], [%4];" ::"l"(
                   reinterpret_cast<uint64_t>(map)),
               "r"(x), "r"(y), "r"(z), "r"(src)
               : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// Waits until every committed bulk store of this thread has completed.
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
// Orders this thread's generic-proxy shared-memory writes before later
// async-proxy (TMA) reads of them.
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Host: a 2-D FP32 tensor map over rows of `row_floats` floats, `rows` rows,
// `pitch_bytes` apart (a multiple of 16), with boxes of box_x x box_y
// elements and the 128-byte shared-memory swizzle (box_x * 4 <= 128).
// Out-of-range elements of a load read as zero; those of a store are
// skipped.
nlos_status make_tmap_2d(CUtensorMap* map, const void* base, uint64_t row_floats, uint64_t rows,
                         uint64_t pitch_bytes, uint32_t box_x, uint32_t box_y);
// Host: the rows [0, 2 pairs) of the same layout as a 3-D map over (float in
// row, row parity, row pair): element (x, p, r) is float x of row 2 r + p.  A
// box {box_x, 1, box_r} then holds box_r rows of one parity, consecutive in
// shared memory.
nlos_status make_tmap_rowpairs(CUtensorMap* map, const void* base, uint64_t row_floats, uint64_t pairs,
                               uint64_t pitch_bytes, uint32_t box_x, uint32_t box_r);

}  // namespace nlos
