// Tensor-memory-accelerator (TMA) helpers: mbarrier and cp.async.bulk.tensor wrappers (inline
// PTX, sm_90+ forms used on sm_103a) and the host-side tensor-map description.
#pragma once

#include <cuda.h>
#include <stdint.h>

#include "common.cuh"

namespace pb {

// Iterations of mbarrier.try_wait before a wait is declared stuck (each try suspends the thread
// for a hardware-defined interval; the bound is far above any legitimate copy latency).
constexpr unsigned kWaitLimit = 1u << 24;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

// Returns a barrier's memory to ordinary use (required before it is initialised again).
__device__ __forceinline__ void mbar_inval(uint64_t* bar) {
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Orders this thread's earlier generic-proxy view of global memory (data other blocks wrote and
// this thread has acquired) before its later async-proxy (TMA) reads.
__device__ __forceinline__ void fence_proxy_async_global() {
    asm volatile("fence.proxy.async.global;" ::: "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

// Bounded wait for phase `parity` of the barrier; returns false if the bound ran out.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity) {
    const uint32_t a = smem_u32(bar);
    for (unsigned it = 0; it < kWaitLimit; ++it) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int x, int y, int z, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
        ::"r"(smem_u32(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* map, int c, int x, int y, int z,
                                            uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], [%6];"
        ::"r"(smem_u32(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(c), "r"(x), "r"(y), "r"(z),
          "r"(smem_u32(bar))
        : "memory");
}

// Device-side references to the tensor maps one tile march reads: param-space maps of a
// one-problem launch, or global-memory maps of the batched launch.
struct TmaRefs {
    const CUtensorMap* halo[3];
    const CUtensorMap* coef;
    const CUtensorMap* cen[3];
};

// Host: the tensor maps one TMA march launch needs (all for one scalar field grid).
struct TmaMaps {
    CUtensorMap halo[3];   // arrays of the input field, box (TX + 2 HX) x (TY + 2) x 1
    CUtensorMap coef;      // coefficient records, box 4 x (TX + 1) x (TY + 1) x 1 (bfloat16: (TX + 2) x (TY + 1) x 1 records)
    CUtensorMap cen[3];    // point operands of the epilogue, box TX x TY x 1
};

// Host helpers (tma_host.cu).  Return false when the array cannot be described by a tensor map
// (row stride not a multiple of 16 bytes, or an unaligned base address).
bool tma_available();
bool tma_state_map(CUtensorMap* m, const void* base, int elem_bytes, int nr, int nt, int np, int box_x, int box_y);
// elem_bytes 2 (bfloat16 records): a 3-D map of 8-byte records, needing n_r even (row stride a
// multiple of 16 bytes).
bool tma_coef_map(CUtensorMap* m, const void* base, int elem_bytes, int nr, int nt, int np, int box_x, int box_y);

}  // namespace pb
