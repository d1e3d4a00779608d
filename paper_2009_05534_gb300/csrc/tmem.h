// Tensor Memory, named-barrier and 1-D bulk-copy helpers shared by the TMEM decoders.
//
// TMEM is used as per-thread private storage: a warp reads and writes its own 32-lane
// quarter (lanes 32 * (warp % 4) .. + 31) with tcgen05.ld / tcgen05.st of shape 32x32b, one
// 32-bit column per register, at warp-uniform run-time column addresses.
#pragma once

#ifndef __CUDACC_RTC__
#include <cstdint>
#endif

namespace ldpc {
namespace tm {


template <int N>
__device__ __forceinline__ void tld(uint32_t taddr, uint32_t *r);
template <>
__device__ __forceinline__ void tld<1>(uint32_t a, uint32_t *r) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x1.b32 {%0}, [%1];" : "=r"(r[0]) : "r"(a));
}
template <>
__device__ __forceinline__ void tld<2>(uint32_t a, uint32_t *r) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x2.b32 {%0, %1}, [%2];"
                 : "=r"(r[0]), "=r"(r[1]) : "r"(a));
}
template <>
__device__ __forceinline__ void tld<4>(uint32_t a, uint32_t *r) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]) : "r"(a));
}
template <>
__device__ __forceinline__ void tld<8>(uint32_t a, uint32_t *r) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
                   "=r"(r[6]), "=r"(r[7])
                 : "r"(a));
}
template <>
__device__ __forceinline__ void tld<16>(uint32_t a, uint32_t *r) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, "
                 "%9, %10, %11, %12, %13, %14, %15}, [%16];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
                   "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]),
                   "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                 : "r"(a));
}
template <int N>
__device__ __forceinline__ void tst(uint32_t taddr, const uint32_t *r);
template <>
__device__ __forceinline__ void tst<1>(uint32_t a, const uint32_t *r) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x1.b32 [%0], {%1};" ::"r"(a), "r"(r[0]));
}
template <>
__device__ __forceinline__ void tst<2>(uint32_t a, const uint32_t *r) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x2.b32 [%0], {%1, %2};" ::"r"(a), "r"(r[0]),
                 "r"(r[1]));
}
template <>
__device__ __forceinline__ void tst<4>(uint32_t a, const uint32_t *r) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1, %2, %3, %4};" ::"r"(a),
                 "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]));
}
template <>
__device__ __forceinline__ void tst<8>(uint32_t a, const uint32_t *r) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"r"(a),
        "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]));
}
template <>
__device__ __forceinline__ void tst<16>(uint32_t a, const uint32_t *r) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, "
                 "%9, %10, %11, %12, %13, %14, %15, %16};" ::"r"(a),
                 "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]),
                 "r"(r[7]), "r"(r[8]), "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]),
                 "r"(r[14]), "r"(r[15]));
}
__device__ __forceinline__ void twait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void twait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// load / store N consecutive columns as power-of-two pieces (N <= 15)
template <int N>
__device__ __forceinline__ void tload(uint32_t a, uint32_t *r) {
    if constexpr (N >= 8) {
        tld<8>(a, r);
        tload<N - 8>(a + 8, r + 8);
    } else if constexpr (N >= 4) {
        tld<4>(a, r);
        tload<N - 4>(a + 4, r + 4);
    } else if constexpr (N >= 2) {
        tld<2>(a, r);
        tload<N - 2>(a + 2, r + 2);
    } else if constexpr (N == 1) {
        tld<1>(a, r);
    }
}
template <int N>
__device__ __forceinline__ void tstore(uint32_t a, const uint32_t *r) {
    if constexpr (N >= 8) {
        tst<8>(a, r);
        tstore<N - 8>(a + 8, r + 8);
    } else if constexpr (N >= 4) {
        tst<4>(a, r);
        tstore<N - 4>(a + 4, r + 4);
    } else if constexpr (N >= 2) {
        tst<2>(a, r);
        tstore<N - 2>(a + 2, r + 2);
    } else if constexpr (N == 1) {
        tst<1>(a, r);
    }
}

__device__ __forceinline__ void named_sync(int id, int nthreads) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}
__device__ __forceinline__ int named_or(int id, int nthreads, int pred) {
    int r;
    asm volatile(
        "{\n .reg .pred p, q;\n setp.ne.s32 p, %1, 0;\n bar.red.or.pred q, %2, %3, p;\n"
        " selp.s32 %0, 1, 0, q;\n}"
        : "=r"(r)
        : "r"(pred), "r"(id), "r"(nthreads)
        : "memory");
    return r;
}

// -------------------------------------------------------- channel LLR staging (TMA 1-D)

constexpr uint32_t kSpinLimit = 1u << 22;   // bounded mbarrier waits (each try_wait may sleep)

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t *bar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(bar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// one thread: expect `bytes` and start the bulk copy global -> shared
__device__ __forceinline__ void bulk_load(void *dst, const void *src, uint32_t bytes,
                                          uint64_t *bar) {
    // order the block's earlier generic reads of the buffer before the async-proxy write
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
                 "r"(bytes)
                 : "memory");
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
            "r"(smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}
// bounded wait for phase `parity` of the barrier; returns false on timeout (after `limit`
// polls, each of which may suspend the thread for a short hardware-defined time)
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity,
                                          uint32_t limit = kSpinLimit) {
    for (uint32_t i = 0; i < limit; ++i) {
        uint32_t ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            " selp.u32 %0, 1, 0, p;\n}"
            : "=r"(ok)
            : "r"(smem_addr(bar)), "r"(parity)
            : "memory");
        if (ok) return true;
    }
    return false;
}

// warp-wide: allocate `ncols` (a power of two >= 32) TMEM columns, base address to *dst
__device__ __forceinline__ void tmem_alloc(uint32_t *dst, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_addr(dst)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t base, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(base), "r"(ncols)
                 : "memory");
}
// block barrier with the TMEM ordering fences around it
__device__ __forceinline__ void tmem_block_sync() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

}  // namespace tm
}  // namespace ldpc
