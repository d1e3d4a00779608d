// binary16x2 helpers shared by the row-pair kernels (values held as 32-bit bit patterns).
#pragma once

#ifndef __CUDACC_RTC__
#include <cstdint>
#endif

namespace ldpc {
namespace h2 {

constexpr uint32_t kOne2 = 0x3C003C00u;     // (1.0, 1.0)
constexpr uint32_t kNegOne2 = 0xBC00BC00u;  // (-1.0, -1.0)
constexpr uint32_t kP127 = 0x57F057F0u;     // 127.0
constexpr uint32_t kBias2 = 0x64806480u;    // 1152.0: message byte c + 128 under exponent 0x64
constexpr uint32_t kInf2 = 0x7C007C00u;
constexpr uint32_t kSign2 = 0x80008000u;
constexpr uint32_t kAbs2 = 0x7FFF7FFFu;
constexpr int kMaxDeg = 20;
// 8-bit decoders: posteriors held as binary16 L + 1279 (exact, spacing 1 on [1152, 1406]),
// so that v + 127 = (L + 1279) - (c + 1152) is one subtraction
constexpr uint32_t kPostBias = 0x64FF64FFu;   // 1279: L = 0
constexpr uint32_t kPostLo = 0x64806480u;     // 1152: L = -127
constexpr uint32_t kPostHi = 0x657E657Eu;     // 1406: L = 127
constexpr uint32_t k254 = 0x5BF05BF0u;        // 254.0



__device__ __forceinline__ uint32_t h2sub(uint32_t a, uint32_t b) {
    uint32_t d;
    asm("sub.rn.f16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
    return d;
}
__device__ __forceinline__ uint32_t h2add(uint32_t a, uint32_t b) {
    uint32_t d;
    asm("add.rn.f16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
    return d;
}
__device__ __forceinline__ uint32_t h2fma(uint32_t a, uint32_t b, uint32_t c) {
    uint32_t d;
    asm("fma.rn.f16x2 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
    return d;
}
__device__ __forceinline__ uint32_t h2relu_fma(uint32_t a, uint32_t b, uint32_t c) {
    uint32_t d;
    asm("fma.rn.relu.f16x2 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
    return d;
}
__device__ __forceinline__ uint32_t h2min(uint32_t a, uint32_t b) {
    uint32_t d;
    asm("min.f16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
    return d;
}
__device__ __forceinline__ uint32_t h2max(uint32_t a, uint32_t b) {
    uint32_t d;
    asm("max.f16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
    return d;
}
// min(|a|, |b|) with sign(a) xor sign(b)
__device__ __forceinline__ uint32_t h2minxs(uint32_t a, uint32_t b) {
    uint32_t d;
    asm("min.xorsign.abs.f16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
    return d;
}
__device__ __forceinline__ uint32_t h2maxxs(uint32_t a, uint32_t b) {
    uint32_t d;
    asm("max.xorsign.abs.f16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
    return d;
}
__device__ __forceinline__ uint32_t prmt(uint32_t a, uint32_t b, uint32_t s) {
    uint32_t d;
    asm("prmt.b32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(s));
    return d;
}
// |a| per lane (a sign-bit clear; foldable into a following add as an operand modifier)
__device__ __forceinline__ uint32_t h2abs(uint32_t a) {
    uint32_t d;
    asm("abs.f16x2 %0, %1;" : "=r"(d) : "r"(a));
    return d;
}
// per-lane (a < b) of binary16 values -> 0xFFFF / 0 per lane
__device__ __forceinline__ uint32_t h2lt_mask(uint32_t a, uint32_t b) {
    uint32_t d;
    asm("set.lt.u32.f16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
    return d;
}

// m1 (the smallest |x| of x[LO .. LO + N), carrying the product of their signs) and m2
// (the second smallest |x|) as a tree: two values give m1 = min.xorsign(a, b) and
// m2 = max(|a|, |b|); two halves combine as m1 = min.xorsign(m1a, m1b) and
// m2 = min(m2a, m2b, max(|m1a|, |m1b|)); one value gives m1 = x, m2 = +inf.  Every step is
// an exact min / max, so the result equals the edge-by-edge scan, with 3N - 4 operations
// (N >= 2) instead of 3N and a dependent chain of about log2 N steps instead of N.
template <int LO, int N, int D>
__device__ __forceinline__ void min_tree(const uint32_t (&x)[D], uint32_t &m1, uint32_t &m2) {
    if constexpr (N == 1) {
        m1 = x[LO];
        m2 = kInf2;
    } else if constexpr (N == 2) {
        m1 = h2minxs(x[LO], x[LO + 1]);
        m2 = h2max(h2abs(x[LO]), h2abs(x[LO + 1]));
    } else if constexpr (N == 3) {
        uint32_t a1, a2;
        min_tree<LO, 2>(x, a1, a2);
        m1 = h2minxs(a1, x[LO + 2]);
        m2 = h2min(a2, h2max(h2abs(a1), h2abs(x[LO + 2])));
    } else {
        constexpr int NA = 2 * ((N / 2 + 1) / 2);    // even, and N - NA >= 2
        uint32_t a1, a2, b1, b2;
        min_tree<LO, NA>(x, a1, a2);
        min_tree<LO + NA, N - NA>(x, b1, b2);
        m1 = h2minxs(a1, b1);
        m2 = h2min(h2min(a2, b2), h2max(h2abs(a1), h2abs(b1)));
    }
}

}  // namespace h2
}  // namespace ldpc
