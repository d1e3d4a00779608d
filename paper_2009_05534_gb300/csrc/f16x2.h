// binary16x2 helpers shared by the row-pair kernels (values held as 32-bit bit patterns).
#pragma once

#include <cstdint>

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


}  // namespace h2
}  // namespace ldpc
