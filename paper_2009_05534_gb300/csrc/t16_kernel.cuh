// Device code of the binary16 decoder (tmem16_kernel): row step, parity and the kernel
// body, shared by decode_tmem16.cu (the generic kernels and the launch) and by the kernels
// compiled at run time for a row sequence (t16_jit.cu).
//
// Layered min-sum on binary16 LLRs (normalised, offset or learned correction) with the
// check-to-variable messages held in Tensor Memory (sm_103a).  Paper: Sec. III (layered
// min-sum with a correction of the minimum, stopping rule), Sec. IV (floating-point
// half-precision variant of the decoder); hot-path steps a0..a6.
//
// Arithmetic is that of the binary16 decode path: every subtraction, correction and
// posterior update is one IEEE binary16 operation rounded to nearest even, and the
// correction parameters enter as binary16 values, so the results equal the scalar binary16
// decoder operation for operation.  The correction of a minimum m is
//     m' = beta * max(m - gamma, 0)
// with (beta, gamma) = (alpha, 0) for normalised, (1, offset) for offset and the table
// entry of (iteration, row) for learned min-sum; with those values each form reduces to
// the same rounded operations as its direct definition (m - 0 = m and 1 * t = t exactly).
//
// Mapping.  A thread block decodes two codewords; in each, thread w owns check rows w and
// w + H (H = Z/2) of every layer as the two binary16 lanes of one 32-bit word.  Posteriors
// live in shared memory as lane pairs (word (c, j) holds rows j and j + H of column block
// c), gathered through the circulant with the same half swap as the 8-bit decoder.  Each
// thread's messages live in its own TMEM lane, one 32-bit column (two binary16 messages)
// per edge: a row of degree D is one D-column tcgen05.ld and one tcgen05.st.  A warp reaches
// only its lane quarter (warp % 4), so the block's warps take column regions of E columns
// in turn; the allocation is ceil(warps / 4) * E columns rounded up to a power of two, and
// as many blocks share an SM as its 512 columns hold.
// When two codewords' regions exceed the 512 columns (BG1-shaped codes at low rate and
// large Z), a block decodes one codeword: the first 4 * floor(512 / E) warps keep their
// messages in TMEM and the rest in shared memory ([E][threads] words, one column each).
//
// Per edge the check rule needs no argmin index: with m1 = min |v| and m2 the second
// minimum (equal to m1 on a tie) the message magnitude is m2' where |v| <= m1 and m1'
// elsewhere, and the sign is the xor of the row's sign product with the edge's own sign.
// Negative zero never reaches the posteriors (channel LLRs are canonicalised to +0 on
// load, and x + c rounds a zero sum to +0), so sign bits decide the hard decisions.
#pragma once

#ifndef __CUDACC_RTC__
#include <cuda_fp16.h>
#endif

#include "f16x2.h"
#include "ldpc_params.h"
#include "tmem.h"

namespace ldpc {
namespace {

using namespace h2;
using namespace tm;

struct EdgeMeta16 {
    int base_nw;       // c*H + u
    int thresh;        // H - u
    uint32_t sel_nw;   // 0x3210 or 0x1032
    uint32_t sel_w;
};

constexpr int kMaxEdges16 = 512;
constexpr int kMaxRows16 = 64;
constexpr int kMaxDeg16 = 20;
constexpr int kTmemCols16 = 512;

struct Tmem16Params {
    DecodeParams p;
    int H;
    int wpc;                     // warps per codeword
    int tcols;                   // TMEM columns allocated (power of two)
    int tm_warps;                // one-codeword blocks: warps whose messages are in TMEM
    int ns;                      // one-codeword blocks: threads with messages in shared memory
    int off_msg;                 // shared-memory offset of those messages ([E][ns] words)
    int use_tma;                 // channel LLRs staged by 1-D bulk copies
    int stage_bytes;             // per-half staging buffer (multiple of 16)
    int off_lb, off_stage;       // shared-memory offsets of the posteriors and the staging
    uint32_t beta2, ngamma2;     // uniform correction as binary16 pairs (not learned)
    int learned;                 // 1: per-(iteration, row) table in p.learned
    int row[kMaxRows16 + 1];
    EdgeMeta16 meta[kMaxEdges16];
};

__device__ __forceinline__ uint32_t h2mul(uint32_t a, uint32_t b) {
    uint32_t d;
    asm("mul.rn.f16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
    return d;
}
// per-lane (a <= b) -> 0xFFFF / 0
__device__ __forceinline__ uint32_t h2le_mask(uint32_t a, uint32_t b) {
    uint32_t d;
    asm("set.le.u32.f16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
    return d;
}
// (x, x) rounded to binary16 (IEEE round to nearest even), as a lane pair
__host__ __device__ __forceinline__ uint32_t h2_from_float(float x) {
#ifdef __CUDA_ARCH__
    unsigned short hs;
    asm("cvt.rn.f16.f32 %0, %1;" : "=h"(hs) : "f"(x));
    const uint32_t h = hs;
#else
    const __half_raw r = __float2half_rn(x);
    const uint32_t h = r.x;
#endif
    return h | (h << 16);
}

// Thread w processes row pair w of a layer of degree D.  Its messages start at TMEM column
// tcol (kTm) or at sm[e0 * ns] in shared memory, one word per edge with stride ns.
template <int D, bool kTm>
__device__ __forceinline__ void row16(const EdgeMeta16 *meta, uint32_t *Lb, uint32_t tcol,
                                      uint32_t *sm, int ns, int e0, int H, int w, bool store,
                                      uint32_t beta2, uint32_t ngamma2) {
    uint32_t cm[D];
    if constexpr (kTm) {
        twait_st();                       // this thread's earlier stores to these columns
        tload<D>(tcol, cm);
    } else {
#pragma unroll
        for (int j = 0; j < D; ++j) cm[j] = sm[(e0 + j) * ns];
    }
    uint32_t X[D];
    int addr[D];
    uint32_t sel[D];
#pragma unroll
    for (int j = 0; j < D; ++j) {
        const EdgeMeta16 mt = meta[e0 + j];            // one broadcast 16-byte load
        const bool wr = w >= mt.thresh;
        addr[j] = w + mt.base_nw - (wr ? H : 0);
        sel[j] = wr ? mt.sel_w : mt.sel_nw;
        X[j] = prmt(Lb[addr[j]], 0u, sel[j]);
    }
    if constexpr (kTm) twait_ld();
    uint32_t m1 = kInf2, m2 = kInf2;
#pragma unroll
    for (int j = 0; j < D; ++j) {
        const uint32_t x = h2sub(X[j], cm[j]);          // a2: v = L - c_old
        m2 = h2min(m2, h2max(h2abs(m1), h2abs(x)));     // second minimum of |v|
        m1 = h2minxs(m1, x);                            // carries the sign product
        X[j] = x;
    }
    const uint32_t SO = (m1 & kSign2) | kOne2;          // +-1.0: sign product per lane
    const uint32_t a1 = m1 & kAbs2, a2 = m2 & kAbs2;
    const uint32_t m1c = h2mul(beta2, h2relu_fma(a1, kOne2, ngamma2));
    const uint32_t m2c = h2mul(beta2, h2relu_fma(a2, kOne2, ngamma2));
#pragma unroll
    for (int j = 0; j < D; ++j) {
        const uint32_t x = X[j];
        const uint32_t is_min = h2le_mask(h2abs(x), a1);
        const uint32_t mag = (is_min & m2c) | (~is_min & m1c);
        const uint32_t sg = (x & kSign2) ^ SO;          // S xor sgn(v), as +-1.0
        cm[j] = h2mul(mag, sg);                         // a4: c_new (exact)
        const uint32_t L = h2fma(mag, sg, x);           // v + c_new, rounded once
        if (store) Lb[addr[j]] = prmt(L, 0u, sel[j]);
    }
    if constexpr (kTm) {
        tstore<D>(tcol, cm);
    } else {
#pragma unroll
        for (int j = 0; j < D; ++j) sm[(e0 + j) * ns] = cm[j];
    }
}

#ifndef LDPC_T16_ROWS
template <bool kTm>
__device__ __forceinline__ void dispatch16(int d, const EdgeMeta16 *meta, uint32_t *Lb,
                                           uint32_t tcol, uint32_t *sm, int ns, int e0, int H,
                                           int w, bool store, uint32_t beta2, uint32_t ngamma2) {
    switch (d) {
#define LDPC_T16_CASE(D)                                                                 \
    case D:                                                                              \
        row16<D, kTm>(meta, Lb, tcol, sm, ns, e0, H, w, store, beta2, ngamma2);          \
        break;
        LDPC_T16_CASE(2) LDPC_T16_CASE(3) LDPC_T16_CASE(4) LDPC_T16_CASE(5) LDPC_T16_CASE(6)
        LDPC_T16_CASE(7) LDPC_T16_CASE(8) LDPC_T16_CASE(9) LDPC_T16_CASE(10)
        LDPC_T16_CASE(11) LDPC_T16_CASE(12) LDPC_T16_CASE(13) LDPC_T16_CASE(14)
        LDPC_T16_CASE(15) LDPC_T16_CASE(16) LDPC_T16_CASE(17) LDPC_T16_CASE(18)
        LDPC_T16_CASE(19) LDPC_T16_CASE(20)
#undef LDPC_T16_CASE
    default:
        break;
    }
}
#endif

// row parity of the hard decisions of row pair w (sign bits of the gathered pairs)
__device__ __forceinline__ uint32_t parity16(const EdgeMeta16 *meta, const uint32_t *Lb, int e0,
                                             int d, int H, int w) {
    uint32_t par = 0;
    for (int j = 0; j < d; ++j) {
        const EdgeMeta16 mt = meta[e0 + j];
        const bool wr = w >= mt.thresh;
        const int a = w + mt.base_nw - (wr ? H : 0);
        par ^= prmt(Lb[a], 0u, wr ? mt.sel_w : mt.sel_nw);
    }
    return par & kSign2;
}

// kCw codewords per block (1, 2 or 4).  Without kHybrid every message is in TMEM; with it
// the first tm_warps warps keep their messages in TMEM and the remaining threads in shared
// memory (shapes whose messages do not fit TMEM for every warp of the block).
// The whole kernel body; tmem16_kernel (decode_tmem16.cu, and the kernels compiled at run
// time for a row sequence, t16_jit.cu) only wraps it.  LDPC_T16_ROWS, when defined, is the
// row sequence as LDPC_T16Q(D, e0, r) entries (possibly inside loops over repeated blocks):
// the layer loop is then straight-line code without the per-row dispatch.
template <int kCw, bool kHybrid>
__device__ __forceinline__ void t16_body(const Tmem16Params &pp) {
    const DecodeParams &p = pp.p;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ uint32_t s_tmem_base;
    __shared__ __align__(8) uint64_t s_bar[kCw];
    __shared__ int s_stop[kCw][2];                    // per codeword: a failing check found
    const int Z = p.Z, H = pp.H, E = p.E, n_rows = p.n_rows, n_cols = p.n_cols;
    const int tid = threadIdx.x, warp = tid >> 5;
    const int nthr_half = pp.wpc * 32;
    const int half = kCw > 1 ? tid / nthr_half : 0;   // codeword slot of this thread
    const int ht = tid - half * nthr_half;            // thread index within the codeword
    const bool store = ht < H;
    const int w = store ? ht : H - 1;                 // spare threads shadow the last row pair
    const bool use_tm = !kHybrid || warp < pp.tm_warps;
    EdgeMeta16 *s_meta = reinterpret_cast<EdgeMeta16 *>(smem);
    uint32_t *Lb = reinterpret_cast<uint32_t *>(smem + pp.off_lb) + (size_t)half * n_cols * H;
    const uint16_t *stage =
        reinterpret_cast<const uint16_t *>(smem + pp.off_stage + (size_t)half * pp.stage_bytes);
    uint64_t *bar = &s_bar[half];
    // shared-memory messages of this thread (kCw = 1, threads beyond the TMEM warps)
    uint32_t *sm = reinterpret_cast<uint32_t *>(smem + pp.off_msg) +
                   (use_tm ? 0 : tid - pp.tm_warps * 32);
    const int ns = pp.ns;

    for (int e = tid; e < E; e += blockDim.x) s_meta[e] = pp.meta[e];
    if (ht == 0 && pp.use_tma) mbar_init(bar);
    if (warp == 0) tmem_alloc(&s_tmem_base, (uint32_t)pp.tcols);
    tmem_block_sync();
    // this warp's lane quarter and column region
    const uint32_t tbase = s_tmem_base + ((uint32_t)((warp & 3) * 32) << 16) +
                           (uint32_t)((warp >> 2) * E);

    const int bar_id = 1 + half;
    const int K = p.K_b * Z;
    const int nbytes = (K + 7) >> 3;
    const int lo = p.punct * Z;
    const uint16_t *llr_all = reinterpret_cast<const uint16_t *>(p.llr);
    const int stride = kCw * gridDim.x;
    const int cw0 = kCw * blockIdx.x + half;
    uint32_t parity = 0;
    bool failed = false;
    if (pp.use_tma && ht == 0 && cw0 < p.batch)
        bulk_load(const_cast<uint16_t *>(stage), llr_all + in_row(p, cw0) * p.n_tx,
                  (uint32_t)(2 * p.n_tx), bar);

    for (int cw = cw0; cw - half < p.batch; cw += stride) {
        if (cw < p.batch && !failed) {
            // a0: zero messages; posteriors from the channel LLRs (-0 becomes +0)
            if (use_tm) {
                uint32_t z[8];
#pragma unroll
                for (int k = 0; k < 8; ++k) z[k] = 0u;
                int c = 0;
                for (; c + 8 <= E; c += 8) tst<8>(tbase + c, z);
                for (; c < E; ++c) tst<1>(tbase + c, z);
            } else {
                for (int e = 0; e < E; ++e) sm[e * ns] = 0u;
            }
            const uint16_t *src = llr_all + in_row(p, cw) * p.n_tx;
            if (pp.use_tma) {
                const bool ok = mbar_wait(bar, parity);
                if (named_or(bar_id, nthr_half, !ok)) {
                    if (ht == 0) atomicCAS(p.status, 0, kStatusTimeout);
                    failed = true;           // parity stays on the copy still in flight
                } else {
                    parity ^= 1u;
                }
                src = stage;
            }
            if (!failed) {
                for (int c = 0; c < n_cols; ++c) {
                    for (int j = ht; j < H; j += nthr_half) {
                        const int t0 = c * Z + j - lo, t1 = t0 + H;
                        const uint32_t b0 = (t0 >= 0 && t0 < p.n_tx) ? src[t0] : 0u;
                        const uint32_t b1 = (t1 >= 0 && t1 < p.n_tx) ? src[t1] : 0u;
                        Lb[c * H + j] = h2add(b0 | (b1 << 16), 0u);
                    }
                }
                named_sync(bar_id, nthr_half);
                if (pp.use_tma && ht == 0 && cw + stride < p.batch)
                    bulk_load(const_cast<uint16_t *>(stage),
                              llr_all + in_row(p, cw + stride) * p.n_tx,
                              (uint32_t)(2 * p.n_tx), bar);

                if (kCw != 4 && ht == 0) s_stop[half][0] = s_stop[half][1] = 0;   // by a barrier
                int r_scan = 0;                      // first layer of this warp's next scan
                int done = p.max_iter;
#pragma unroll 1
                for (int t = 1; t <= p.max_iter; ++t) {
#ifdef LDPC_T16_ROWS
#define LDPC_T16Q(D, E0, R)                                                                \
    {                                                                                      \
        uint32_t beta2 = pp.beta2, ngamma2 = pp.ngamma2;                                   \
        if (pp.learned) {                                                                  \
            const float *q = p.learned + ((size_t)(t - 1) * n_rows + (R)) * 2;             \
            beta2 = h2_from_float(q[0]);                                                   \
            ngamma2 = h2_from_float(-q[1]);                                                \
        }                                                                                  \
        if (use_tm)                                                                        \
            row16<D, true>(s_meta, Lb, tbase + (uint32_t)(E0), sm, ns, E0, H, w, store,    \
                           beta2, ngamma2);                                                \
        else                                                                               \
            row16<D, false>(s_meta, Lb, 0u, sm, ns, E0, H, w, store, beta2, ngamma2);      \
        named_sync(bar_id, nthr_half);                                                     \
    }
                    LDPC_T16_ROWS
#undef LDPC_T16Q
#else
#pragma unroll 1
                    for (int r = 0; r < n_rows; ++r) {
                        const int e0 = pp.row[r], d = pp.row[r + 1] - e0;
                        uint32_t beta2 = pp.beta2, ngamma2 = pp.ngamma2;
                        if (pp.learned) {
                            const float *q = p.learned + ((size_t)(t - 1) * n_rows + r) * 2;
                            beta2 = h2_from_float(q[0]);
                            ngamma2 = h2_from_float(-q[1]);
                        }
                        if (use_tm)
                            dispatch16<true>(d, s_meta, Lb, tbase + (uint32_t)e0, sm, ns, e0, H,
                                             w, store, beta2, ngamma2);
                        else
                            dispatch16<false>(d, s_meta, Lb, 0u, sm, ns, e0, H, w, store, beta2,
                                              ngamma2);
                        named_sync(bar_id, nthr_half);
                    }
#endif
                    if (p.early_stop) {
                        if constexpr (kCw == 4) {
                            // four codewords per block: the plain per-warp scan (measured
                            // faster for this instance than the block-wide exit below)
                            int bad = 0;
                            for (int r = 0; r < n_rows && !bad; ++r) {
                                const int e0 = pp.row[r], d = pp.row[r + 1] - e0;
                                bad = __any_sync(0xffffffffu,
                                                 parity16(s_meta, Lb, e0, d, H, w) != 0u);
                            }
                            if (named_or(bar_id, nthr_half, bad) == 0) {
                                done = t;
                                break;
                            }
                        } else {
                            // block-wide exit within the codeword's half: the first warp to
                            // find a failing check raises its flag and every warp of the half
                            // stops; each warp starts at its last failing layer
                            volatile int *vstop = &s_stop[half][t & 1];
                            int bad = 0, r = r_scan;
                            for (int q = 0; q < n_rows && !bad && !*vstop;
                                 ++q, r = (r + 1 == n_rows) ? 0 : r + 1) {
                                const int e0 = pp.row[r], d = pp.row[r + 1] - e0;
                                bad = __any_sync(0xffffffffu,
                                                 parity16(s_meta, Lb, e0, d, H, w) != 0u);
                                if (bad) {
                                    if ((tid & 31) == 0) *vstop = 1;
                                    r_scan = r;
                                }
                            }
                            const int any = named_or(bar_id, nthr_half, bad);
                            if (ht == 0) s_stop[half][(t + 1) & 1] = 0;   // read an iteration ago
                            if (any == 0) {
                                done = t;
                                break;
                            }
                        }
                    }
                }

                // a6: outputs
                for (int b = ht; b < nbytes; b += nthr_half) {
                    unsigned x = 0;
                    int c = (8 * b) / Z, i = 8 * b - c * Z;    // bit j = c Z + i, stepped
                    for (int kk = 0; kk < 8 && 8 * b + kk < K; ++kk) {
                        const int lane = i >= H ? 1 : 0;
                        const uint32_t wd = Lb[c * H + i - lane * H];
                        if ((lane ? (wd >> 31) : (wd >> 15)) & 1u) x |= 1u << kk;
                        if (++i == Z) {
                            i = 0;
                            ++c;
                        }
                    }
                    p.bits[out_row(p, cw) * nbytes + b] = (uint8_t)x;
                }
                if (ht == 0) p.iters[out_row(p, cw)] = done;
                if (p.post) {
                    uint16_t *po = reinterpret_cast<uint16_t *>(p.post) + (size_t)cw * n_cols * Z;
                    for (int c = 0; c < n_cols; ++c)
                        for (int i = ht; i < Z; i += nthr_half) {
                            const int lane = i >= H ? 1 : 0;
                            const uint32_t wd = Lb[c * H + i - lane * H];
                            po[c * Z + i] = (uint16_t)(lane ? (wd >> 16) : (wd & 0xffffu));
                        }
                }
                if (p.c2v) {
                    if (use_tm) twait_st();
                    uint16_t *co = reinterpret_cast<uint16_t *>(p.c2v) + (size_t)cw * E * Z;
                    for (int e = 0; e < E; ++e) {
                        uint32_t v;
                        if (use_tm) {
                            tld<1>(tbase + (uint32_t)e, &v);
                            twait_ld();
                        } else {
                            v = sm[e * ns];
                        }
                        if (store) {
                            co[e * Z + w] = (uint16_t)(v & 0xffffu);
                            co[e * Z + w + H] = (uint16_t)(v >> 16);
                        }
                    }
                }
            }
        }
        named_sync(bar_id, nthr_half);
    }
    // a copy that never completed must not outlive the block: wait for it (bounded)
    if (failed && ht == 0) mbar_wait(bar, parity);

    if (use_tm) twait_st();
    tmem_block_sync();
    if (warp == 0) tmem_dealloc(s_tmem_base, (uint32_t)pp.tcols);
}

}  // namespace
}  // namespace ldpc

#ifdef LDPC_T16_ROWS
// the kernel of a runtime-compiled module (LDPC_T16_CW codewords per block, LDPC_T16_HYB:
// messages of the warps beyond TMEM's 512 columns in shared memory)
extern "C" __global__ void __launch_bounds__(384, 1)
    tmem16_kernel(const __grid_constant__ ldpc::Tmem16Params pp) {
    ldpc::t16_body<LDPC_T16_CW, LDPC_T16_HYB>(pp);
}
#endif
