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
#include <cuda_fp16.h>

#include "f16x2.h"
#include "ldpc_internal.h"
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
// (x, x) rounded to binary16, as a lane pair
__host__ __device__ __forceinline__ uint32_t h2_from_float(float x) {
    const __half_raw r = __float2half_rn(x);
    const uint32_t h = r.x;
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
template <int kCw, bool kHybrid>
__global__ void __launch_bounds__(384, 1) tmem16_kernel(const __grid_constant__ Tmem16Params pp) {
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
                    if (ht == 0) atomicCAS(p.status, 0, (int)LDPC_ERR_TIMEOUT);
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

// Block shape: codewords per block, warps per codeword, warps with messages in TMEM (the
// rest in shared memory), and TMEM columns allocated.
struct Shape16 {
    int cw, wpc, tm_warps, ns, tcols;
};

Shape16 make_shape16(const DecodeParams &p, int cw) {
    Shape16 s;
    s.cw = cw;
    s.wpc = (p.Z / 2 + 31) / 32;
    const int fit = p.E > 0 ? kTmemCols16 / p.E : 0;       // column regions that fit
    const int warps = cw * s.wpc;
    s.tm_warps = warps < 4 * fit ? warps : 4 * fit;
    s.ns = (warps - s.tm_warps) * 32;
    const int need = ((s.tm_warps + 3) / 4) * p.E;
    s.tcols = 32;
    while (s.tcols < need) s.tcols <<= 1;
    return s;
}

struct Layout16 {
    size_t off_lb, off_msg, off_stage, stage_bytes, total;
};

Layout16 layout16(const DecodeParams &p, const Shape16 &sh, bool tma) {
    Layout16 l;
    const int H = p.Z / 2;
    size_t off = (size_t)p.E * sizeof(EdgeMeta16);
    off = (off + 15) & ~(size_t)15;
    l.off_lb = off;
    off += (size_t)sh.cw * p.n_cols * H * 4;
    l.off_msg = off;
    off += (size_t)p.E * sh.ns * 4;
    off = (off + 15) & ~(size_t)15;                  // bulk-copy destinations: 16-byte aligned
    l.off_stage = off;
    l.stage_bytes = ((size_t)2 * p.n_tx + 15) & ~(size_t)15;
    if (tma) off += (size_t)sh.cw * l.stage_bytes;
    l.total = off;
    return l;
}

// Preference: four codewords per block when its warps fit one block (small Z), the shared
// memory holds them and the batch fills every SM with more than two codewords (throughput);
// else two codewords with every message in TMEM (also the lower-latency choice for small
// batches, which then spread over more SMs); else one.
Shape16 shape16(const DecodeParams &p, size_t smem_optin, int n_sm) {
    const int wpc = (p.Z / 2 + 31) / 32;
    if (4 * wpc <= 12 && p.batch > 2 * n_sm) {
        const Shape16 s4 = make_shape16(p, 4);
        if (s4.tm_warps >= 1 && layout16(p, s4, false).total <= smem_optin) return s4;
    }
    const Shape16 s2 = make_shape16(p, 2);
    if (s2.ns == 0) return s2;
    return make_shape16(p, 1);
}

}  // namespace

bool tmem16_supported(const DecodeParams &p, int llr_type, int max_deg, size_t smem_optin) {
    if (llr_type != LDPC_LLR_FP16) return false;
    if (p.algo != LDPC_NORMALISED && p.algo != LDPC_OFFSET && p.algo != LDPC_LEARNED) return false;
    if ((p.Z & 1) || p.Z < 2 || p.Z > 384 || max_deg > kMaxDeg16 || max_deg < 2) return false;
    if (p.E > kMaxEdges16 || p.n_rows > kMaxRows16) return false;
    // supported when the two-codeword or one-codeword shape fits (the four-codeword shape
    // is an alternative for large batches only)
    const Shape16 sh = shape16(p, smem_optin, 1 << 30);
    if (sh.tm_warps < 1 || sh.tcols > kTmemCols16) return false;
    return layout16(p, sh, false).total <= smem_optin;
}

ldpc_status launch_tmem16(const DecodeParams &p, cudaStream_t stream) {
    static thread_local Tmem16Params pp;   // ~9 kB: kept off the stack
    pp.p = p;
    const int H = p.Z / 2;
    int dev = 0, smem_optin = 0, n_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return LDPC_ERR_CUDA;
    cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    const Shape16 sh = shape16(p, (size_t)smem_optin, n_sm);
    pp.H = H;
    pp.wpc = sh.wpc;
    pp.tcols = sh.tcols;
    pp.tm_warps = sh.tm_warps;
    pp.ns = sh.ns;
    pp.learned = p.algo == LDPC_LEARNED ? 1 : 0;
    if (p.algo == LDPC_NORMALISED) {
        pp.beta2 = h2_from_float(p.alpha);
        pp.ngamma2 = 0u;
    } else {
        pp.beta2 = kOne2;
        pp.ngamma2 = h2_from_float(-p.offset);
    }
    for (int r = 0; r <= p.n_rows; ++r) pp.row[r] = p.h_row_ptr[r];
    for (int e = 0; e < p.E; ++e) {
        const uint32_t ed = p.h_edges[e];
        const int c = (int)(ed >> 16), s = (int)(ed & 0xffffu);
        const int q = s >= H ? 1 : 0, u = s - q * H;
        pp.meta[e].base_nw = c * H + u;
        pp.meta[e].thresh = H - u;
        pp.meta[e].sel_nw = q ? 0x1032u : 0x3210u;
        pp.meta[e].sel_w = q ? 0x3210u : 0x1032u;
    }
    const bool aligned = ((uintptr_t)p.llr % 16 == 0) && (p.n_tx % 8 == 0) && p.n_tx > 0;
    pp.use_tma = (aligned && layout16(p, sh, true).total <= (size_t)smem_optin) ? 1 : 0;
    const Layout16 l = layout16(p, sh, pp.use_tma != 0);
    pp.off_lb = (int)l.off_lb;
    pp.off_msg = (int)l.off_msg;
    pp.off_stage = (int)l.off_stage;
    pp.stage_bytes = (int)l.stage_bytes;
    const bool hybrid = sh.ns > 0;
    auto kern = sh.cw == 4 ? (hybrid ? tmem16_kernel<4, true> : tmem16_kernel<4, false>)
              : sh.cw == 2 ? tmem16_kernel<2, false>
                           : (hybrid ? tmem16_kernel<1, true> : tmem16_kernel<1, false>);
    // blocks per SM: as many as shared memory and the 512 TMEM columns allow; the shared
    // memory request is raised so that no more blocks fit than TMEM can hold (a block
    // beyond that would only wait in tcgen05.alloc)
    const int by_tmem = kTmemCols16 / sh.tcols;
    int smem_sm = 0;
    cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    size_t smem = l.total;
    const size_t floor_b = (size_t)smem_sm / (by_tmem + 1) + 1024;
    if (smem < floor_b && floor_b <= (size_t)smem_optin) smem = floor_b;
    if (set_dyn_smem(reinterpret_cast<const void *>(kern), smem) !=
        cudaSuccess)
        return LDPC_ERR_CUDA;
    const int threads = sh.cw * sh.wpc * 32;
    int per_sm = 0;
    if (blocks_per_sm(&per_sm, reinterpret_cast<const void *>(kern), threads, smem) !=
            cudaSuccess ||
        per_sm < 1)
        return LDPC_ERR_UNSUPPORTED;
    if (per_sm > by_tmem) per_sm = by_tmem;
    int grid = n_sm * per_sm;
    const int units = (p.batch + sh.cw - 1) / sh.cw;
    if (grid > units) grid = units;
    if (grid < 1) grid = 1;
    kern<<<grid, threads, smem, stream>>>(pp);
    count_launch();
    if (cudaGetLastError() != cudaSuccess) return LDPC_ERR_CUDA;
    return LDPC_OK;
}

}  // namespace ldpc
