// Layered min-sum, 8-bit offset variant, with the check-to-variable messages held in
// Tensor Memory (sm_103a).  Paper: Sec. III (layered min-sum with correction, stopping
// rule), Sec. IV (per-row m1 / m2 / sign quantities); hot-path steps a0..a6.
//
// Why TMEM.  A BG1-shaped codeword at Z = 384 needs 52 kB of posteriors (shared by all
// check rows through the circulant gather) and 124 kB of messages that only their own
// check row ever reads.  Shared memory can hold one codeword, which leaves one codeword's
// serial chain of 460 layer barriers per SM and a latency-bound SM.  The messages are
// private per row, so they go to Tensor Memory instead: tcgen05.ld / tcgen05.st of shape
// 32x32b give every thread its own TMEM lane with warp-uniform, run-time column indices.
// The 256 kB of TMEM hold the messages of two codewords; shared memory holds their two
// posterior arrays.  A thread block decodes two codewords at once, each with its own
// named barrier, so one codeword's barrier and load latency overlaps the other's work.
//
// Mapping (per codeword half of the block): thread w owns check rows w and w + H
// (H = Z/2) of every layer, carried as two binary16 lanes (exact for 8-bit values); the
// posterior words, circulant gather with half swap, and xorsign min-sum follow
// decode_rowpair.cu, with two changes that move work from the integer / min-max pipe to the
// FMA pipe: posteriors are biased by 1279 (binary16 L + 1279 on [1152, 1406]) so that
// v + 127 = (L + 1279) - (c + 1152) is one subtraction, and the saturation of v to
// [-127, 127] is done by two relu FMAs, y = max(v + 127, 0), z = max(254 - y, 0),
// sat(v) = 127 - z (exact on these integers); the second minimum comes from plain
// min / max of magnitudes.  Messages are stored as
// bytes c + 128, two edges per 32-bit TMEM column, packed tightly across rows (edge e at
// column e/2, byte pair e%2), so a row's messages arrive with one or two tcgen05.ld per
// thread and leave with one or two tcgen05.st; a column shared with the neighbouring row
// is written back with that row's half unchanged.
#include "f16x2.h"
#include "ldpc_internal.h"
#include "tmem.h"

namespace ldpc {
namespace {

using namespace h2;
using namespace tm;

struct EdgeMetaT {
    int base_nw;       // c*H + u
    int thresh;        // H - u
    uint32_t sel_nw;   // 0x3210 or 0x1032
    uint32_t sel_w;
};

constexpr int kMaxEdgesT = 1024;
constexpr int kMaxRowsT = 64;
constexpr int kTmemCols = 512;

struct TmemParams {
    DecodeParams p;
    int H;
    int wpc;                     // warps per codeword half
    int ncols;                   // TMEM columns per thread: ceil(E / 2)
    int use_tma;                 // channel LLRs staged by 1-D bulk copies
    int stage_bytes;             // per-half staging buffer (multiple of 16)
    int off_lb, off_stage;       // shared-memory offsets of the posteriors and the staging
    int row[kMaxRowsT + 1];      // edge offsets of the rows
    EdgeMetaT meta[kMaxEdgesT];
};

// --------------------------------------------------------------------------- one layer

// Thread w of a codeword half processes row pair w of a layer of degree D whose first edge
// sits in the upper half of its TMEM column when P = 1.
template <int D, int P>
__device__ __forceinline__ void tm_row(const EdgeMetaT *meta, uint32_t *Lb, uint32_t tcolumn,
                                       int e0, int H, int w, bool store) {
    constexpr int NC = (P + D + 1) / 2;   // columns touched by the row
    uint32_t cm[NC];
    twait_st();                           // this thread's earlier stores to these columns
    tload<NC>(tcolumn, cm);
    uint32_t X[D];
    int addr[D];
    uint32_t sel[D];
#pragma unroll
    for (int j = 0; j < D; ++j) {
        const EdgeMetaT mt = meta[e0 + j];             // one broadcast 16-byte load
        const bool wr = w >= mt.thresh;
        addr[j] = w + mt.base_nw - (wr ? H : 0);
        sel[j] = wr ? mt.sel_w : mt.sel_nw;
        X[j] = prmt(Lb[addr[j]], 0u, sel[j]);
    }
    twait_ld();
    uint32_t m1 = kInf2, m2 = kInf2;
#pragma unroll
    for (int j = 0; j < D; ++j) {
        // message byte pair -> binary16 (c + 1152) under the exponent byte 0x64
        const uint32_t M =
            prmt(cm[(P + j) >> 1], 0x64646464u, ((P + j) & 1) ? 0x4342u : 0x4140u);
        // v = sat(L - c) from posteriors biased by 1279 through two relu FMAs (exact for
        // these integers): y = max(L - c + 127, 0), z = max(254 - y, 0), v = 127 - z
        const uint32_t y = h2relu_fma(M, kNegOne2, X[j]);
        const uint32_t z = h2relu_fma(y, kNegOne2, k254);
        const uint32_t x = h2sub(kP127, z);
        // m2 from plain min / max of magnitudes; m1 carries the sign product
        m2 = h2min(m2, h2max(h2abs(m1), h2abs(x)));
        m1 = h2minxs(m1, x);
        X[j] = x;
    }
    const uint32_t SO = (m1 & kSign2) | kOne2;               // +-1.0: sign product per lane
    const uint32_t a1 = m1 & kAbs2, a2 = m2 & kAbs2;
    const uint32_t m1c = h2relu_fma(a1, kOne2, kNegOne2);    // max(m1 - 1, 0)
    const uint32_t T1 = h2add(h2add(a1, a2), kNegOne2);       // m1 + m2 - 1
    uint32_t C[D];
#pragma unroll
    for (int j = 0; j < D; ++j) {
        const uint32_t x = X[j];
        const uint32_t ex = h2max(m1c, h2sub(T1, h2abs(x)));
        const uint32_t sg = (x & kSign2) ^ SO;                 // S xor sgn(x), as +-1.0
        C[j] = h2fma(ex, sg, kBias2);                          // c' + 1152
        uint32_t L = h2add(C[j], h2add(x, kP127));             // (x + c') + 1279
        L = h2max(h2min(L, kPostHi), kPostLo);
        if (store) Lb[addr[j]] = prmt(L, 0u, sel[j]);
    }
    // repack: low bytes of both lanes of each edge; foreign halves of the boundary columns
    // (neighbouring rows) are kept as loaded
#pragma unroll
    for (int k = 0; k < NC; ++k) {
        const int jl = 2 * k - P, jh = 2 * k + 1 - P;
        const int il = jl < 0 ? 0 : jl, ih = jh >= D ? D - 1 : jh;   // in-range indices
        if (jl >= 0 && jh < D)
            cm[k] = prmt(C[il], C[ih], 0x6420u);
        else if (jl >= 0)
            cm[k] = prmt(C[il], cm[k], 0x7620u);
        else
            cm[k] = prmt(cm[k], C[ih], 0x6410u);
    }
    tstore<NC>(tcolumn, cm);
}

template <int D>
__device__ __forceinline__ void tm_row_any(const EdgeMetaT *meta, uint32_t *Lb,
                                           uint32_t tbase, int e0, int H, int w, bool store) {
    if (e0 & 1)
        tm_row<D, 1>(meta, Lb, tbase + (uint32_t)(e0 >> 1), e0, H, w, store);
    else
        tm_row<D, 0>(meta, Lb, tbase + (uint32_t)(e0 >> 1), e0, H, w, store);
}

__device__ __forceinline__ void tm_dispatch(int d, const EdgeMetaT *meta, uint32_t *Lb,
                                            uint32_t tbase, int e0, int H, int w, bool store) {
    switch (d) {
#define LDPC_TM_CASE(D) \
    case D:             \
        tm_row_any<D>(meta, Lb, tbase, e0, H, w, store); \
        break;
        LDPC_TM_CASE(2) LDPC_TM_CASE(3) LDPC_TM_CASE(4) LDPC_TM_CASE(5) LDPC_TM_CASE(6)
        LDPC_TM_CASE(7) LDPC_TM_CASE(8) LDPC_TM_CASE(9) LDPC_TM_CASE(10) LDPC_TM_CASE(11)
        LDPC_TM_CASE(12) LDPC_TM_CASE(13) LDPC_TM_CASE(14) LDPC_TM_CASE(15) LDPC_TM_CASE(16)
        LDPC_TM_CASE(17) LDPC_TM_CASE(18) LDPC_TM_CASE(19) LDPC_TM_CASE(20)
#undef LDPC_TM_CASE
    default:
        break;
    }
}

__device__ __forceinline__ uint32_t tm_parity(const EdgeMetaT *meta, const uint32_t *Lb, int e0,
                                              int d, int H, int w) {
    uint32_t par = 0;
    for (int j = 0; j < d; ++j) {
        const EdgeMetaT mt = meta[e0 + j];
        const bool wr = w >= mt.thresh;
        const int a = w + mt.base_nw - (wr ? H : 0);
        par ^= h2lt_mask(prmt(Lb[a], 0u, wr ? mt.sel_w : mt.sel_nw), kPostBias);
    }
    return par;
}

// ---------------------------------------------------------------------------- the kernel

__global__ void __launch_bounds__(384, 1) tmem_kernel(const __grid_constant__ TmemParams pp) {
    const DecodeParams &p = pp.p;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ uint32_t s_tmem_base;
    __shared__ __align__(8) uint64_t s_bar[2];
    const int Z = p.Z, H = pp.H, E = p.E, n_rows = p.n_rows, n_cols = p.n_cols;
    const int tid = threadIdx.x, warp = tid >> 5;
    const int nthr_half = pp.wpc * 32;
    const int half = tid / nthr_half;                 // codeword slot of this thread
    const int ht = tid - half * nthr_half;            // thread index within the half
    const bool store = ht < H;
    const int w = store ? ht : H - 1;                 // spare threads shadow the last row pair
    // shared memory: edge metadata | two posterior arrays | two LLR staging buffers
    EdgeMetaT *s_meta = reinterpret_cast<EdgeMetaT *>(smem);
    uint32_t *Lb = reinterpret_cast<uint32_t *>(smem + pp.off_lb) + (size_t)half * n_cols * H;
    const int8_t *stage =
        reinterpret_cast<const int8_t *>(smem + pp.off_stage) + (size_t)half * pp.stage_bytes;
    uint64_t *bar = &s_bar[half];

    for (int e = tid; e < E; e += blockDim.x) s_meta[e] = pp.meta[e];
    if (ht == 0 && pp.use_tma) mbar_init(bar);
    // TMEM: warp 0 allocates all 512 columns for the block
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_addr(&s_tmem_base)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    // this warp's lane quarter and column region
    const uint32_t tbase = s_tmem_base + ((uint32_t)((warp & 3) * 32) << 16) +
                           (uint32_t)((warp >> 2) * pp.ncols);

    const int bar_id = 1 + half;
    const int K = p.K_b * Z;
    const int nbytes = (K + 7) >> 3;
    const int lo = p.punct * Z;
    const int8_t *llr_all = reinterpret_cast<const int8_t *>(p.llr);
    const int stride = 2 * gridDim.x;
    const int cw0 = 2 * blockIdx.x + half;
    uint32_t parity = 0;
    bool failed = false;
    if (pp.use_tma && ht == 0 && cw0 < p.batch)
        bulk_load(const_cast<int8_t *>(stage), llr_all + in_row(p, cw0) * p.n_tx,
                  (uint32_t)p.n_tx, bar);

    for (int cw = cw0; cw - half < p.batch; cw += stride) {
        // both halves run the same number of passes; a half without a codeword idles
        if (cw < p.batch && !failed) {
            // a0: zero messages; biased posteriors from the channel LLRs
            {
                uint32_t z[8];
#pragma unroll
                for (int k = 0; k < 8; ++k) z[k] = 0x80808080u;
                int c = 0;
                for (; c + 8 <= pp.ncols; c += 8) tst<8>(tbase + c, z);
                for (; c < pp.ncols; ++c) tst<1>(tbase + c, z);
            }
            const int8_t *src = llr_all + in_row(p, cw) * p.n_tx;
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
                // word (c, j) holds rows j and j + H of column block c
                for (int c = 0; c < n_cols; ++c) {
                    for (int j = ht; j < H; j += nthr_half) {
                        const int t0 = c * Z + j - lo, t1 = t0 + H;
                        // binary16 L + 1279 = 1024 + (L + 255): bit pattern 0x6400 + L + 255
                        const int q0 = (t0 >= 0 && t0 < p.n_tx) ? (int)src[t0] : 0;
                        const int q1 = (t1 >= 0 && t1 < p.n_tx) ? (int)src[t1] : 0;
                        Lb[c * H + j] = (uint32_t)(0x64FF + q0) | ((uint32_t)(0x64FF + q1) << 16);
                    }
                }
                named_sync(bar_id, nthr_half);
                // the staging buffer is free: start the copy of this half's next codeword
                if (pp.use_tma && ht == 0 && cw + stride < p.batch)
                    bulk_load(const_cast<int8_t *>(stage), llr_all + in_row(p, cw + stride) * p.n_tx,
                              (uint32_t)p.n_tx, bar);

                int done = p.max_iter;
#pragma unroll 1
                for (int t = 1; t <= p.max_iter; ++t) {
#pragma unroll 1
                    for (int r = 0; r < n_rows; ++r) {
                        const int e0 = pp.row[r], d = pp.row[r + 1] - e0;
                        tm_dispatch(d, s_meta, Lb, tbase, e0, H, w, store);
                        named_sync(bar_id, nthr_half);
                    }
                    if (p.early_stop) {
                        int bad = 0;
                        for (int r = 0; r < n_rows && !bad; ++r) {
                            const int e0 = pp.row[r], d = pp.row[r + 1] - e0;
                            bad = __any_sync(0xffffffffu,
                                             tm_parity(s_meta, Lb, e0, d, H, w) != 0u);
                        }
                        if (named_or(bar_id, nthr_half, bad) == 0) {
                            done = t;
                            break;
                        }
                    }
                }

                // a6: outputs
                for (int b = ht; b < nbytes; b += nthr_half) {
                    unsigned x = 0;
                    for (int kk = 0; kk < 8; ++kk) {
                        const int j = 8 * b + kk;
                        if (j >= K) break;
                        const int c = j / Z, i = j - c * Z;
                        const int lane = i >= H ? 1 : 0;
                        const uint32_t wd = Lb[c * H + i - lane * H];
                        const uint32_t h = lane ? (wd >> 16) : (wd & 0xffffu);
                        if (h < 0x64FFu) x |= 1u << kk;
                    }
                    p.bits[out_row(p, cw) * nbytes + b] = (uint8_t)x;
                }
                if (ht == 0) p.iters[out_row(p, cw)] = done;
                if (p.post) {
                    int8_t *po = reinterpret_cast<int8_t *>(p.post) + (size_t)cw * n_cols * Z;
                    for (int c = 0; c < n_cols; ++c)
                        for (int i = ht; i < Z; i += nthr_half) {
                            const int lane = i >= H ? 1 : 0;
                            const uint32_t wd = Lb[c * H + i - lane * H];
                            const uint32_t h = lane ? (wd >> 16) : (wd & 0xffffu);
                            po[c * Z + i] = (int8_t)((int)h - 0x64FF);
                        }
                }
                if (p.c2v) {
                    // each thread reads its own TMEM lane: messages of rows w and w + H
                    twait_st();
                    int8_t *co = reinterpret_cast<int8_t *>(p.c2v) + (size_t)cw * E * Z;
                    for (int e = 0; e < E; ++e) {
                        uint32_t v;
                        tld<1>(tbase + (uint32_t)(e >> 1), &v);
                        twait_ld();
                        const uint32_t pr = (e & 1) ? (v >> 16) : (v & 0xffffu);
                        if (store) {
                            co[e * Z + w] = (int8_t)(uint8_t)((pr & 0xffu) ^ 0x80u);
                            co[e * Z + w + H] =
                                (int8_t)(uint8_t)(((pr >> 8) & 0xffu) ^ 0x80u);
                        }
                    }
                }
            }
        }
        named_sync(bar_id, nthr_half);
    }
    // a copy that never completed must not outlive the block: wait for it (bounded)
    if (failed && ht == 0) mbar_wait(bar, parity);

    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(s_tmem_base),
                     "r"(kTmemCols)
                     : "memory");
}

int tmem_columns_per_thread(const DecodeParams &p) { return (p.E + 1) / 2; }

}  // namespace

bool tmem_supported(const DecodeParams &p, int llr_type, int max_deg, size_t smem_optin) {
    if (llr_type != LDPC_LLR_INT8 || p.algo != LDPC_OFFSET || p.offset_q != 1) return false;
    if ((p.Z & 1) || p.Z < 2 || p.Z > 384 || max_deg > kMaxDeg || max_deg < 2) return false;
    if (p.E > kMaxEdgesT || p.n_rows > kMaxRowsT) return false;
    const int H = p.Z / 2, wpc = (H + 31) / 32;
    const int depth = (2 * wpc + 3) / 4;
    if (depth * tmem_columns_per_thread(p) > kTmemCols) return false;
    const size_t need = (size_t)p.E * sizeof(EdgeMetaT) + 32 + (size_t)2 * p.n_cols * H * 4 +
                        2 * (size_t)p.n_tx + 64;
    return need <= smem_optin;
}

ldpc_status launch_tmem(const DecodeParams &p, cudaStream_t stream) {
    static thread_local TmemParams pp;     // ~17 kB: kept off the stack
    pp.p = p;
    const int H = p.Z / 2;
    pp.H = H;
    pp.wpc = (H + 31) / 32;
    for (int r = 0; r <= p.n_rows; ++r) pp.row[r] = p.h_row_ptr[r];
    pp.ncols = tmem_columns_per_thread(p);
    for (int e = 0; e < p.E; ++e) {
        const uint32_t ed = p.h_edges[e];
        const int c = (int)(ed >> 16), sh = (int)(ed & 0xffffu);
        const int q = sh >= H ? 1 : 0, u = sh - q * H;
        pp.meta[e].base_nw = c * H + u;
        pp.meta[e].thresh = H - u;
        pp.meta[e].sel_nw = q ? 0x1032u : 0x3210u;
        pp.meta[e].sel_w = q ? 0x3210u : 0x1032u;
    }
    // shared memory: metadata | two posterior arrays | two LLR staging buffers; at least
    // 120 kB so that a single block occupies the SM (its TMEM allocation takes all 512
    // columns).  Bulk copies need 16-byte aligned rows.
    pp.use_tma = ((reinterpret_cast<uintptr_t>(p.llr) & 15u) == 0 && (p.n_tx % 16) == 0 &&
                  p.n_tx > 0 && p.n_tx < (1 << 20))
                     ? 1
                     : 0;
    pp.stage_bytes = pp.use_tma ? p.n_tx : 0;
    pp.off_lb = (int)(((size_t)p.E * sizeof(EdgeMetaT) + 15) & ~(size_t)15);
    pp.off_stage = (pp.off_lb + 2 * p.n_cols * H * 4 + 15) & ~15;
    size_t smem = (size_t)pp.off_stage + 2 * (size_t)pp.stage_bytes;
    if (smem < 120 * 1024) smem = 120 * 1024;
    int dev = 0, n_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return LDPC_ERR_CUDA;
    cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    if (cudaFuncSetAttribute(tmem_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem) != cudaSuccess)
        return LDPC_ERR_CUDA;
    const int threads = 2 * pp.wpc * 32;
    int grid = (p.batch + 1) / 2;
    if (grid > n_sm) grid = n_sm;
    tmem_kernel<<<grid, threads, smem, stream>>>(pp);
    count_launch();
    if (cudaGetLastError() != cudaSuccess) return LDPC_ERR_CUDA;
    return LDPC_OK;
}

}  // namespace ldpc
