// Row step of the low-latency strategy and the body of its work-list kernel, shared by
// decode_tmem_ll.cu (tmem_ll_kernel and the generic list_ll_kernel) and by the list kernels
// compiled at run time for a set of row sequences (list_jit.cu).  Device code only.
//
// Layered min-sum, 8-bit offset variant, low-latency strategy: A cooperating threads per
// check-row pair (paper Sec. IV, the low-latency decoder: N_thread = (alpha / rho) Z with
// rho = 2 rows per thread here, and the min / sub-min / sign of a row combined across the
// alpha threads by a parallel reduce in log2(alpha) warp-shuffle steps, Fig. 3).
//
// One codeword per thread block (the decode of a lone codeword, or of a batch no larger
// than the SM count).  Thread t serves row pair w = t / A of every layer, as cooperating
// thread k = t % A: of a layer's d circulants it takes edges k, k + A, k + 2A, ...  Every
// thread runs ceil(d / A) edge slots; a slot past the row's last edge is a dummy whose
// v2c is +127 (the largest magnitude, sign +), which changes neither the minimum, the
// second minimum nor the sign product, and which writes nothing back.
//
// Arithmetic and exactness follow the batch kernel (pair_kernel.cuh): posteriors as
// binary16 L + 1279 in shared memory, messages as bytes c + 128 in Tensor Memory,
// saturation of v by two relu FMAs, new magnitude max(m1', (m1 + m2 - 1) - |v|).  The lanes
// hold rows j and j + Z/2 of the one codeword (as in decode_rowpair.cu): row pair j of a
// circulant with shift s = qH + u reads word (j + u) mod H, halves exchanged when q xor
// wrap.  Messages: two edge slots per 32-bit column of the thread's own lane, packed
// tightly across rows (a thread's slots of row r follow those of row r - 1).  The reduce
// across the A threads is exact: m1 and the sign product combine by min.xorsign, and
// m2 = min(m2a, m2b, max(|m1a|, |m1b|)).
#pragma once

#include "f16x2.h"
#include "ldpc_params.h"
#include "tmem.h"

namespace ldpc {
namespace {

using namespace h2;
using namespace tm;

struct EdgeMetaL {
    int base_nw;       // c*H + u
    int thresh;        // H - u
    uint32_t sel_nw;   // 0x3210 or 0x1032
    uint32_t sel_w;
};

constexpr int kMaxEdgesL = 1024;
constexpr int kMaxRowsL = 64;
constexpr int kTmemColsL = 512;

// --------------------------------------------------------------------------- one layer

// Cooperating thread k of row pair w on a layer of degree D, with DA = ceil(D / A) slots
// whose first slot sits in the upper half of its TMEM column when P = 1.
template <int A, int DA, int P>
__device__ __forceinline__ void ll_row(const EdgeMetaL *meta, uint32_t *Lb, uint32_t tcolumn,
                                       int e0, int D, int H, int w, int k, bool store) {
    constexpr int NC = (P + DA + 1) / 2;   // columns touched by the row's slots
    uint32_t cm[NC];
    twait_st();                            // this thread's earlier stores to these columns
    tload<NC>(tcolumn, cm);
    const bool last_real = k + A * (DA - 1) < D;
    uint32_t X[DA];
    int addr[DA];
    uint32_t sel[DA];
#pragma unroll
    for (int i = 0; i < DA; ++i) {
        const int j = (i == DA - 1 && !last_real) ? D - 1 : k + A * i;   // dummy reads a real edge
        const EdgeMetaL mt = meta[e0 + j];
        const bool wr = w >= mt.thresh;
        addr[i] = w + mt.base_nw - (wr ? H : 0);
        sel[i] = wr ? mt.sel_w : mt.sel_nw;
        X[i] = prmt(Lb[addr[i]], 0u, sel[i]);
    }
    twait_ld();
    uint32_t m1 = kInf2, m2 = kInf2;
#pragma unroll
    for (int i = 0; i < DA; ++i) {
        const uint32_t M =
            prmt(cm[(P + i) >> 1], 0x64646464u, ((P + i) & 1) ? 0x4342u : 0x4140u);
        const uint32_t y = h2relu_fma(M, kNegOne2, X[i]);   // max(v + 127, 0)
        const uint32_t z = h2relu_fma(y, kNegOne2, k254);   // max(254 - y, 0)
        uint32_t x = h2sub(kP127, z);                       // sat(v)
        if (i == DA - 1 && !last_real) x = kP127;
        m2 = h2min(m2, h2max(h2abs(m1), h2abs(x)));
        m1 = h2minxs(m1, x);
        X[i] = x;
    }
    // parallel reduce across the A threads of the row pair (adjacent lanes of one warp)
#pragma unroll
    for (int o = 1; o < A; o <<= 1) {
        const uint32_t o1 = __shfl_xor_sync(0xffffffffu, m1, o);
        const uint32_t o2 = __shfl_xor_sync(0xffffffffu, m2, o);
        m2 = h2min(h2min(m2, o2), h2max(h2abs(m1), h2abs(o1)));
        m1 = h2minxs(m1, o1);
    }
    const uint32_t SO = (m1 & kSign2) | kOne2;               // +-1.0: sign product per lane
    const uint32_t a1 = m1 & kAbs2, a2 = m2 & kAbs2;
    const uint32_t m1c = h2relu_fma(a1, kOne2, kNegOne2);    // max(m1 - 1, 0)
    const uint32_t T1 = h2add(h2add(a1, a2), kNegOne2);       // m1 + m2 - 1
    uint32_t C[DA];
#pragma unroll
    for (int i = 0; i < DA; ++i) {
        const uint32_t x = X[i];
        const uint32_t ex = h2max(m1c, h2sub(T1, h2abs(x)));
        const uint32_t sg = (x & kSign2) ^ SO;
        C[i] = h2fma(ex, sg, kBias2);                          // c' + 1152
        uint32_t L = h2add(C[i], h2add(x, kP127));             // (x + c') + 1279
        L = h2max(h2min(L, kPostHi), kPostLo);
        if (store && (i < DA - 1 || last_real)) Lb[addr[i]] = prmt(L, 0u, sel[i]);
    }
#pragma unroll
    for (int q = 0; q < NC; ++q) {
        const int jl = 2 * q - P, jh = 2 * q + 1 - P;
        const int il = jl < 0 ? 0 : jl, ih = jh >= DA ? DA - 1 : jh;
        if (jl >= 0 && jh < DA)
            cm[q] = prmt(C[il], C[ih], 0x6420u);
        else if (jl >= 0)
            cm[q] = prmt(C[il], cm[q], 0x7620u);
        else
            cm[q] = prmt(cm[q], C[ih], 0x6410u);
    }
    tstore<NC>(tcolumn, cm);
}

template <int A, int DA>
__device__ __forceinline__ void ll_row_any(const EdgeMetaL *meta, uint32_t *Lb, uint32_t tbase,
                                           int s0, int e0, int D, int H, int w, int k,
                                           bool store) {
    if (s0 & 1)
        ll_row<A, DA, 1>(meta, Lb, tbase + (uint32_t)(s0 >> 1), e0, D, H, w, k, store);
    else
        ll_row<A, DA, 0>(meta, Lb, tbase + (uint32_t)(s0 >> 1), e0, D, H, w, k, store);
}

template <int A>
__device__ __forceinline__ void ll_dispatch(int D, const EdgeMetaL *meta, uint32_t *Lb,
                                            uint32_t tbase, int s0, int e0, int H, int w, int k,
                                            bool store) {
    const int DA = (D + A - 1) / A;
    switch (DA) {
#define LDPC_LL_CASE(N)                                                          \
    case N:                                                                      \
        if constexpr (N * A < kMaxDeg + A)                                       \
            ll_row_any<A, N>(meta, Lb, tbase, s0, e0, D, H, w, k, store);         \
        break;
        LDPC_LL_CASE(1) LDPC_LL_CASE(2) LDPC_LL_CASE(3) LDPC_LL_CASE(4) LDPC_LL_CASE(5)
        LDPC_LL_CASE(6) LDPC_LL_CASE(7) LDPC_LL_CASE(8) LDPC_LL_CASE(9) LDPC_LL_CASE(10)
#undef LDPC_LL_CASE
    default:
        break;
    }
}

// parity of the hard decisions of row pair w over a row's edges, combined over the A
// threads (each takes edges k, k + A, ...); 0 when both rows of the pair are satisfied
template <int A>
__device__ __forceinline__ uint32_t ll_parity(const EdgeMetaL *meta, const uint32_t *Lb, int e0,
                                              int D, int H, int w, int k) {
    uint32_t par = 0;
    for (int j = k; j < D; j += A) {
        const EdgeMetaL mt = meta[e0 + j];
        const bool wr = w >= mt.thresh;
        const int a = w + mt.base_nw - (wr ? H : 0);
        par ^= h2lt_mask(prmt(Lb[a], 0u, wr ? mt.sel_w : mt.sel_nw), kPostBias);
    }
#pragma unroll
    for (int o = 1; o < A; o <<= 1) par ^= __shfl_xor_sync(0xffffffffu, par, o);
    return par;
}

struct LlParams {
    DecodeParams p;
    int H;
    int ncols;                   // TMEM columns per thread: ceil(total slots / 2)
    int use_tma;                 // channel LLRs staged by a 1-D bulk copy
    int off_lb, off_stage;       // shared-memory offsets of the posteriors and the staging
    int row[kMaxRowsL + 1];      // edge offsets of the rows
    int slot[kMaxRowsL + 1];     // slot offsets of the rows in every thread's TMEM lane
    EdgeMetaL meta[kMaxEdgesL];
};

// The low-latency kernel's body (one codeword per block, A cooperating threads per row
// pair); tmem_ll_kernel (decode_tmem_ll.cu, and the kernels compiled at run time for a row
// sequence, list_jit.cu) only wraps it.  LDPC_LL_ROWS, when defined, is the row sequence
// as LDPC_LLR(D, P, s0, e0) entries: the layer loop is then straight-line code.
template <int A>
__device__ __forceinline__ void ll_body(const LlParams &pp) {
    const DecodeParams &p = pp.p;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ uint32_t s_tmem_base;
    __shared__ __align__(8) uint64_t s_bar;
    __shared__ int s_stop[2];                         // a failing check found (per iteration parity)
    const int Z = p.Z, H = pp.H, E = p.E, n_rows = p.n_rows, n_cols = p.n_cols;
    const int tid = threadIdx.x, warp = tid >> 5, nthr = blockDim.x;
    const int k = tid % A;                            // cooperating thread of the row pair
    const bool store = tid / A < H;
    const int w = store ? tid / A : H - 1;            // spare groups shadow the last row pair
    // shared memory: edge metadata | posterior words | LLR staging buffer
    EdgeMetaL *s_meta = reinterpret_cast<EdgeMetaL *>(smem);
    uint32_t *Lb = reinterpret_cast<uint32_t *>(smem + pp.off_lb);
    const int8_t *stage = reinterpret_cast<const int8_t *>(smem + pp.off_stage);
    uint64_t *bar = &s_bar;

    for (int e = tid; e < E; e += nthr) s_meta[e] = pp.meta[e];
    if (tid == 0 && pp.use_tma) mbar_init(bar);
    if (warp == 0) tmem_alloc(&s_tmem_base, kTmemColsL);
    tmem_block_sync();
    // this warp's lane quarter and column region
    const uint32_t tbase = s_tmem_base + ((uint32_t)((warp & 3) * 32) << 16) +
                           (uint32_t)((warp >> 2) * pp.ncols);

    const int K = p.K_b * Z;
    const int nbytes = (K + 7) >> 3;
    const int lo = p.punct * Z;
    const int8_t *llr_all = reinterpret_cast<const int8_t *>(p.llr);
    uint32_t parity = 0;
    bool failed = false;
    if (pp.use_tma && tid == 0 && (int)blockIdx.x < p.batch)
        bulk_load(const_cast<int8_t *>(stage), llr_all + in_row(p, blockIdx.x) * p.n_tx,
                  (uint32_t)p.n_tx, bar);

    for (int cw = blockIdx.x; cw < p.batch && !failed; cw += gridDim.x) {
        // a0: zero messages; biased posteriors from the channel LLRs
        {
            uint32_t z[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) z[q] = 0x80808080u;
            int c = 0;
            for (; c + 8 <= pp.ncols; c += 8) tst<8>(tbase + c, z);
            for (; c < pp.ncols; ++c) tst<1>(tbase + c, z);
        }
        const int8_t *src = llr_all + in_row(p, cw) * p.n_tx;
        if (pp.use_tma) {
            const bool ok = mbar_wait(bar, parity);
            if (named_or(1, nthr, !ok)) {
                if (tid == 0) atomicCAS(p.status, 0, kStatusTimeout);
                failed = true;               // parity stays on the copy still in flight
                break;
            }
            parity ^= 1u;
            src = stage;
        }
        // word (c, j) holds rows j and j + H of column block c, biased by 1279
        for (int c = 0; c < n_cols; ++c) {
            for (int j = tid; j < H; j += nthr) {
                const int t0 = c * Z + j - lo, t1 = t0 + H;
                const int q0 = (t0 >= 0 && t0 < p.n_tx) ? (int)src[t0] : 0;
                const int q1 = (t1 >= 0 && t1 < p.n_tx) ? (int)src[t1] : 0;
                Lb[c * H + j] = (uint32_t)(0x64FF + q0) | ((uint32_t)(0x64FF + q1) << 16);
            }
        }
        named_sync(1, nthr);
        // the staging buffer is free: start the copy of the next codeword of this block
        if (pp.use_tma && tid == 0 && cw + (int)gridDim.x < p.batch)
            bulk_load(const_cast<int8_t *>(stage),
                      llr_all + in_row(p, cw + gridDim.x) * p.n_tx, (uint32_t)p.n_tx, bar);

        if (tid == 0) s_stop[0] = s_stop[1] = 0;     // published by the first layer barrier
        int r_scan = 0;                              // first layer of this warp's next scan
        int done = p.max_iter;
#pragma unroll 1
        for (int t = 1; t <= p.max_iter; ++t) {
#ifdef LDPC_LL_ROWS
#define LDPC_LLR(D, P, S0, E0)                                                            \
    ll_row<A, ((D) + A - 1) / A, P>(s_meta, Lb, tbase + (uint32_t)((S0) >> 1), E0, D, H, \
                                    w, k, store);                                         \
    named_sync(1, nthr);
            LDPC_LL_ROWS
#undef LDPC_LLR
#else
#pragma unroll 1
            for (int r = 0; r < n_rows; ++r) {
                const int e0 = pp.row[r];
                ll_dispatch<A>(pp.row[r + 1] - e0, s_meta, Lb, tbase, pp.slot[r], e0, H, w, k,
                               store);
                named_sync(1, nthr);
            }
#endif
            if (p.early_stop) {
                // block-wide exit: the first warp to find a failing check raises
                // s_stop[t & 1] and every warp stops; each starts at its last failing layer
                volatile int *vstop = &s_stop[t & 1];
                int bad = 0, r = r_scan;
                for (int q = 0; q < n_rows && !bad && !*vstop;
                     ++q, r = (r + 1 == n_rows) ? 0 : r + 1) {
                    const int e0 = pp.row[r];
                    bad = __any_sync(0xffffffffu, ll_parity<A>(s_meta, Lb, e0,
                                                                pp.row[r + 1] - e0, H, w, k) != 0u);
                    if (bad) {
                        if ((tid & 31) == 0) *vstop = 1;
                        r_scan = r;
                    }
                }
                const int any = named_or(1, nthr, bad);
                if (tid == 0) s_stop[(t + 1) & 1] = 0;  // read by everyone an iteration ago
                if (any == 0) {
                    done = t;
                    break;
                }
            }
        }

        // a6: outputs
        for (int b = tid; b < nbytes; b += nthr) {
            unsigned x = 0;
            int c = (8 * b) / Z, i = 8 * b - c * Z;            // bit j = c Z + i, stepped
            for (int kk = 0; kk < 8 && 8 * b + kk < K; ++kk) {
                const int lane = i >= H ? 1 : 0;
                const uint32_t wd = Lb[c * H + i - lane * H];
                const uint32_t h = lane ? (wd >> 16) : (wd & 0xffffu);
                if (h < 0x64FFu) x |= 1u << kk;
                if (++i == Z) {
                    i = 0;
                    ++c;
                }
            }
            p.bits[out_row(p, cw) * nbytes + b] = (uint8_t)x;
        }
        if (tid == 0) p.iters[out_row(p, cw)] = done;
        if (p.post) {
            int8_t *po = reinterpret_cast<int8_t *>(p.post) + (size_t)cw * n_cols * Z;
            for (int c = 0; c < n_cols; ++c)
                for (int i = tid; i < Z; i += nthr) {
                    const int lane = i >= H ? 1 : 0;
                    const uint32_t wd = Lb[c * H + i - lane * H];
                    const uint32_t h = lane ? (wd >> 16) : (wd & 0xffffu);
                    po[c * Z + i] = (int8_t)((int)h - 0x64FF);
                }
        }
        if (p.c2v) {
            // each thread reads its own TMEM lane: slot i of row r is edge k + A i
            twait_st();
            int8_t *co = reinterpret_cast<int8_t *>(p.c2v) + (size_t)cw * E * Z;
            for (int r = 0; r < n_rows; ++r) {
                const int e0 = pp.row[r], D = pp.row[r + 1] - e0;
                const int DA = (D + A - 1) / A;
                for (int i = 0; i < DA; ++i) {
                    const int s = pp.slot[r] + i, j = k + A * i;
                    uint32_t v;
                    tld<1>(tbase + (uint32_t)(s >> 1), &v);
                    twait_ld();
                    const uint32_t pr = (s & 1) ? (v >> 16) : (v & 0xffffu);
                    if (store && j < D) {
                        co[(size_t)(e0 + j) * Z + w] = (int8_t)(uint8_t)((pr & 0xffu) ^ 0x80u);
                        co[(size_t)(e0 + j) * Z + w + H] =
                            (int8_t)(uint8_t)(((pr >> 8) & 0xffu) ^ 0x80u);
                    }
                }
            }
        }
        named_sync(1, nthr);
    }
    // a copy that never completed must not outlive the block: wait for it (bounded)
    if (failed && tid == 0) mbar_wait(bar, parity);

    tmem_block_sync();
    if (warp == 0) tmem_dealloc(s_tmem_base, kTmemColsL);
}

// ------------------------------------------------------------ work list, low latency
//
// The same strategy for a heterogeneous work list (items of different graphs, lifting
// sizes and rates in one launch): one persistent block of kThreadsLL threads per SM claims
// items from a counter and decodes each with alpha = 2 threads per row pair.  An item's
// graph tables (gather metadata, row offsets, TMEM slot offsets) are built in shared
// memory when the block takes it, from the graph's device edge table; the warps beyond the
// item's 2 * Z/2 threads only take part in the barriers.  The item's channel LLRs are
// staged in shared memory by 16-byte loads of the aligned part of the row (all in flight
// at once) and byte loads of its ragged ends, then spread into the posterior words.


constexpr int kThreadsLL = 384;          // alpha * Z / 2 for Z <= 384

__device__ __forceinline__ EdgeMetaL meta_l(uint32_t edge, int H) {
    const int c = (int)(edge >> 16), sh = (int)(edge & 0xffffu);
    const int q = sh >= H ? 1 : 0, u = sh - q * H;
    EdgeMetaL m;
    m.base_nw = c * H + u;
    m.thresh = H - u;
    m.sel_nw = q ? 0x1032u : 0x3210u;
    m.sel_w = q ? 0x3210u : 0x1032u;
    return m;
}

// The work-list kernel's body; list_ll_kernel (decode_tmem_ll.cu, and the kernels compiled
// at run time for a set of row sequences) only wraps it.  LDPC_LL_SEQS, when defined, holds
// one `case n:` per compiled row sequence with its rows as LDPC_LLQ(D, P, s0, e0) entries
// (s0: the row's first message slot, P = s0 mod 2), ending in `break;`; an item whose `seq`
// names one of them runs its layers as straight-line code, any other item the generic row
// loop.
__device__ __forceinline__ void list_ll_body(const ListItem *__restrict__ items, int n_items,
                                             int *counter, int early_stop) {
    constexpr int A = 2;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ uint32_t s_tmem_base;
    __shared__ int s_idx, s_stop[2];
    __shared__ int s_row[kMaxRowsL + 1], s_slot[kMaxRowsL + 1];
    const int tid = threadIdx.x, warp = tid >> 5, nthr = blockDim.x;
    const int k = tid % A;
    EdgeMetaL *s_meta = reinterpret_cast<EdgeMetaL *>(smem);

    if (warp == 0) tmem_alloc(&s_tmem_base, kTmemColsL);
    tmem_block_sync();
#pragma unroll 1
    for (;;) {
        if (tid == 0) s_idx = atomicAdd(counter, 1);
        __syncthreads();
        const int idx = s_idx;
        if (idx >= n_items) break;
        const ListItem it = items[idx];
        const int Z = it.Z, H = Z / 2, E = it.E, n_rows = it.n_rows, n_cols = it.n_cols;
        const int off_lb = (int)(((size_t)E * sizeof(EdgeMetaL) + 15) & ~(size_t)15);
        const int off_stage = (off_lb + n_cols * H * 4 + 15) & ~15;
        uint32_t *Lb = reinterpret_cast<uint32_t *>(smem + off_lb);
        // LLR byte t of the item sits at S[t]: the 16-byte words of the row that lie wholly
        // inside it land on 16-byte boundaries of the staging area
        const int n_tx = it.n_tx;
        const int hd = (int)((16u - ((uint32_t)reinterpret_cast<uintptr_t>(it.llr) & 15u)) & 15u);
        const int n16 = n_tx > hd ? (n_tx - hd) >> 4 : 0;      // whole 16-byte words
        int8_t *S = reinterpret_cast<int8_t *>(smem + off_stage) + 16 - hd;
        {
            const int4 *src4 = reinterpret_cast<const int4 *>(it.llr + hd);
            int4 *dst4 = reinterpret_cast<int4 *>(S + hd);
            for (int i0 = tid; i0 < n16; i0 += 4 * nthr) {   // four loads in flight
                int4 v[4];
#pragma unroll
                for (int u = 0; u < 4; ++u)
                    if (i0 + u * nthr < n16) v[u] = __ldg(src4 + i0 + u * nthr);
#pragma unroll
                for (int u = 0; u < 4; ++u)
                    if (i0 + u * nthr < n16) dst4[i0 + u * nthr] = v[u];
            }
        }
        for (int t = tid; t < hd && t < n_tx; t += nthr) S[t] = it.llr[t];
        for (int t = hd + 16 * n16 + tid; t < n_tx; t += nthr) S[t] = it.llr[t];
        for (int e = tid; e < E; e += nthr) s_meta[e] = meta_l(it.edges[e], H);
        for (int r = tid; r <= n_rows; r += nthr) s_row[r] = it.row_ptr[r];
        __syncthreads();
        // a0: biased posteriors from the channel LLRs (word (c, j): rows j and j + H); the
        // block splits into nthr / H groups of H threads, group g taking columns g, g + G, ..
        {
            const int lo = it.punct * Z, G = nthr / H, g = tid / H, j = tid - g * H;
            if (g < G)
                for (int c = g; c < n_cols; c += G) {
                    const int t0 = c * Z + j - lo, t1 = t0 + H;
                    const int q0 = (t0 >= 0 && t0 < n_tx) ? (int)S[t0] : 0;
                    const int q1 = (t1 >= 0 && t1 < n_tx) ? (int)S[t1] : 0;
                    Lb[c * H + j] = (uint32_t)(0x64FF + q0) | ((uint32_t)(0x64FF + q1) << 16);
                }
        }
        __syncthreads();
        if (tid == 0) {
            int sl = 0;
            for (int r = 0; r < n_rows; ++r) {
                s_slot[r] = sl;
                sl += (s_row[r + 1] - s_row[r] + A - 1) / A;
            }
            s_slot[n_rows] = sl;
            s_stop[0] = s_stop[1] = 0;
        }
        __syncthreads();
        const int ncols = (s_slot[n_rows] + 1) / 2;
        // warps holding at least one real row pair; the rest only meet the barriers
        const bool active = warp * 32 < A * H;
        const bool store = tid / A < H;
        const int w = store ? tid / A : H - 1;          // spare threads shadow the last pair
        const uint32_t tbase = s_tmem_base + ((uint32_t)((warp & 3) * 32) << 16) +
                               (uint32_t)((warp >> 2) * ncols);
        if (active) {                                   // zero messages (bytes c + 128)
            uint32_t z[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) z[q] = 0x80808080u;
            int c = 0;
            for (; c + 8 <= ncols; c += 8) tst<8>(tbase + c, z);
            for (; c < ncols; ++c) tst<1>(tbase + c, z);
        }
        int r_scan = 0;
        int done = it.max_iter;
#pragma unroll 1
        for (int t = 1; t <= it.max_iter; ++t) {
#ifdef LDPC_LL_SEQS
            switch (it.seq) {
#define LDPC_LLQ(D, P, S0, E0)                                                            \
    if (active)                                                                           \
        ll_row<A, ((D) + A - 1) / A, P>(s_meta, Lb, tbase + (uint32_t)((S0) >> 1), E0, D, \
                                        H, w, k, store);                                  \
    named_sync(1, nthr);
                LDPC_LL_SEQS
#undef LDPC_LLQ
            default:
#endif
#pragma unroll 1
            for (int r = 0; r < n_rows; ++r) {
                const int e0 = s_row[r];
                if (active)
                    ll_dispatch<A>(s_row[r + 1] - e0, s_meta, Lb, tbase, s_slot[r], e0, H, w,
                                   k, store);
                named_sync(1, nthr);
            }
#ifdef LDPC_LL_SEQS
            }
#endif
            if (early_stop) {
                volatile int *vstop = &s_stop[t & 1];
                int bad = 0;
                if (active) {
                    int r = r_scan;
                    for (int q = 0; q < n_rows && !bad && !*vstop;
                         ++q, r = (r + 1 == n_rows) ? 0 : r + 1) {
                        const int e0 = s_row[r];
                        bad = __any_sync(0xffffffffu,
                                         ll_parity<A>(s_meta, Lb, e0, s_row[r + 1] - e0, H, w,
                                                      k) != 0u);
                        if (bad) {
                            if ((tid & 31) == 0) *vstop = 1;
                            r_scan = r;
                        }
                    }
                }
                const int any = named_or(1, nthr, bad);
                if (tid == 0) s_stop[(t + 1) & 1] = 0;
                if (any == 0) {
                    done = t;
                    break;
                }
            }
        }
        // a6: outputs
        const int K = it.K_b * Z, nbytes = (K + 7) >> 3;
        for (int b = tid; b < nbytes; b += nthr) {
            unsigned x = 0;
            int c = (8 * b) / Z, i = 8 * b - c * Z;            // bit j = c Z + i, stepped
            for (int kk = 0; kk < 8 && 8 * b + kk < K; ++kk) {
                const int lane = i >= H ? 1 : 0;
                const uint32_t wd = Lb[c * H + i - lane * H];
                const uint32_t h = lane ? (wd >> 16) : (wd & 0xffffu);
                if (h < 0x64FFu) x |= 1u << kk;
                if (++i == Z) {
                    i = 0;
                    ++c;
                }
            }
            it.bits[b] = (uint8_t)x;
        }
        if (tid == 0) it.iters[0] = done;
        // the next item places its TMEM regions and shared tables differently: every
        // thread's message stores and table reads of this item end here
        if (active) twait_st();
        tmem_block_sync();
    }
    tmem_block_sync();
    if (warp == 0) tmem_dealloc(s_tmem_base, kTmemColsL);
}

}  // namespace
}  // namespace ldpc

#ifdef LDPC_LL_ROWS
// the one-codeword kernel of a runtime-compiled module (LDPC_LL_A cooperating threads)
extern "C" __global__ void __launch_bounds__(LDPC_LL_A * 192, 1)
    tmem_ll_kernel(const __grid_constant__ ldpc::LlParams pp) {
    ldpc::ll_body<LDPC_LL_A>(pp);
}
#endif

#ifdef LDPC_LL_SEQS
// the work-list kernel of a runtime-compiled module
extern "C" __global__ void __launch_bounds__(ldpc::kThreadsLL, 1)
    list_ll_kernel(const ldpc::ListItem *__restrict__ items, int n_items, int *counter,
                   int early_stop) {
    ldpc::list_ll_body(items, n_items, counter, early_stop);
}
#endif
