// Layered min-sum, 8-bit offset variant, with the two binary16 lanes of every register
// carrying the same check row of two different codewords (sm_103a).  Paper: Sec. III
// (layered min-sum with correction, stopping rule), Sec. IV (per-row m1 / m2 / sign,
// several codewords decoded in parallel); hot-path steps a0..a6.
//
// Compared with a row-pair mapping (decode_rowpair.cu, decode_tmem_ll.cu), whose lanes
// hold rows j and j + Z/2 of one codeword and must exchange the halves whenever a shift
// wraps one row of the pair but not the other, this mapping needs no half exchange: row i
// of a circulant with shift s reads word c*Z + (i + s) mod Z for both codewords at once, so
// neither the gather nor the write-back permutes the halves (measured: 9 % less time per
// iteration than the row-pair TMEM kernel it replaced).  Thread i owns check row i of every
// layer (Z threads); two codewords per block, one block per SM.
//
// Why TMEM.  A BG1-shaped codeword at Z = 384 needs 52 kB of posteriors (read by every
// check row through the circulant gather) and 124 kB of messages that only their own check
// row ever reads.  The messages are private per row, so they live in Tensor Memory:
// tcgen05.ld / tcgen05.st of shape 32x32b give every thread its own TMEM lane with
// warp-uniform column indices, and the 256 kB of TMEM hold the messages of the block's
// two codewords while shared memory holds their posteriors.
//
// The two codewords of a block advance in lockstep through the layers, but each lane keeps
// its own codeword and iteration count: after every full iteration each lane applies the
// stopping rule (or the iteration cap) on its own, writes its outputs when it stops, and is
// refilled at once with the block's next codeword (its LLRs staged ahead by a 1-D bulk copy,
// or, near the end of the batch, claimed and copied then), which starts its first
// iteration at layer 0 while the other lane carries on.  A lane with no codeword left runs
// along without writing anything.
//
// Arithmetic (exact on these integers, so bit-identical to 8-bit fixed point): posteriors
// as binary16 L + 1279 in shared memory (on [1152, 1406] binary16 has spacing 1; word
// (c, i) holds the two codewords' values), messages as bytes c + 128 in Tensor Memory
// (edge e at column e/2, byte 2(e%2) + lane), turned into binary16 c + 1152 by one PRMT
// under the exponent byte 0x64, so v + 127 = (L + 1279) - (c + 1152) is one subtraction;
// x + 127 = sat(v) + 127 by a relu FMA and a min, sat(v) by one subtraction;
// min.xorsign.abs for m1 and the sign product, plain min / max for m2, both as a tree over
// the row's edges; new magnitude max(m1', (m1 + m2 - 1) - |v|), which is m2' on the argmin
// edge and m1' elsewhere, so no argmin index is kept; the new posterior
// (x + c') + 1279 = (c' + 1152) + (x + 127), clamped to [1152, 1406].
#pragma once

#include "f16x2.h"
#include "ldpc_params.h"
#include "tmem.h"

namespace ldpc {
namespace {

using namespace h2;
using namespace tm;

// Per edge: the circulant's shift and the column's place in the posterior array, both in
// bytes (copied to shared memory; every thread of a row step reads the same entry).
struct __align__(8) EdgeMetaQ {
    int s4;        // 4 * s
    int col4;      // 4 * c * Z
};

constexpr int kMaxEdgesQ = 1024;
constexpr int kMaxRowsQ = 64;
constexpr int kTmemColsQ = 512;
constexpr int kThreadsQ = 384;
constexpr uint32_t kPostZero = 0x64FFu;   // binary16 1279: posterior L = 0

struct PairParams {
    DecodeParams p;
    int ncols;                   // TMEM columns per thread: ceil(E / 2)
    int use_tma;                 // channel LLRs staged by 1-D bulk copies
    int stage_bytes;             // per-lane staging buffer (multiple of 16)
    int off_meta, off_stage;     // shared-memory offsets of the edge table and the staging
    int row[kMaxRowsQ + 1];      // edge offsets of the rows
    EdgeMetaQ meta[kMaxEdgesQ];
};

// --------------------------------------------------------------------------- one layer

// Thread i processes check row i (both lanes) of a layer of degree D whose first edge sits
// in the upper half of its TMEM column when P = 1.  Posterior word (c, j) sits at byte
// 4 (c Z + j) of shared memory.  The row waits at the layer barrier (nthr threads) after
// loading its own messages and computing its addresses.
template <int D, int P>
__device__ __forceinline__ void pq_row(const EdgeMetaQ *meta, unsigned char *Lbytes,
                                       uint32_t tcolumn, int e0, uint32_t i4, uint32_t i4z,
                                       bool store, int nthr, uint32_t &carry) {
    constexpr int NC = (P + D + 1) / 2;
    uint32_t cm[NC];
    // a row that starts mid-column takes that column from the previous row's registers
    // (its upper half, this row's first message, passed through the previous row intact)
    if constexpr (P == 1) {
        cm[0] = carry;
        tload<NC - 1>(tcolumn + 1, cm + 1);
    } else {
        tload<NC>(tcolumn, cm);
    }
    uint32_t X[D], XB[D];
    uint32_t off[D];
#pragma unroll
    for (int j = 0; j < D; ++j) {
        const EdgeMetaQ mt = meta[e0 + j];
        // (i + s) mod Z without a compare: i + s - Z is negative (a huge unsigned value)
        // unless the circulant wraps row i
        off[j] = min(i4 + (uint32_t)mt.s4, i4z + (uint32_t)mt.s4) + (uint32_t)mt.col4;
    }
    named_sync(1, nthr);
#pragma unroll
    for (int j = 0; j < D; ++j) X[j] = *reinterpret_cast<const uint32_t *>(Lbytes + off[j]);
    twait_ld();
    uint32_t M[D];
#pragma unroll
    for (int j = 0; j < D; ++j)
        M[j] = prmt(cm[(P + j) >> 1], 0x64646464u, ((P + j) & 1) ? 0x4342u : 0x4140u);
#pragma unroll
    for (int j = 0; j < D; ++j) {
        // (L + 1279) - (c + 1152) = v + 127: its lower clamp in the relu FMA, the upper one
        // by a min (x + 127 = min(max(v + 127, 0), 254)), then x = sat(v)
        XB[j] = h2min(h2relu_fma(M[j], kNegOne2, X[j]), k254);
        X[j] = h2sub(XB[j], kP127);
    }
    uint32_t m1, m2;
    min_tree<0, D>(X, m1, m2);
    const uint32_t SO = (m1 & kSign2) | kOne2;
    const uint32_t a1 = m1 & kAbs2;
    const uint32_t m1c = h2relu_fma(a1, kOne2, kNegOne2);
    const uint32_t T1 = h2add(h2add(a1, m2), kNegOne2);       // m2 is never negative
    uint32_t C[D];
#pragma unroll
    for (int j = 0; j < D; ++j) {
        const uint32_t x = X[j];
        const uint32_t ex = h2max(m1c, h2sub(T1, h2abs(x)));
        const uint32_t sg = (x & kSign2) ^ SO;
        C[j] = h2fma(ex, sg, kBias2);                          // c' + 1152
        uint32_t L = h2add(C[j], XB[j]);                       // (x + c') + 1279
        L = h2max(h2min(L, kPostHi), kPostLo);
        if (store) *reinterpret_cast<uint32_t *>(Lbytes + off[j]) = L;
    }
#pragma unroll
    for (int k = 0; k < NC; ++k) {
        const int jl = 2 * k - P, jh = 2 * k + 1 - P;
        const int il = jl < 0 ? 0 : jl, ih = jh >= D ? D - 1 : jh;
        if (jl >= 0 && jh < D)
            cm[k] = prmt(C[il], C[ih], 0x6420u);
        else if (jl >= 0)
            cm[k] = prmt(C[il], cm[k], 0x7620u);
        else
            cm[k] = prmt(cm[k], C[ih], 0x6410u);
    }
    // a column shared with the next row is stored by that row (its lower half travels in
    // carry), so every column is stored once per iteration
    if constexpr (((P + D) & 1) == 1) {
        tstore<NC - 1>(tcolumn, cm);
        carry = cm[NC - 1];
    } else {
        tstore<NC>(tcolumn, cm);
    }
}

#ifndef LDPC_PAIR_ROWS
// One dispatch per row on key = 2 D + P (the row's degree and the parity of its first
// edge), computed a row ahead; the branch happens before the row's layer barrier.
__device__ __forceinline__ void pq_dispatch(int key, const EdgeMetaQ *meta, unsigned char *Lbytes,
                                            uint32_t tbase, int e0, uint32_t i4, uint32_t i4z,
                                            bool store, int nthr, uint32_t &carry) {
    const uint32_t tc = tbase + (uint32_t)(e0 >> 1);
    switch (key) {
#define LDPC_PQ_CASE(D)                                                   \
    case 2 * D:                                                           \
        pq_row<D, 0>(meta, Lbytes, tc, e0, i4, i4z, store, nthr, carry);  \
        break;                                                            \
    case 2 * D + 1:                                                       \
        pq_row<D, 1>(meta, Lbytes, tc, e0, i4, i4z, store, nthr, carry);  \
        break;
        LDPC_PQ_CASE(2) LDPC_PQ_CASE(3) LDPC_PQ_CASE(4) LDPC_PQ_CASE(5) LDPC_PQ_CASE(6)
        LDPC_PQ_CASE(7) LDPC_PQ_CASE(8) LDPC_PQ_CASE(9) LDPC_PQ_CASE(10) LDPC_PQ_CASE(11)
        LDPC_PQ_CASE(12) LDPC_PQ_CASE(13) LDPC_PQ_CASE(14) LDPC_PQ_CASE(15) LDPC_PQ_CASE(16)
        LDPC_PQ_CASE(17) LDPC_PQ_CASE(18) LDPC_PQ_CASE(19) LDPC_PQ_CASE(20)
#undef LDPC_PQ_CASE
    default:
        __builtin_unreachable();
    }
}
#endif

// parity masks of check row i over a row's edges: 0xFFFF in a lane whose codeword has an
// odd number of negative posteriors on the row
__device__ __forceinline__ uint32_t pq_parity(const EdgeMetaQ *meta, const unsigned char *Lbytes,
                                              int e0, int d, uint32_t i4, uint32_t i4z) {
    uint32_t par = 0;
    for (int j = 0; j < d; ++j) {
        const EdgeMetaQ mt = meta[e0 + j];
        const uint32_t off =
            min(i4 + (uint32_t)mt.s4, i4z + (uint32_t)mt.s4) + (uint32_t)mt.col4;
        par ^= h2lt_mask(*reinterpret_cast<const uint32_t *>(Lbytes + off), kPostBias);
    }
    return par;
}

// ---------------------------------------------------------------------------- the kernel

// The whole kernel body; pair_kernel (below, and the per-graph kernels compiled at run
// time) only wraps it.  LDPC_PAIR_ROWS, when defined, is the graph's row sequence as
// LDPC_PQ(D, P, e0) entries: the layer loop is then straight-line code without the per-row
// dispatch (measured 19 % less time per headline launch).
__device__ __forceinline__ void pair_body(const PairParams &pp) {
    const DecodeParams &p = pp.p;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ uint32_t s_tmem_base;
    __shared__ __align__(8) uint64_t s_bar[2];
    __shared__ uint32_t s_bad[2];
    const int Z = p.Z, E = p.E, n_rows = p.n_rows, n_cols = p.n_cols;
    const int tid = threadIdx.x, warp = tid >> 5, nthr = blockDim.x;
    const bool store = tid < Z;
    const int i = store ? tid : Z - 1;                // spare threads shadow the last row
    const uint32_t i4 = 4u * (uint32_t)i, i4z = 4u * (uint32_t)(i - Z);
    // shared memory: posterior words (from offset 0) | edge table | two LLR staging buffers
    EdgeMetaQ *s_meta = reinterpret_cast<EdgeMetaQ *>(smem + pp.off_meta);
    unsigned char *Lbytes = smem;
    uint32_t *Lb = reinterpret_cast<uint32_t *>(smem);
    uint16_t *Lh = reinterpret_cast<uint16_t *>(smem);   // lane X of word j: Lh[2j + X]
    int8_t *stage = reinterpret_cast<int8_t *>(smem + pp.off_stage);

    for (int e = tid; e < E; e += nthr) s_meta[e] = pp.meta[e];
#ifndef LDPC_PAIR_ROWS
    // per row: first edge and dispatch key 2 D + P (one entry past the last row, unused)
    __shared__ int s_row[kMaxRowsQ + 1], s_key[kMaxRowsQ + 1];
    for (int r = tid; r <= n_rows; r += nthr) {
        s_row[r] = pp.row[r];
        s_key[r] = r < n_rows ? 2 * (pp.row[r + 1] - pp.row[r]) + (pp.row[r] & 1) : 0;
    }
#endif
    if (tid == 0) {
        if (pp.use_tma) {
            mbar_init(&s_bar[0]);
            mbar_init(&s_bar[1]);
        }
        s_bad[0] = s_bad[1] = 0u;
    }
    if (warp == 0) tmem_alloc(&s_tmem_base, kTmemColsQ);
    tmem_block_sync();
    const uint32_t tbase = s_tmem_base + ((uint32_t)((warp & 3) * 32) << 16) +
                           (uint32_t)((warp >> 2) * pp.ncols);

    const int K = p.K_b * Z;
    const int nbytes = (K + 7) >> 3;
    const int lo = p.punct * Z;
    const int NV = n_cols * Z;
    const int8_t *llr_all = reinterpret_cast<const int8_t *>(p.llr);
    // Work distribution: codewords are claimed one at a time from a counter shared by the
    // blocks of the launch (p.queue[0]), so a block whose codewords stop early takes more
    // of them; without a counter block b takes b, b + G, b + 2G, ...  A claim is staged at
    // once in one of the two buffers, and the block holds at most one claimed codeword that
    // no lane has started.  Every thread keeps the same copy of this state.
    __shared__ int s_claim[2];
    int cw[2] = {-1, -1}, t[2] = {0, 0}, buf[2] = {0, 1};
    int staged = -1, sbuf = 0, lastb = 1, n_claims = 0;
    bool drained = false;
    uint32_t parity = 0u;                // bit S: phase parity of staging buffer S
    uint32_t pending = 0u;               // bit S: a copy into buffer S issued, not consumed
    bool failed = false;
    // thread 0 claims the next codeword and starts its copy into buffer S (free: no thread
    // reads it); every thread gets the codeword, or -1 once the batch is exhausted.  A claim
    // to stage ahead (ahead = true) is skipped near the end of the batch: blocks refill at
    // about the same time (always, at a fixed iteration count), and a block that staged one
    // of the last codewords would take it from a block whose lane is still empty (a batch
    // of k full rounds took k + 1 rounds).
    int k_last = 0;                      // thread 0: the index of its last claim
    auto claim = [&](int S, bool ahead) -> int {
        if (drained) return -1;
        const int slot = n_claims & 1;   // two slots: one barrier per claim suffices
        if (tid == 0) {
            int c = -2;                  // -2: not staged (lanes claim on demand)
            // what remains is at most batch - k_last; other blocks may have claimed up to
            // a round of lanes since, hence the margin of twice the lanes
            if (!ahead || !p.queue || p.batch - k_last > 4 * (int)gridDim.x) {
                const int k = p.queue ? atomicAdd(p.queue, 1)
                                      : (int)blockIdx.x + n_claims * (int)gridDim.x;
                k_last = k;
                c = k < p.batch ? k : -1;
            }
            s_claim[slot] = c;
            if (c >= 0 && pp.use_tma)
                bulk_load(stage + S * pp.stage_bytes, llr_all + in_row(p, c) * p.n_tx,
                          (uint32_t)p.n_tx, &s_bar[S]);
        }
        named_sync(1, nthr);
        const int c = s_claim[slot];
        if (c != -2) ++n_claims;
        if (c == -1)
            drained = true;
        else if (c >= 0 && pp.use_tma)
            pending |= 1u << S;
        return c < 0 ? -1 : c;
    };
    // a0 for lane X: its messages to zero (byte 0x80), its posteriors from the channel
    // LLRs; false (for every thread) if the staged copy timed out
    auto init_lane = [&](int X) -> bool {
        const uint32_t keep = X ? 0x00FF00FFu : 0xFF00FF00u;
        const uint32_t set = X ? 0x80008000u : 0x00800080u;
        twait_st();
        int c = 0;
        for (; c + 16 <= pp.ncols; c += 16) {
            uint32_t v[16];
            tld<16>(tbase + c, v);
            twait_ld();
#pragma unroll
            for (int q = 0; q < 16; ++q) v[q] = (v[q] & keep) | set;
            tst<16>(tbase + c, v);
        }
        for (; c < pp.ncols; ++c) {
            uint32_t v;
            tld<1>(tbase + c, &v);
            twait_ld();
            v = (v & keep) | set;
            tst<1>(tbase + c, &v);
        }
        const int8_t *src = llr_all + in_row(p, cw[X]) * p.n_tx;
        if (pp.use_tma) {
            const int S = buf[X];
            const bool ok = mbar_wait(&s_bar[S], (parity >> S) & 1u);
            if (named_or(1, nthr, !ok)) {
                if (tid == 0) atomicCAS(p.status, 0, kStatusTimeout);
                return false;                // parity stays on the copy still in flight
            }
            parity ^= 1u << S;
            pending &= ~(1u << S);
            src = stage + S * pp.stage_bytes;
        }
        // binary16 L + 1279 = 1024 + (L + 255): bit pattern 0x6400 + L + 255
        for (int j = tid; j < NV; j += nthr) {
            const int t0 = j - lo;
            const int q = (t0 >= 0 && t0 < p.n_tx) ? (int)src[t0] : 0;
            Lh[2 * j + X] = (uint16_t)(kPostZero + q);
        }
        return true;
    };
    // a6 for lane X: hard bits, iteration count, and the debug outputs
    auto emit = [&](int X) {
        // byte b packs the hard decisions of posterior words 8b .. 8b + 7 (32 bytes, read as
        // two 16-byte words); words past K exist (parity columns follow) and are masked off
        const int sh = 16 * X;
        for (int b = tid; b < nbytes; b += nthr) {
            const uint4 q0 = reinterpret_cast<const uint4 *>(Lb)[2 * b];
            const uint4 q1 = reinterpret_cast<const uint4 *>(Lb)[2 * b + 1];
            const uint32_t wv[8] = {q0.x, q0.y, q0.z, q0.w, q1.x, q1.y, q1.z, q1.w};
            unsigned x = 0;
#pragma unroll
            for (int kk = 0; kk < 8; ++kk)
                x |= (((wv[kk] >> sh) & 0xffffu) < kPostZero ? 1u : 0u) << kk;
            const int rest = K - 8 * b;
            if (rest < 8) x &= (1u << rest) - 1u;
            p.bits[out_row(p, cw[X]) * nbytes + b] = (uint8_t)x;
        }
        if (tid == 0) p.iters[out_row(p, cw[X])] = t[X];
        if (p.post) {
            int8_t *po = reinterpret_cast<int8_t *>(p.post) + (size_t)cw[X] * NV;
            for (int j = tid; j < NV; j += nthr)
                po[j] = (int8_t)((int)Lh[2 * j + X] - (int)kPostZero);
        }
        if (p.c2v) {
            twait_st();
            int8_t *co = reinterpret_cast<int8_t *>(p.c2v) + (size_t)cw[X] * E * Z;
            for (int e = 0; e < E; ++e) {
                uint32_t v;
                tld<1>(tbase + (uint32_t)(e >> 1), &v);
                twait_ld();
                const uint32_t byte = (v >> (8 * (2 * (e & 1) + X))) & 0xffu;
                if (store) co[(size_t)e * Z + i] = (int8_t)(uint8_t)(byte ^ 0x80u);
            }
        }
    };

    cw[0] = claim(0, false);
    cw[1] = claim(1, false);
#pragma unroll
    for (int X = 0; X < 2 && !failed; ++X)
        if (cw[X] >= 0) failed = !init_lane(X);
    named_sync(1, nthr);                             // buffer 0 free again
    if (!failed) {
        sbuf = 0;
        staged = claim(sbuf, true);
    }

    int ib = 0;                                      // iterations run by the block
    int r_scan = 0;                                  // first layer of this warp's next scan
#pragma unroll 1
    while (!failed && (cw[0] >= 0 || cw[1] >= 0)) {
        uint32_t carry = 0u;                         // set by a row that ends mid-column
        twait_st();                                  // rows starting on a column do not wait
#ifdef LDPC_PAIR_ROWS
#define LDPC_PQ(D, P, E0) \
    pq_row<D, P>(s_meta, Lbytes, tbase + (uint32_t)((E0) >> 1), E0, i4, i4z, store, nthr, carry);
        LDPC_PAIR_ROWS
#undef LDPC_PQ
#else
        int e0 = s_row[0], key = s_key[0];
#pragma unroll 1
        for (int r = 0; r < n_rows; ++r) {
            const int e0r = e0, keyr = key;
            e0 = s_row[r + 1];                       // the next row's, read before the barrier
            key = s_key[r + 1];
            pq_dispatch(keyr, s_meta, Lbytes, tbase, e0r, i4, i4z, store, nthr, carry);
        }
#endif
        // the last row ends mid-column when E is odd: its last column has no next row
        if (E & 1) tstore<1>(tbase + (uint32_t)(E >> 1), &carry);
        named_sync(1, nthr);                         // the iteration's last layer is done
        ++t[0];
        ++t[1];
        // a5: the stopping rule per lane (bits 0..15: lane 0, 16..31: lane 1); a lane with
        // no codeword counts as failing.  The scan ends block-wide: each warp publishes the
        // failing-lane bits it finds, and every warp stops once the block's bits show both
        // lanes failing (neither lane is done, whatever the other rows say); only a lane
        // that satisfies every check needs the whole scan.  Each warp starts at the layer
        // where it last found a failing check (the order does not change the result).
        uint32_t bad = 0xFFFFFFFFu;
        if (p.early_stop) {
            const int sb = ib & 1;
            const uint32_t ghost = (cw[0] < 0 ? 0x0000FFFFu : 0u) | (cw[1] < 0 ? 0xFFFF0000u : 0u);
            volatile uint32_t *vbad = &s_bad[sb];
            uint32_t acc = ghost, seen = ghost;
            int r = r_scan;
            for (int k = 0; k < n_rows; ++k, r = (r + 1 == n_rows) ? 0 : r + 1) {
                const uint32_t wacc = __reduce_or_sync(0xffffffffu, acc);
                if (wacc != seen) {                  // new failing lanes: publish them
                    if ((tid & 31) == 0) atomicOr(&s_bad[sb], wacc);
                    if (seen == ghost) r_scan = r == 0 ? n_rows - 1 : r - 1;
                    seen = wacc;
                }
                if ((wacc | *vbad) == 0xFFFFFFFFu) break;
                const int e0 = pp.row[r];
                acc |= pq_parity(s_meta, Lbytes, e0, pp.row[r + 1] - e0, i4, i4z);
            }
            const uint32_t wacc = __reduce_or_sync(0xffffffffu, acc);
            if ((tid & 31) == 0 && wacc != seen) atomicOr(&s_bad[sb], wacc);
            named_sync(1, nthr);
            bad = s_bad[sb] | ghost;
            if (tid == 0) s_bad[sb ^ 1] = 0u;        // read by everyone one iteration ago
        }
        ++ib;
        bool done[2];
#pragma unroll
        for (int X = 0; X < 2; ++X)
            done[X] = cw[X] >= 0 &&
                      (t[X] >= p.max_iter || ((bad >> (16 * X)) & 0xFFFFu) == 0u);
        if (!done[0] && !done[1]) continue;
#pragma unroll
        for (int X = 0; X < 2; ++X)
            if (done[X]) emit(X);
        named_sync(1, nthr);                         // outputs read before the refill
#pragma unroll
        for (int X = 0; X < 2 && !failed; ++X) {
            if (!done[X]) continue;
            int b;
            if (staged >= 0) {
                cw[X] = staged;
                b = sbuf;
                staged = -1;
            } else {
                b = lastb ^ 1;                       // the other buffer may still be read
                cw[X] = claim(b, false);
            }
            lastb = b;
            buf[X] = b;
            t[X] = 0;
            if (cw[X] >= 0) failed = !init_lane(X);
        }
        named_sync(1, nthr);                         // refilled posteriors visible; staging free
        if (!failed && staged < 0) {
            sbuf = lastb ^ 1;
            staged = claim(sbuf, true);
        }
    }
    // a copy still in flight after a timeout must not outlive the block (bounded waits)
    if (failed && tid == 0)
#pragma unroll
        for (int S = 0; S < 2; ++S)
            if ((pending >> S) & 1u) mbar_wait(&s_bar[S], (parity >> S) & 1u);

    // the last block of the launch to finish resets the shared counter for the next launch
    // on this stream
    if (p.queue && tid == 0) {
        __threadfence();
        if (atomicAdd(p.queue + 1, 1) == (int)gridDim.x - 1) {
            p.queue[0] = 0;
            p.queue[1] = 0;
        }
    }

    tmem_block_sync();
    if (warp == 0) tmem_dealloc(s_tmem_base, kTmemColsQ);
}

}  // namespace
}  // namespace ldpc

#ifdef LDPC_PAIR_ROWS
// the per-graph kernel of a runtime-compiled module
extern "C" __global__ void __launch_bounds__(ldpc::kThreadsQ, 1)
    pair_kernel(const __grid_constant__ ldpc::PairParams pp) {
    ldpc::pair_body(pp);
}
#endif
