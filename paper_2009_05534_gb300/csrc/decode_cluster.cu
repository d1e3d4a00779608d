// Layered min-sum, 8-bit offset variant, one codeword split across a cluster of two thread
// blocks on two SMs (the latency mode for a lone codeword).  Paper: Sec. III (layered
// min-sum with correction, stopping rule), Sec. IV (the low-latency strategy, alpha threads
// per row with a parallel reduce); hot-path steps a0..a6.
//
// Each block of the pair owns half of the check-row pairs of every layer (rank 0 the first
// ceil(H/2), rank 1 the rest; H = Z/2) and decodes them with the low-latency kernel's
// arithmetic (decode_tmem_ll.cu: alpha = 2 threads per row pair, a warp-shuffle reduce,
// messages as bytes in Tensor Memory, posteriors as binary16 L + 1279).  Both blocks keep a
// full copy of the posteriors in their own shared memory.  A posterior a block updates is
// stored in its own copy and, with st.async through distributed shared memory, in the
// peer's copy; every remote store signals the peer's receive barrier of that layer
// (mbarrier complete_tx), armed with the number of bytes the peer sends in that layer.
// Before a block starts the next layer it waits for its own barrier: the peer's half of
// the layer has then landed.  The receive barriers alternate by layer parity, so a block
// is at most one layer ahead of its peer and no layer's bytes are counted for another.
// The stopping rule combines both halves the same way (one word per iteration), so both
// blocks stop at the same iteration; at each codeword boundary each block tells its peer
// that its copy is initialised before any store of the new codeword may reach it.
//
// Every wait is bounded.  A block whose wait runs out records LDPC_ERR_TIMEOUT, stops
// waiting and keeps sending (and asks for every iteration), so that both blocks still walk
// the same sequence of steps and neither exits while stores to it may be in flight.
#include "f16x2.h"
#include "ldpc_internal.h"
#include "tmem.h"

namespace ldpc {
namespace {

using namespace h2;
using namespace tm;

struct EdgeMetaC {
    int base_nw;       // c*H + u
    int thresh;        // H - u
    uint32_t sel_nw;   // 0x3210 or 0x1032
    uint32_t sel_w;
};

constexpr int kAC = 2;                  // cooperating threads per row pair
constexpr int kMaxEdgesC = 1024;
constexpr int kMaxRowsC = 64;
constexpr int kTmemColsC = 512;
constexpr uint32_t kWaitLimit = 1u << 20;

struct ClusterParams {
    DecodeParams p;
    int H;                       // row pairs per layer
    int Hh[2];                   // row pairs of rank 0 ([0, Hh[0])) and rank 1 (the rest)
    int ncols;                   // TMEM columns per thread
    int off_lb;                  // shared-memory offset of the posteriors
    int row[kMaxRowsC + 1];      // edge offsets of the rows
    int slot[kMaxRowsC + 1];     // message slots of the rows in every thread's TMEM lane
    int rx_bytes[2][kMaxRowsC];  // bytes rank k receives from its peer in layer r
    EdgeMetaC meta[kMaxEdgesC];
};

// ------------------------------------------------------------- cluster and barrier helpers

__device__ __forceinline__ uint32_t cluster_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
// the address `a` of this block's shared memory, as seen in block `rank` of the cluster
__device__ __forceinline__ uint32_t peer_addr(uint32_t a, uint32_t rank) {
    uint32_t d;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(rank));
    return d;
}
// 4-byte store into the peer's shared memory that signals the peer's barrier `rbar`
__device__ __forceinline__ void st_remote(uint32_t raddr, uint32_t v, uint32_t rbar) {
    asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.b32 [%0], %1, [%2];" ::"r"(
                     raddr),
                 "r"(v), "r"(rbar)
                 : "memory");
}
__device__ __forceinline__ void cluster_sync() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\t"
                 "barrier.cluster.wait.acquire.aligned;" ::
                     : "memory");
}
// expect `bytes` more and arrive (the barrier's one arrival per phase)
__device__ __forceinline__ void arm(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
                 "r"(bytes)
                 : "memory");
}
// bounded wait for phase `parity`, acquiring at cluster scope (data stored by the peer)
__device__ __forceinline__ bool wait_cluster(uint64_t *bar, uint32_t parity) {
    for (uint32_t n = 0; n < kWaitLimit; ++n) {
        uint32_t ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n"
            " selp.u32 %0, 1, 0, p;\n}"
            : "=r"(ok)
            : "r"(smem_addr(bar)), "r"(parity)
            : "memory");
        if (ok) return true;
    }
    return false;
}

// --------------------------------------------------------------------------- one layer

// Cooperating thread k of row pair w (A = 2 threads per pair, DA = ceil(D / 2) edge slots),
// as in the low-latency kernel, with every posterior it writes also sent to the peer's
// copy (at the same offset) against the peer's barrier `rbar`.
template <int DA, int P>
__device__ __forceinline__ void cl_row(const EdgeMetaC *meta, uint32_t *Lb, uint32_t lb_peer,
                                       uint32_t rbar, uint32_t tcolumn, int e0, int D, int H,
                                       int w, int k, bool store) {
    constexpr int A = kAC;
    constexpr int NC = (P + DA + 1) / 2;
    uint32_t cm[NC];
    twait_st();
    tload<NC>(tcolumn, cm);
    const bool last_real = k + A * (DA - 1) < D;
    uint32_t X[DA];
    int addr[DA];
    uint32_t sel[DA];
#pragma unroll
    for (int i = 0; i < DA; ++i) {
        const int j = (i == DA - 1 && !last_real) ? D - 1 : k + A * i;
        const EdgeMetaC mt = meta[e0 + j];
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
        const uint32_t y = h2relu_fma(M, kNegOne2, X[i]);
        const uint32_t z = h2relu_fma(y, kNegOne2, k254);
        uint32_t x = h2sub(kP127, z);
        if (i == DA - 1 && !last_real) x = kP127;
        m2 = h2min(m2, h2max(h2abs(m1), h2abs(x)));
        m1 = h2minxs(m1, x);
        X[i] = x;
    }
    {
        const uint32_t o1 = __shfl_xor_sync(0xffffffffu, m1, 1);
        const uint32_t o2 = __shfl_xor_sync(0xffffffffu, m2, 1);
        m2 = h2min(h2min(m2, o2), h2max(h2abs(m1), h2abs(o1)));
        m1 = h2minxs(m1, o1);
    }
    const uint32_t SO = (m1 & kSign2) | kOne2;
    const uint32_t a1 = m1 & kAbs2, a2 = m2 & kAbs2;
    const uint32_t m1c = h2relu_fma(a1, kOne2, kNegOne2);
    const uint32_t T1 = h2add(h2add(a1, a2), kNegOne2);
    uint32_t C[DA];
#pragma unroll
    for (int i = 0; i < DA; ++i) {
        const uint32_t x = X[i];
        const uint32_t ex = h2max(m1c, h2sub(T1, h2abs(x)));
        const uint32_t sg = (x & kSign2) ^ SO;
        C[i] = h2fma(ex, sg, kBias2);
        uint32_t L = h2add(C[i], h2add(x, kP127));
        L = h2max(h2min(L, kPostHi), kPostLo);
        if (store && (i < DA - 1 || last_real)) {
            const uint32_t v = prmt(L, 0u, sel[i]);
            Lb[addr[i]] = v;
            st_remote(lb_peer + 4u * (uint32_t)addr[i], v, rbar);
        }
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

template <int DA>
__device__ __forceinline__ void cl_row_any(const EdgeMetaC *meta, uint32_t *Lb, uint32_t lb_peer,
                                           uint32_t rbar, uint32_t tbase, int s0, int e0, int D,
                                           int H, int w, int k, bool store) {
    if (s0 & 1)
        cl_row<DA, 1>(meta, Lb, lb_peer, rbar, tbase + (uint32_t)(s0 >> 1), e0, D, H, w, k, store);
    else
        cl_row<DA, 0>(meta, Lb, lb_peer, rbar, tbase + (uint32_t)(s0 >> 1), e0, D, H, w, k, store);
}

__device__ __forceinline__ void cl_dispatch(int D, const EdgeMetaC *meta, uint32_t *Lb,
                                            uint32_t lb_peer, uint32_t rbar, uint32_t tbase,
                                            int s0, int e0, int H, int w, int k, bool store) {
    switch ((D + kAC - 1) / kAC) {
#define LDPC_CL_CASE(N)                                                                    \
    case N:                                                                                \
        cl_row_any<N>(meta, Lb, lb_peer, rbar, tbase, s0, e0, D, H, w, k, store);          \
        break;
        LDPC_CL_CASE(1) LDPC_CL_CASE(2) LDPC_CL_CASE(3) LDPC_CL_CASE(4) LDPC_CL_CASE(5)
        LDPC_CL_CASE(6) LDPC_CL_CASE(7) LDPC_CL_CASE(8) LDPC_CL_CASE(9) LDPC_CL_CASE(10)
#undef LDPC_CL_CASE
    default:
        break;
    }
}

// parity of the hard decisions of row pair w over a row, combined over the pair's threads
__device__ __forceinline__ uint32_t cl_parity(const EdgeMetaC *meta, const uint32_t *Lb, int e0,
                                              int D, int H, int w, int k) {
    uint32_t par = 0;
    for (int j = k; j < D; j += kAC) {
        const EdgeMetaC mt = meta[e0 + j];
        const bool wr = w >= mt.thresh;
        const int a = w + mt.base_nw - (wr ? H : 0);
        par ^= h2lt_mask(prmt(Lb[a], 0u, wr ? mt.sel_w : mt.sel_nw), kPostBias);
    }
    par ^= __shfl_xor_sync(0xffffffffu, par, 1);
    return par;
}

// ---------------------------------------------------------------------------- the kernel

__global__ void __launch_bounds__(kAC * 96, 1)
    cluster_kernel(const __grid_constant__ ClusterParams pp) {
    const DecodeParams &p = pp.p;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ uint32_t s_tmem_base;
    __shared__ __align__(8) uint64_t s_rx[2];   // the peer's posterior stores, by layer parity
    __shared__ __align__(8) uint64_t s_sx[2];   // the peer's stopping-rule word, by iteration parity
    __shared__ __align__(8) uint64_t s_go[2];   // the peer's copy is initialised, by codeword parity
    __shared__ uint32_t s_word[4];              // stored by the peer: stop words [0..1], go [2..3]
    const uint32_t rank = cluster_rank(), peer = rank ^ 1u;
    const int Z = p.Z, H = pp.H, E = p.E, n_rows = p.n_rows, n_cols = p.n_cols;
    const int tid = threadIdx.x, warp = tid >> 5, nthr = blockDim.x;
    const int Hh = pp.Hh[rank], w0 = rank ? pp.Hh[0] : 0;
    const int k = tid % kAC;
    const bool store = tid / kAC < Hh;
    const int w = w0 + (store ? tid / kAC : Hh - 1);   // spare threads shadow the last pair
    EdgeMetaC *s_meta = reinterpret_cast<EdgeMetaC *>(smem);
    uint32_t *Lb = reinterpret_cast<uint32_t *>(smem + pp.off_lb);
    const uint32_t lb_peer = peer_addr(smem_addr(Lb), peer);

    for (int e = tid; e < E; e += nthr) s_meta[e] = pp.meta[e];
    if (tid == 0) {
#pragma unroll
        for (int b = 0; b < 2; ++b) {
            mbar_init(&s_rx[b]);
            mbar_init(&s_sx[b]);
            mbar_init(&s_go[b]);
        }
        // the first two layers, iterations and codewords
        arm(&s_rx[0], (uint32_t)pp.rx_bytes[rank][0]);
        arm(&s_rx[1], (uint32_t)pp.rx_bytes[rank][1 % n_rows]);
        arm(&s_sx[0], 4u);
        arm(&s_sx[1], 4u);
        arm(&s_go[0], 4u);
        arm(&s_go[1], 4u);
    }
    if (warp == 0) tmem_alloc(&s_tmem_base, kTmemColsC);
    tmem_block_sync();
    cluster_sync();        // both blocks' barriers are initialised and armed before any store
    const uint32_t tbase = s_tmem_base + ((uint32_t)((warp & 3) * 32) << 16) +
                           (uint32_t)((warp >> 2) * pp.ncols);

    const int K = p.K_b * Z;
    const int nbytes = (K + 7) >> 3;
    const int lo = p.punct * Z;
    const int8_t *llr_all = reinterpret_cast<const int8_t *>(p.llr);
    const int n_cl = (int)gridDim.x / 2, cl = (int)blockIdx.x / 2;
    uint32_t rx_par = 0u, sx_par = 0u, go_par = 0u;   // bit b: the phase to wait on barrier b
    int L = 0, it = 0, ncw = 0;                        // layers, iterations, codewords run
    bool failed = false;

    for (int cw = cl; cw < p.batch; cw += n_cl, ++ncw) {
        // a0: zero this block's messages; its copy of the posteriors from the channel LLRs
        {
            uint32_t z[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) z[q] = 0x80808080u;
            int c = 0;
            for (; c + 8 <= pp.ncols; c += 8) tst<8>(tbase + c, z);
            for (; c < pp.ncols; ++c) tst<1>(tbase + c, z);
        }
        const int8_t *src = llr_all + in_row(p, cw) * p.n_tx;
        for (int c = 0; c < n_cols; ++c)
            for (int j = tid; j < H; j += nthr) {
                const int t0 = c * Z + j - lo, t1 = t0 + H;
                const int q0 = (t0 >= 0 && t0 < p.n_tx) ? (int)src[t0] : 0;
                const int q1 = (t1 >= 0 && t1 < p.n_tx) ? (int)src[t1] : 0;
                Lb[c * H + j] = (uint32_t)(0x64FF + q0) | ((uint32_t)(0x64FF + q1) << 16);
            }
        named_sync(1, nthr);
        // tell the peer that this copy is ready for its stores; wait for the same from it
        {
            const int gb = ncw & 1;
            if (tid == 0)
                st_remote(peer_addr(smem_addr(&s_word[2 + gb]), peer), 1u,
                          peer_addr(smem_addr(&s_go[gb]), peer));
            if (!failed && !wait_cluster(&s_go[gb], (go_par >> gb) & 1u)) failed = true;
            go_par ^= 1u << gb;
            if (tid == 0 && !failed) arm(&s_go[gb], 4u);      // codeword ncw + 2
            named_sync(1, nthr);
        }

        int done = p.max_iter;
#pragma unroll 1
        for (int t = 1; t <= p.max_iter; ++t) {
#pragma unroll 1
            for (int r = 0; r < n_rows; ++r, ++L) {
                const int rb = L & 1;
                const int e0 = pp.row[r];
                cl_dispatch(pp.row[r + 1] - e0, s_meta, Lb, lb_peer,
                            peer_addr(smem_addr(&s_rx[rb]), peer), tbase, pp.slot[r], e0, H, w,
                            k, store);
                // the peer's half of this layer has landed in this copy
                if (!failed && !wait_cluster(&s_rx[rb], (rx_par >> rb) & 1u)) failed = true;
                rx_par ^= 1u << rb;
                if (tid == 0 && !failed)
                    arm(&s_rx[rb], (uint32_t)pp.rx_bytes[rank][(r + 2) % n_rows]);   // layer L + 2
                named_sync(1, nthr);
            }
            if (p.early_stop) {
                // a5 over this block's rows, then the two halves combined through the peer
                int bad = 0;
                for (int r = 0; r < n_rows && !bad; ++r) {
                    const int e0 = pp.row[r];
                    bad = __any_sync(0xffffffffu,
                                     cl_parity(s_meta, Lb, e0, pp.row[r + 1] - e0, H, w, k) != 0u);
                }
                bad = named_or(1, nthr, bad || failed);
                const int sb = it & 1;
                if (tid == 0)
                    st_remote(peer_addr(smem_addr(&s_word[sb]), peer), (uint32_t)bad,
                              peer_addr(smem_addr(&s_sx[sb]), peer));
                if (!failed && !wait_cluster(&s_sx[sb], (sx_par >> sb) & 1u)) failed = true;
                sx_par ^= 1u << sb;
                const uint32_t pbad = s_word[sb];
                if (tid == 0 && !failed) arm(&s_sx[sb], 4u);   // iteration it + 2
                ++it;
                if (named_or(1, nthr, bad || pbad != 0u || failed) == 0) {
                    done = t;
                    break;
                }
            }
        }

        // a6: outputs; rank 0 writes the hard bits, the iteration count and the posteriors,
        // each block its own rows' messages
        if (rank == 0) {
            for (int b = tid; b < nbytes; b += nthr) {
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
        }
        if (p.c2v) {
            twait_st();
            int8_t *co = reinterpret_cast<int8_t *>(p.c2v) + (size_t)cw * E * Z;
            for (int r = 0; r < n_rows; ++r) {
                const int e0 = pp.row[r], D = pp.row[r + 1] - e0;
                const int DA = (D + kAC - 1) / kAC;
                for (int i = 0; i < DA; ++i) {
                    const int s = pp.slot[r] + i, j = k + kAC * i;
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
    if (failed) atomicCAS(p.status, 0, (int)LDPC_ERR_TIMEOUT);

    tmem_block_sync();
    if (warp == 0) tmem_dealloc(s_tmem_base, kTmemColsC);
    cluster_sync();        // neither block exits while the other may still store into it
}

int cl_slots(const int *row_ptr, int n_rows, int *slot) {
    int s = 0;
    for (int r = 0; r < n_rows; ++r) {
        if (slot) slot[r] = s;
        s += (row_ptr[r + 1] - row_ptr[r] + kAC - 1) / kAC;
    }
    if (slot) slot[n_rows] = s;
    return s;
}

size_t cl_smem_bytes(const DecodeParams &p) {
    const size_t off = ((size_t)p.E * sizeof(EdgeMetaC) + 15) & ~(size_t)15;
    return off + (size_t)p.n_cols * (p.Z / 2) * 4;
}

}  // namespace

bool cluster_supported(const DecodeParams &p, int llr_type, int max_deg, size_t smem_optin) {
    if (llr_type != LDPC_LLR_INT8 || p.algo != LDPC_OFFSET || p.offset_q != 1) return false;
    if ((p.Z & 3) || p.Z < 4 || p.Z > 384 || max_deg > kMaxDeg || max_deg < 2) return false;
    if (p.E > kMaxEdgesC || p.n_rows > kMaxRowsC) return false;
    const int H = p.Z / 2, hh = (H + 1) / 2;
    const int nwarps = (kAC * hh + 31) / 32;
    const int depth = (nwarps + 3) / 4;
    if (depth * ((cl_slots(p.h_row_ptr, p.n_rows, nullptr) + 1) / 2) > kTmemColsC) return false;
    return cl_smem_bytes(p) + 64 <= smem_optin;
}

ldpc_status launch_cluster(const DecodeParams &p, cudaStream_t stream) {
    static thread_local ClusterParams pp;   // ~18 kB: kept off the stack
    pp.p = p;
    const int H = p.Z / 2;
    pp.H = H;
    pp.Hh[0] = (H + 1) / 2;
    pp.Hh[1] = H - pp.Hh[0];
    for (int r = 0; r <= p.n_rows; ++r) pp.row[r] = p.h_row_ptr[r];
    pp.ncols = (cl_slots(p.h_row_ptr, p.n_rows, pp.slot) + 1) / 2;
    for (int r = 0; r < p.n_rows; ++r) {
        const int d = p.h_row_ptr[r + 1] - p.h_row_ptr[r];
        pp.rx_bytes[0][r] = 4 * d * pp.Hh[1];       // rank 0 receives rank 1's stores
        pp.rx_bytes[1][r] = 4 * d * pp.Hh[0];
    }
    for (int e = 0; e < p.E; ++e) {
        const uint32_t ed = p.h_edges[e];
        const int c = (int)(ed >> 16), sh = (int)(ed & 0xffffu);
        const int q = sh >= H ? 1 : 0, u = sh - q * H;
        pp.meta[e].base_nw = c * H + u;
        pp.meta[e].thresh = H - u;
        pp.meta[e].sel_nw = q ? 0x1032u : 0x3210u;
        pp.meta[e].sel_w = q ? 0x3210u : 0x1032u;
    }
    pp.off_lb = (int)(((size_t)p.E * sizeof(EdgeMetaC) + 15) & ~(size_t)15);
    // at least 120 kB of shared memory so that one block occupies an SM (its TMEM
    // allocation takes all 512 columns; two blocks of a cluster on one SM would wait)
    size_t smem = cl_smem_bytes(p);
    if (smem < 120 * 1024) smem = 120 * 1024;
    int dev = 0, n_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return LDPC_ERR_CUDA;
    cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    if (set_dyn_smem(reinterpret_cast<const void *>(cluster_kernel), smem) != cudaSuccess)
        return LDPC_ERR_CUDA;
    int n_cl = n_sm / 2;
    if (n_cl > p.batch) n_cl = p.batch;
    if (n_cl < 1) n_cl = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(2 * n_cl, 1, 1);
    cfg.blockDim = dim3(((kAC * pp.Hh[0] + 31) / 32) * 32, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (cudaLaunchKernelEx(&cfg, cluster_kernel, pp) != cudaSuccess) return LDPC_ERR_CUDA;
    count_launch();
    if (cudaGetLastError() != cudaSuccess) return LDPC_ERR_CUDA;
    return LDPC_OK;
}

}  // namespace ldpc
