// Row-pair fp16x2 layered min-sum kernel for 8-bit offset min-sum (sm_103a).
//
// Same method as the generic kernel (paper Sec. III layered min-sum with correction,
// Sec. IV per-row m1 / m2 / sign quantities, a1..a6 of the hot path), mapped for
// throughput on GB300:
//
// * Lanes.  Check rows i and i + H (H = Z/2) of a layer travel together in one 32-bit
//   register as two binary16 lanes.  The 8-bit LLRs are integers in [-127, 127]; every
//   intermediate value is an integer of magnitude below 2048, so binary16 holds it
//   exactly and the results are bit-identical to 8-bit fixed-point arithmetic.
// * Posteriors in shared memory are stored biased by 1152: a word holds
//   (L[cZ+j] + 1152, L[cZ+j+H] + 1152) for j < H.  Biased values lie in [1025, 1279],
//   where binary16 has spacing 1, and the bit pattern of 1024 + b is 0x6400 | b.
// * Check-to-variable messages are kept expanded, one byte per (edge, row), as c + 128.
//   One PRMT that inserts the byte under the exponent 0x64 turns it into binary16
//   c + 1152, so v = (L + 1152) - (c + 1152) needs no further conversion, and the new
//   message c' + 1152 = fma(|m'|, +-1, 1152) is stored back by taking its low byte.
// * Circulant gather: row j (< H) of a circulant with shift s = qH + u reads word
//   (j + u) mod H with its halves exchanged when q xor [j + u >= H]; the same
//   permutation writes the result back.
// * Check node: min.xorsign.abs.f16x2 gives min(|m1|, |v|) with the sign product in one
//   instruction; m2 follows from max.xorsign / min.xorsign.  The new message magnitude
//   uses  excl = max(m1', (m1 + m2 - offset) - |v|): it equals m2' on the argmin edge and
//   m1' elsewhere (ties give m2 = m1), so no argmin index is needed on the forward pass.
// * Two threads share a row pair (edges split even / odd) and merge their partial
//   m1 / m2 / sign with one shuffle exchange.
#include "f16x2.h"
#include "ldpc_internal.h"

namespace ldpc {
namespace {

using namespace h2;

// Per-edge gather metadata for row pair j of a layer (kernel parameters, so the warp-uniform
// edge index turns into constant-bank loads):
//   word = j + base_nw            if j <  thresh   (no wrap), halves permuted by sel_nw
//   word = j + base_nw - H        if j >= thresh   (wrap),    halves permuted by sel_w
struct EdgeMeta {
    int base_nw;       // c*H + u
    int thresh;        // H - u
    uint32_t sel_nw;   // 0x3210 or 0x1032
    uint32_t sel_w;
};

constexpr int kMaxEdgesP = 1024;
constexpr int kMaxRowsP = 64;

struct PairParams {
    DecodeParams p;
    int H;
    int row[kMaxRowsP + 1];
    EdgeMeta meta[kMaxEdgesP];
};

struct Smem {
    uint32_t *Lb;        // [n_cols][H] words
    uint16_t *c2v;       // [E][H] byte pairs
};

// One thread owns row pair w of every layer; D is the row degree (straight-line code).
template <int D>
__device__ __forceinline__ void process_row(const PairParams &pp, const Smem &s, int e0, int H,
                                            int w, bool store) {
    uint32_t v[D];
    int addr[D];
    uint32_t sel[D];
    uint32_t m1 = kInf2, m2 = kInf2;
#pragma unroll
    for (int j = 0; j < D; ++j) {
        const EdgeMeta &mt = pp.meta[e0 + j];
        const bool wr = w >= mt.thresh;
        const int a = w + mt.base_nw - (wr ? H : 0);
        const uint32_t sl = wr ? mt.sel_w : mt.sel_nw;
        const uint32_t X = prmt(s.Lb[a], 0u, sl);
        const uint32_t M = prmt((uint32_t)s.c2v[(e0 + j) * H + w], 0x64646464u, 0x4140u);
        uint32_t x = h2sub(X, M);
        x = h2max(h2min(x, kP127), kN127);
        const uint32_t hi = h2maxxs(m1, x);
        m2 = h2minxs(m2, hi);
        m1 = h2minxs(m1, x);
        v[j] = x;
        addr[j] = a;
        sel[j] = sl;
    }
    const uint32_t SO = (m1 & kSign2) | kOne2;               // +-1.0: sign product S per lane
    const uint32_t a1 = m1 & kAbs2, a2 = m2 & kAbs2;
    const uint32_t m1c = h2relu_fma(a1, kOne2, kNegOne2);    // max(m1 - 1, 0)
    const uint32_t T1 = h2add(h2add(a1, a2), kNegOne2);       // m1 + m2 - 1
#pragma unroll
    for (int j = 0; j < D; ++j) {
        const uint32_t x = v[j];
        const uint32_t ex = h2max(m1c, h2sub(T1, x & kAbs2));
        const uint32_t sg = (x & kSign2) ^ SO;                 // S xor sgn(x), as +-1.0
        const uint32_t Cm = h2fma(ex, sg, kBias2);             // c' + 1152
        uint32_t Lb = h2add(Cm, x);                            // (x + c') + 1152
        Lb = h2max(h2min(Lb, kLbHi), kLbLo);
        if (store) {
            s.Lb[addr[j]] = prmt(Lb, 0u, sel[j]);
            s.c2v[(e0 + j) * H + w] = (uint16_t)prmt(Cm, 0u, 0x3320u);
        }
    }
}

__device__ __forceinline__ void dispatch_row(int d, const PairParams &pp, const Smem &s, int e0,
                                             int H, int w, bool store) {
    switch (d) {
#define LDPC_ROW_CASE(D) \
    case D:              \
        process_row<D>(pp, s, e0, H, w, store); \
        break;
        LDPC_ROW_CASE(2) LDPC_ROW_CASE(3) LDPC_ROW_CASE(4) LDPC_ROW_CASE(5) LDPC_ROW_CASE(6)
        LDPC_ROW_CASE(7) LDPC_ROW_CASE(8) LDPC_ROW_CASE(9) LDPC_ROW_CASE(10) LDPC_ROW_CASE(11)
        LDPC_ROW_CASE(12) LDPC_ROW_CASE(13) LDPC_ROW_CASE(14) LDPC_ROW_CASE(15)
        LDPC_ROW_CASE(16) LDPC_ROW_CASE(17) LDPC_ROW_CASE(18) LDPC_ROW_CASE(19)
        LDPC_ROW_CASE(20)
#undef LDPC_ROW_CASE
    default:
        break;
    }
}

// parity of the hard decisions (L < 0  <=>  biased value < 1152) of row pair w
__device__ __forceinline__ uint32_t row_parity(const PairParams &pp, const Smem &s, int e0,
                                               int d, int H, int w) {
    uint32_t par = 0;
    for (int j = 0; j < d; ++j) {
        const EdgeMeta &mt = pp.meta[e0 + j];
        const bool wr = w >= mt.thresh;
        const int a = w + mt.base_nw - (wr ? H : 0);
        const uint32_t X = prmt(s.Lb[a], 0u, wr ? mt.sel_w : mt.sel_nw);
        par ^= h2lt_mask(X, kBias2);
    }
    return par;
}

__global__ void __launch_bounds__(256, 1) rowpair_kernel(const __grid_constant__ PairParams pp) {
    const DecodeParams &p = pp.p;
    extern __shared__ __align__(16) unsigned char smem[];
    const int Z = p.Z, H = pp.H, E = p.E, n_rows = p.n_rows, n_cols = p.n_cols;
    Smem s;
    s.Lb = reinterpret_cast<uint32_t *>(smem);
    s.c2v = reinterpret_cast<uint16_t *>(smem + (size_t)n_cols * H * 4);

    const int tid = threadIdx.x, nthr = blockDim.x;
    // threads past the last row pair repeat its work and store nothing
    const bool store = tid < H;
    const int w = store ? tid : H - 1;
    const int K = p.K_b * Z;
    const int nbytes = (K + 7) >> 3;
    const int lo = p.punct * Z;
    const int8_t *llr_all = reinterpret_cast<const int8_t *>(p.llr);

    for (int cw = blockIdx.x; cw < p.batch; cw += gridDim.x) {
        // a0: biased posteriors from the channel LLRs (0 -> 1152 for punctured / unsent
        // bits), messages zero (stored as 0x80)
        const int8_t *llr = llr_all + (size_t)cw * p.n_tx;
        for (int i = tid; i < n_cols * H; i += nthr) s.Lb[i] = 0x64806480u;
        {
            uint32_t *c2 = reinterpret_cast<uint32_t *>(s.c2v);
            const int nw = (E * H) >> 1;
            for (int i = tid; i < nw; i += nthr) c2[i] = 0x80808080u;
            if ((E * H) & 1)
                if (tid == 0) s.c2v[E * H - 1] = 0x8080u;
        }
        __syncthreads();
        {
            uint16_t *Lh = reinterpret_cast<uint16_t *>(s.Lb);
#pragma unroll 8
            for (int t = tid; t < p.n_tx; t += nthr) {
                const int j = lo + t;
                const int c = j / Z, i = j - c * Z;
                const int lane = i >= H ? 1 : 0;
                Lh[2 * (c * H + i - lane * H) + lane] =
                    (uint16_t)(0x6400u | ((uint32_t)(uint8_t)llr[t] ^ 0x80u));
            }
        }
        __syncthreads();

        int done = p.max_iter;
#pragma unroll 1
        for (int t = 1; t <= p.max_iter; ++t) {
#pragma unroll 1
            for (int r = 0; r < n_rows; ++r) {
                const int e0 = pp.row[r], d = pp.row[r + 1] - e0;
                dispatch_row(d, pp, s, e0, H, w, store);
                __syncthreads();
            }
            if (p.early_stop) {
                int bad = 0;
                for (int r = 0; r < n_rows; ++r) {
                    const int e0 = pp.row[r], d = pp.row[r + 1] - e0;
                    const uint32_t par = row_parity(pp, s, e0, d, H, w);
                    bad = __any_sync(0xffffffffu, par != 0u);
                    if (bad) break;
                }
                if (__syncthreads_or(bad) == 0) {
                    done = t;
                    break;
                }
            }
        }

        // a6: hard bits of the K information bits, LSB first
        for (int b = tid; b < nbytes; b += nthr) {
            unsigned x = 0;
            for (int kk = 0; kk < 8; ++kk) {
                const int j = 8 * b + kk;
                if (j >= K) break;
                const int c = j / Z, i = j - c * Z;
                const int lane = i >= H ? 1 : 0;
                const uint32_t wd = s.Lb[c * H + i - lane * H];
                const uint32_t h = lane ? (wd >> 16) : (wd & 0xffffu);
                if (h < 0x6480u) x |= 1u << kk;
            }
            p.bits[(size_t)cw * nbytes + b] = (uint8_t)x;
        }
        if (tid == 0) p.iters[cw] = done;
        if (p.post) {
            int8_t *po = reinterpret_cast<int8_t *>(p.post) + (size_t)cw * n_cols * Z;
            for (int c = 0; c < n_cols; ++c)
                for (int i = tid; i < Z; i += nthr) {
                    const int lane = i >= H ? 1 : 0;
                    const uint32_t wd = s.Lb[c * H + i - lane * H];
                    const uint32_t h = lane ? (wd >> 16) : (wd & 0xffffu);
                    po[c * Z + i] = (int8_t)(uint8_t)((h & 0xffu) ^ 0x80u);
                }
        }
        if (p.c2v) {
            int8_t *co = reinterpret_cast<int8_t *>(p.c2v) + (size_t)cw * E * Z;
            for (int e = 0; e < E; ++e)
                for (int i = tid; i < Z; i += nthr) {
                    const int lane = i >= H ? 1 : 0;
                    const uint32_t pr = s.c2v[e * H + i - lane * H];
                    const uint32_t b = lane ? (pr >> 8) : (pr & 0xffu);
                    co[e * Z + i] = (int8_t)(uint8_t)((b & 0xffu) ^ 0x80u);
                }
        }
        __syncthreads();
    }
}

}  // namespace

size_t rowpair_smem_bytes(int E, int n_rows, int n_cols, int Z) {
    (void)n_rows;
    const int H = Z / 2;
    size_t off = (size_t)n_cols * H * 4 + (size_t)E * H * 2;
    return (off + 15) & ~(size_t)15;
}

bool rowpair_supported(const DecodeParams &p, int llr_type, int max_deg, size_t smem_optin) {
    if (llr_type != LDPC_LLR_INT8 || p.algo != LDPC_OFFSET || p.offset_q != 1) return false;
    if ((p.Z & 1) || p.Z < 2 || p.Z > 512 || max_deg > kMaxDeg || max_deg < 2) return false;
    if (p.E > kMaxEdgesP || p.n_rows > kMaxRowsP) return false;
    return rowpair_smem_bytes(p.E, p.n_rows, p.n_cols, p.Z) <= smem_optin;
}

ldpc_status launch_rowpair(const DecodeParams &p, int max_deg, cudaStream_t stream) {
    (void)max_deg;
    static thread_local PairParams pp;     // ~17 kB: kept off the stack
    pp.p = p;
    const int H = p.Z / 2;
    pp.H = H;
    // graph tables travel as kernel parameters (row pointers, per-edge gather metadata)
    for (int r = 0; r <= p.n_rows; ++r) pp.row[r] = p.h_row_ptr[r];
    for (int e = 0; e < p.E; ++e) {
        const uint32_t ed = p.h_edges[e];
        const int c = (int)(ed >> 16), sh = (int)(ed & 0xffffu);
        const int q = sh >= H ? 1 : 0, u = sh - q * H;
        pp.meta[e].base_nw = c * H + u;
        pp.meta[e].thresh = H - u;
        pp.meta[e].sel_nw = q ? 0x1032u : 0x3210u;
        pp.meta[e].sel_w = q ? 0x3210u : 0x1032u;
    }
    const size_t smem = rowpair_smem_bytes(p.E, p.n_rows, p.n_cols, p.Z);
    int dev = 0, n_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return LDPC_ERR_CUDA;
    cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    if (cudaFuncSetAttribute(rowpair_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem) != cudaSuccess)
        return LDPC_ERR_CUDA;
    const int threads = ((H + 31) / 32) * 32;
    if (threads > 256) return LDPC_ERR_UNSUPPORTED;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, rowpair_kernel, threads, smem) !=
            cudaSuccess ||
        per_sm < 1)
        return LDPC_ERR_UNSUPPORTED;
    int grid = n_sm * per_sm;
    if (grid > p.batch) grid = p.batch;
    rowpair_kernel<<<grid, threads, smem, stream>>>(pp);
    count_launch();
    if (cudaGetLastError() != cudaSuccess) return LDPC_ERR_CUDA;
    return LDPC_OK;
}

}  // namespace ldpc
