// Row-pair fp16x2 layered min-sum for 8-bit offset min-sum, messages in shared memory
// (sm_103a).  Used by the batch decode when the Tensor-Memory kernel does not take the shape,
// and by the work-list decode, which decodes a heterogeneous list of codewords (different
// graphs, lifting sizes and rates) in one launch.
//
// Same method as the generic kernel (paper Sec. III layered min-sum with correction,
// Sec. IV per-row m1 / m2 / sign quantities, hot-path steps a0..a6), mapped for GB300:
//
// * Lanes.  Check rows i and i + H (H = Z/2) of a layer travel together in one 32-bit
//   register as two binary16 lanes.  The 8-bit LLRs are integers in [-127, 127]; every
//   intermediate value is an integer of magnitude below 2048, so binary16 holds it
//   exactly and the results are bit-identical to 8-bit fixed-point arithmetic.
// * Posteriors in shared memory are stored biased by 1279: a word holds
//   (L[cZ+j] + 1279, L[cZ+j+H] + 1279) for j < H.  Biased values lie in [1152, 1406],
//   where binary16 has spacing 1, and the bit pattern of 1024 + b is 0x6400 + b.
// * Check-to-variable messages are kept expanded, one byte per (edge, row), as c + 128.
//   One PRMT that inserts the byte under the exponent 0x64 turns it into binary16
//   c + 1152, so (L + 1279) - (c + 1152) = v + 127 is one subtraction; two relu FMAs
//   give sat(v) = 127 - max(254 - max(v + 127, 0), 0) without min/max, and the new
//   message c' + 1152 = fma(|m'|, +-1, 1152) is stored back by taking its low byte.
// * Circulant gather: row j (< H) of a circulant with shift s = qH + u reads word
//   (j + u) mod H with its halves exchanged when q xor [j + u >= H]; the same
//   permutation writes the result back.
// * Check node: min.xorsign.abs.f16x2 gives min(|m1|, |v|) with the sign product in one
//   instruction; m2 follows from max.xorsign / min.xorsign.  The new message magnitude
//   uses  excl = max(m1', (m1 + m2 - offset) - |v|): it equals m2' on the argmin edge and
//   m1' elsewhere (ties give m2 = m1), so no argmin index is needed on the forward pass.
// * One thread owns one row pair of every layer; the per-edge gather metadata sits in
//   shared memory and is read with one broadcast 16-byte load per edge.
#include <mutex>

#include "f16x2.h"
#include "ldpc_internal.h"

namespace ldpc {
namespace {

using namespace h2;

// Per-edge gather metadata for row pair j of a layer:
//   word = j + base_nw            if j <  thresh   (no wrap), halves permuted by sel_nw
//   word = j + base_nw - H        if j >= thresh   (wrap),    halves permuted by sel_w
struct EdgeMeta {
    int base_nw;       // c*H + u
    int thresh;        // H - u
    uint32_t sel_nw;   // 0x3210 or 0x1032
    uint32_t sel_w;
};

__host__ __device__ __forceinline__ EdgeMeta make_meta(uint32_t edge, int H) {
    const int c = (int)(edge >> 16), sh = (int)(edge & 0xffffu);
    const int q = sh >= H ? 1 : 0, u = sh - q * H;
    EdgeMeta m;
    m.base_nw = c * H + u;
    m.thresh = H - u;
    m.sel_nw = q ? 0x1032u : 0x3210u;
    m.sel_w = q ? 0x3210u : 0x1032u;
    return m;
}

constexpr int kMaxEdgesP = 1024;
constexpr int kMaxRowsP = 64;
constexpr int kThreadsP = 192;      // one thread per row pair, Z <= 384

// Everything one codeword's decode needs.
struct CwArgs {
    int Z, H, K_b, n_rows, n_cols, E;
    int punct, n_tx, max_iter, early_stop;
    const int8_t *llr;     // [n_tx]
    uint8_t *bits;         // [ceil(K/8)]
    int32_t *iters;        // [1]
    int8_t *post;          // [n_cols * Z] or null
    int8_t *c2v;           // [E * Z] or null
};

struct Smem {
    const EdgeMeta *meta;   // [E]
    const int *row;         // [n_rows + 1]
    uint32_t *Lb;           // [n_cols][H] words
    uint16_t *c2v;          // [E][H] byte pairs
};

// One thread owns row pair w of every layer; D is the row degree (straight-line code).
template <int D>
__device__ __forceinline__ void process_row(const Smem &s, int e0, int H, int w, bool store) {
    uint32_t v[D];
    int addr[D];
    uint32_t sel[D];
    uint32_t m1 = kInf2, m2 = kInf2;
#pragma unroll
    for (int j = 0; j < D; ++j) {
        const EdgeMeta mt = s.meta[e0 + j];
        const bool wr = w >= mt.thresh;
        const int a = w + mt.base_nw - (wr ? H : 0);
        const uint32_t sl = wr ? mt.sel_w : mt.sel_nw;
        const uint32_t X = prmt(s.Lb[a], 0u, sl);
        const uint32_t M = prmt((uint32_t)s.c2v[(e0 + j) * H + w], 0x64646464u, 0x4140u);
        // sat(L - c) through two relu FMAs: y = max(v + 127, 0), z = max(254 - y, 0)
        const uint32_t y = h2relu_fma(M, kNegOne2, X);
        const uint32_t x = h2sub(kP127, h2relu_fma(y, kNegOne2, k254));
        m2 = h2min(m2, h2max(h2abs(m1), h2abs(x)));
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
        const uint32_t ex = h2max(m1c, h2sub(T1, h2abs(x)));
        const uint32_t sg = (x & kSign2) ^ SO;                 // S xor sgn(x), as +-1.0
        const uint32_t Cm = h2fma(ex, sg, kBias2);             // c' + 1152
        uint32_t Lb = h2add(Cm, h2add(x, kP127));              // (x + c') + 1279
        Lb = h2max(h2min(Lb, kPostHi), kPostLo);
        if (store) {
            s.Lb[addr[j]] = prmt(Lb, 0u, sel[j]);
            s.c2v[(e0 + j) * H + w] = (uint16_t)prmt(Cm, 0u, 0x3320u);
        }
    }
}

__device__ __forceinline__ void dispatch_row(int d, const Smem &s, int e0, int H, int w,
                                             bool store) {
    switch (d) {
#define LDPC_ROW_CASE(D) \
    case D:              \
        process_row<D>(s, e0, H, w, store); \
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

// parity of the hard decisions (L < 0  <=>  biased value < 1279) of row pair w
__device__ __forceinline__ uint32_t row_parity(const Smem &s, int e0, int d, int H, int w) {
    uint32_t par = 0;
    for (int j = 0; j < d; ++j) {
        const EdgeMeta mt = s.meta[e0 + j];
        const bool wr = w >= mt.thresh;
        const int a = w + mt.base_nw - (wr ? H : 0);
        par ^= h2lt_mask(prmt(s.Lb[a], 0u, wr ? mt.sel_w : mt.sel_nw), kPostBias);
    }
    return par;
}

// Decode one codeword with the whole block (blockDim.x >= H threads; the graph metadata is
// already in shared memory).  Starts and ends with the block synchronised.
__device__ void decode_codeword(const CwArgs &a, const Smem &s) {
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int Z = a.Z, H = a.H, E = a.E, n_cols = a.n_cols;
    const bool store = tid < H;
    const int w = store ? tid : H - 1;       // spare threads shadow the last row pair
    const int lo = a.punct * Z;

    // a0: biased posteriors from the channel LLRs, zero messages (stored as 0x80)
    for (int c = 0; c < n_cols; ++c)
        for (int j = tid; j < H; j += nthr) {
            const int t0 = c * Z + j - lo, t1 = t0 + H;
            // binary16 L + 1279 = 1024 + (L + 255): bit pattern 0x6400 + L + 255
            const int q0 = (t0 >= 0 && t0 < a.n_tx) ? (int)a.llr[t0] : 0;
            const int q1 = (t1 >= 0 && t1 < a.n_tx) ? (int)a.llr[t1] : 0;
            s.Lb[c * H + j] = (uint32_t)(0x64FF + q0) | ((uint32_t)(0x64FF + q1) << 16);
        }
    {
        uint32_t *c2 = reinterpret_cast<uint32_t *>(s.c2v);
        const int nw = (E * H) >> 1;
        for (int i = tid; i < nw; i += nthr) c2[i] = 0x80808080u;
        if (((E * H) & 1) && tid == 0) s.c2v[E * H - 1] = 0x8080u;
    }
    __syncthreads();

    int done = a.max_iter;
#pragma unroll 1
    for (int t = 1; t <= a.max_iter; ++t) {
#pragma unroll 1
        for (int r = 0; r < a.n_rows; ++r) {
            const int e0 = s.row[r], d = s.row[r + 1] - e0;
            dispatch_row(d, s, e0, H, w, store);
            __syncthreads();
        }
        if (a.early_stop) {
            int bad = 0;
            for (int r = 0; r < a.n_rows && !bad; ++r) {
                const int e0 = s.row[r], d = s.row[r + 1] - e0;
                bad = __any_sync(0xffffffffu, row_parity(s, e0, d, H, w) != 0u);
            }
            if (__syncthreads_or(bad) == 0) {
                done = t;
                break;
            }
        }
    }

    // a6: hard bits of the K information bits, LSB first; iteration count
    const int K = a.K_b * Z, nbytes = (K + 7) >> 3;
    for (int b = tid; b < nbytes; b += nthr) {
        unsigned x = 0;
        for (int kk = 0; kk < 8; ++kk) {
            const int j = 8 * b + kk;
            if (j >= K) break;
            const int c = j / Z, i = j - c * Z;
            const int lane = i >= H ? 1 : 0;
            const uint32_t wd = s.Lb[c * H + i - lane * H];
            const uint32_t h = lane ? (wd >> 16) : (wd & 0xffffu);
            if (h < 0x64FFu) x |= 1u << kk;
        }
        a.bits[b] = (uint8_t)x;
    }
    if (tid == 0) a.iters[0] = done;
    if (a.post)
        for (int c = 0; c < n_cols; ++c)
            for (int i = tid; i < Z; i += nthr) {
                const int lane = i >= H ? 1 : 0;
                const uint32_t wd = s.Lb[c * H + i - lane * H];
                const uint32_t h = lane ? (wd >> 16) : (wd & 0xffffu);
                a.post[c * Z + i] = (int8_t)((int)h - 0x64FF);
            }
    if (a.c2v)
        for (int e = 0; e < E; ++e)
            for (int i = tid; i < Z; i += nthr) {
                const int lane = i >= H ? 1 : 0;
                const uint32_t pr = s.c2v[e * H + i - lane * H];
                const uint32_t b = lane ? (pr >> 8) : (pr & 0xffu);
                a.c2v[e * Z + i] = (int8_t)(uint8_t)((b & 0xffu) ^ 0x80u);
            }
    __syncthreads();
}

// shared-memory carve-up: metadata | row pointers | posteriors | messages
__host__ __device__ __forceinline__ size_t smem_layout(int E, int n_rows, int n_cols, int H,
                                                       size_t *off_row, size_t *off_lb,
                                                       size_t *off_c2v) {
    size_t off = (size_t)E * sizeof(EdgeMeta);
    *off_row = off;
    off += (size_t)(n_rows + 1) * 4;
    off = (off + 15) & ~(size_t)15;
    *off_lb = off;
    off += (size_t)n_cols * H * 4;
    *off_c2v = off;
    off += (size_t)E * H * 2;
    return (off + 15) & ~(size_t)15;
}

// ----------------------------------------------------------------------- batch kernel

struct PairParams {
    DecodeParams p;
    int H;
    int row[kMaxRowsP + 1];
    EdgeMeta meta[kMaxEdgesP];
};

__global__ void __launch_bounds__(kThreadsP, 1) rowpair_kernel(const __grid_constant__ PairParams pp) {
    const DecodeParams &p = pp.p;
    extern __shared__ __align__(16) unsigned char smem[];
    const int H = pp.H;
    size_t off_row, off_lb, off_c2v;
    smem_layout(p.E, p.n_rows, p.n_cols, H, &off_row, &off_lb, &off_c2v);
    EdgeMeta *s_meta = reinterpret_cast<EdgeMeta *>(smem);
    int *s_row = reinterpret_cast<int *>(smem + off_row);
    for (int e = threadIdx.x; e < p.E; e += blockDim.x) s_meta[e] = pp.meta[e];
    for (int r = threadIdx.x; r <= p.n_rows; r += blockDim.x) s_row[r] = pp.row[r];
    Smem s{s_meta, s_row, reinterpret_cast<uint32_t *>(smem + off_lb),
           reinterpret_cast<uint16_t *>(smem + off_c2v)};
    __syncthreads();
    const int nbytes = (p.K_b * p.Z + 7) >> 3;
    for (int cw = blockIdx.x; cw < p.batch; cw += gridDim.x) {
        CwArgs a;
        a.Z = p.Z; a.H = H; a.K_b = p.K_b; a.n_rows = p.n_rows; a.n_cols = p.n_cols; a.E = p.E;
        a.punct = p.punct; a.n_tx = p.n_tx; a.max_iter = p.max_iter; a.early_stop = p.early_stop;
        a.llr = reinterpret_cast<const int8_t *>(p.llr) + (size_t)cw * p.n_tx;
        a.bits = p.bits + (size_t)cw * nbytes;
        a.iters = p.iters + cw;
        a.post = p.post ? reinterpret_cast<int8_t *>(p.post) + (size_t)cw * p.n_cols * p.Z : nullptr;
        a.c2v = p.c2v ? reinterpret_cast<int8_t *>(p.c2v) + (size_t)cw * p.E * p.Z : nullptr;
        decode_codeword(a, s);
    }
}

// ------------------------------------------------------------------- work-list kernel

__global__ void __launch_bounds__(kThreadsP, 1)
    list_kernel(const ListItem *__restrict__ items, int n_items, int *counter, int early_stop) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_idx;
    for (;;) {
        if (threadIdx.x == 0) s_idx = atomicAdd(counter, 1);
        __syncthreads();
        const int idx = s_idx;
        __syncthreads();
        if (idx >= n_items) break;
        const ListItem it = items[idx];
        const int H = it.Z / 2;
        size_t off_row, off_lb, off_c2v;
        smem_layout(it.E, it.n_rows, it.n_cols, H, &off_row, &off_lb, &off_c2v);
        EdgeMeta *s_meta = reinterpret_cast<EdgeMeta *>(smem);
        int *s_row = reinterpret_cast<int *>(smem + off_row);
        for (int e = threadIdx.x; e < it.E; e += blockDim.x) s_meta[e] = make_meta(it.edges[e], H);
        for (int r = threadIdx.x; r <= it.n_rows; r += blockDim.x) s_row[r] = it.row_ptr[r];
        __syncthreads();
        Smem s{s_meta, s_row, reinterpret_cast<uint32_t *>(smem + off_lb),
               reinterpret_cast<uint16_t *>(smem + off_c2v)};
        CwArgs a;
        a.Z = it.Z; a.H = H; a.K_b = it.K_b; a.n_rows = it.n_rows; a.n_cols = it.n_cols;
        a.E = it.E; a.punct = it.punct; a.n_tx = it.n_tx; a.max_iter = it.max_iter;
        a.early_stop = early_stop;
        a.llr = it.llr; a.bits = it.bits; a.iters = it.iters; a.post = nullptr; a.c2v = nullptr;
        decode_codeword(a, s);
    }
}

}  // namespace

size_t rowpair_smem_bytes(int E, int n_rows, int n_cols, int Z) {
    size_t a, b, c;
    return smem_layout(E, n_rows, n_cols, Z / 2, &a, &b, &c);
}

bool rowpair_supported(const DecodeParams &p, int llr_type, int max_deg, size_t smem_optin) {
    if (llr_type != LDPC_LLR_INT8 || p.algo != LDPC_OFFSET || p.offset_q != 1) return false;
    if ((p.Z & 1) || p.Z < 2 || p.Z > 2 * kThreadsP || max_deg > kMaxDeg || max_deg < 2)
        return false;
    if (p.E > kMaxEdgesP || p.n_rows > kMaxRowsP) return false;
    return rowpair_smem_bytes(p.E, p.n_rows, p.n_cols, p.Z) <= smem_optin;
}

bool list_item_supported(int Z, int E, int n_rows, int max_deg) {
    return !(Z & 1) && Z >= 2 && Z <= 2 * kThreadsP && max_deg >= 2 && max_deg <= kMaxDeg &&
           E <= kMaxEdgesP && n_rows <= kMaxRowsP;
}

ldpc_status launch_rowpair(const DecodeParams &p, int max_deg, cudaStream_t stream) {
    (void)max_deg;
    static thread_local PairParams pp;     // ~17 kB: kept off the stack
    pp.p = p;
    const int H = p.Z / 2;
    pp.H = H;
    // graph tables travel as kernel parameters (row pointers, per-edge gather metadata)
    for (int r = 0; r <= p.n_rows; ++r) pp.row[r] = p.h_row_ptr[r];
    for (int e = 0; e < p.E; ++e) pp.meta[e] = make_meta(p.h_edges[e], H);
    const size_t smem = rowpair_smem_bytes(p.E, p.n_rows, p.n_cols, p.Z);
    int dev = 0, n_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return LDPC_ERR_CUDA;
    cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    if (set_dyn_smem(reinterpret_cast<const void *>(rowpair_kernel), smem) != cudaSuccess)
        return LDPC_ERR_CUDA;
    const int threads = ((H + 31) / 32) * 32;
    int per_sm = 0;
    if (blocks_per_sm(&per_sm, reinterpret_cast<const void *>(rowpair_kernel), threads, smem) !=
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

ldpc_status launch_list(const ListItem *d_items, int n_items, int *d_counter, size_t smem,
                        int early_stop, cudaStream_t stream) {
    int dev = 0, n_sm = 0, optin = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return LDPC_ERR_CUDA;
    cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (smem > (size_t)optin) return LDPC_ERR_UNSUPPORTED;
    if (set_dyn_smem(reinterpret_cast<const void *>(list_kernel), smem) != cudaSuccess)
        return LDPC_ERR_CUDA;
    int per_sm = 0;
    if (blocks_per_sm(&per_sm, reinterpret_cast<const void *>(list_kernel), kThreadsP, smem) !=
            cudaSuccess ||
        per_sm < 1)
        return LDPC_ERR_UNSUPPORTED;
    int grid = n_sm * per_sm;
    if (grid > n_items) grid = n_items;
    list_kernel<<<grid, kThreadsP, smem, stream>>>(d_items, n_items, d_counter, early_stop);
    count_launch();
    if (cudaGetLastError() != cudaSuccess) return LDPC_ERR_CUDA;
    return LDPC_OK;
}

size_t list_item_smem_bytes(int E, int n_rows, int n_cols, int Z) {
    return rowpair_smem_bytes(E, n_rows, n_cols, Z);
}

// ------------------------------------------------- work list without allocation
//
// Some callers cannot allocate device memory: code that runs inside another framework's
// memory pool, under a driver or RTOS layer with a fixed memory map, or on a path where a
// cudaMalloc would synchronise the device.  For them the work table and the work counter
// of the work-list decode live in this file-scope array, which every GPU that loads the
// library keeps until exit.  Host code only ever sees the array's host-side stand-in, so
// its device address is looked up once per device with cudaGetSymbolAddress.

namespace {
struct NoAllocScratch {
    ListItem items[kNoAllocMaxItems];
    int counter;
};
static __device__ __align__(256) NoAllocScratch g_noalloc_scratch;

std::mutex g_noalloc_mu;                         // guards the host-side staging below
NoAllocScratch *g_noalloc_dev[64] = {};          // device address, per device ordinal
ListItem g_noalloc_host[kNoAllocMaxItems];        // host staging of the sorted table
}  // namespace

ldpc_status launch_list_noalloc(const ListItem *h_items, int n_items, size_t smem,
                                int early_stop, bool ll, cudaStream_t stream) {
    if (n_items < 0 || n_items > kNoAllocMaxItems) return LDPC_ERR_INVALID_ARG;
    if (n_items == 0) return LDPC_OK;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return LDPC_ERR_CUDA;
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_dev[dev]) {
        // set-up: once per device, with that device current
        void *ptr = nullptr;
        if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) {
            cudaGetLastError();
            return LDPC_ERR_CUDA;
        }
        g_noalloc_dev[dev] = static_cast<NoAllocScratch *>(ptr);
    }
    NoAllocScratch *d = g_noalloc_dev[dev];
    for (int k = 0; k < n_items; ++k) g_noalloc_host[k] = h_items[k];
    // pageable source: this relies on the behaviour CUDA documents for asynchronous copies
    // from pageable host memory, which copy the source into a driver staging buffer before
    // the call returns; the static staging array is then free for the next call
    if (cudaMemcpyAsync(d->items, g_noalloc_host, (size_t)n_items * sizeof(ListItem),
                        cudaMemcpyHostToDevice, stream) != cudaSuccess ||
        cudaMemsetAsync(&d->counter, 0, sizeof(int), stream) != cudaSuccess)
        return LDPC_ERR_CUDA;
    return ll ? launch_list_ll(d->items, n_items, &d->counter, smem, early_stop, stream)
              : launch_list(d->items, n_items, &d->counter, smem, early_stop, stream);
}

}  // namespace ldpc
