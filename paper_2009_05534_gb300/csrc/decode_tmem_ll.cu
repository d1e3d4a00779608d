// Low-latency decoders of the 8-bit offset min-sum: tmem_ll_kernel (one codeword per
// block, A = 2 or 4 cooperating threads per row pair) and the generic work-list kernel
// list_ll_kernel, with their launches.  The row step and the list kernel's body are in
// ll_kernel.cuh, whose header describes the mapping and the arithmetic.
#include "ldpc_internal.h"
#include "ll_kernel.cuh"

namespace ldpc {
namespace {

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

// ---------------------------------------------------------------------------- the kernel

template <int A>
__global__ void __launch_bounds__(A * 192, 1) tmem_ll_kernel(const __grid_constant__ LlParams pp) {
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
                if (tid == 0) atomicCAS(p.status, 0, (int)LDPC_ERR_TIMEOUT);
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
#pragma unroll 1
            for (int r = 0; r < n_rows; ++r) {
                const int e0 = pp.row[r];
                ll_dispatch<A>(pp.row[r + 1] - e0, s_meta, Lb, tbase, pp.slot[r], e0, H, w, k,
                               store);
                named_sync(1, nthr);
            }
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

int ll_slots(const int *row_ptr, int n_rows, int A, int *slot) {
    int s = 0;
    for (int r = 0; r < n_rows; ++r) {
        if (slot) slot[r] = s;
        s += (row_ptr[r + 1] - row_ptr[r] + A - 1) / A;
    }
    if (slot) slot[n_rows] = s;
    return s;
}

size_t ll_smem_bytes(const DecodeParams &p, bool tma) {
    const int H = p.Z / 2;
    size_t off = ((size_t)p.E * sizeof(EdgeMetaL) + 15) & ~(size_t)15;
    off = (off + (size_t)p.n_cols * H * 4 + 15) & ~(size_t)15;
    return off + (tma ? (size_t)p.n_tx : 0);
}

}  // namespace

bool tmem_ll_supported(const DecodeParams &p, int llr_type, int max_deg, int A,
                       size_t smem_optin) {
    if (A != 2 && A != 4) return false;
    if (llr_type != LDPC_LLR_INT8 || p.algo != LDPC_OFFSET || p.offset_q != 1) return false;
    if ((p.Z & 1) || p.Z < 2 || p.Z > 384 || max_deg > kMaxDeg || max_deg < 2) return false;
    if (p.E > kMaxEdgesL || p.n_rows > kMaxRowsL) return false;
    const int H = p.Z / 2;
    const int nwarps = (A * H + 31) / 32;
    const int depth = (nwarps + 3) / 4;                  // warps sharing a lane quarter
    const int ncols = (ll_slots(p.h_row_ptr, p.n_rows, A, nullptr) + 1) / 2;
    if (depth * ncols > kTmemColsL) return false;
    return ll_smem_bytes(p, true) + 64 <= smem_optin;
}

ldpc_status launch_tmem_ll(const DecodeParams &p, int A, cudaStream_t stream) {
    static thread_local LlParams pp;     // ~17 kB: kept off the stack
    pp.p = p;
    const int H = p.Z / 2;
    pp.H = H;
    for (int r = 0; r <= p.n_rows; ++r) pp.row[r] = p.h_row_ptr[r];
    pp.ncols = (ll_slots(p.h_row_ptr, p.n_rows, A, pp.slot) + 1) / 2;
    for (int e = 0; e < p.E; ++e) {
        const uint32_t ed = p.h_edges[e];
        const int c = (int)(ed >> 16), sh = (int)(ed & 0xffffu);
        const int q = sh >= H ? 1 : 0, u = sh - q * H;
        pp.meta[e].base_nw = c * H + u;
        pp.meta[e].thresh = H - u;
        pp.meta[e].sel_nw = q ? 0x1032u : 0x3210u;
        pp.meta[e].sel_w = q ? 0x3210u : 0x1032u;
    }
    // bulk copies need 16-byte aligned rows; at least 120 kB of shared memory so that one
    // block occupies the SM (its TMEM allocation takes all 512 columns)
    pp.use_tma = ((reinterpret_cast<uintptr_t>(p.llr) & 15u) == 0 && (p.n_tx % 16) == 0 &&
                  p.n_tx > 0 && p.n_tx < (1 << 20))
                     ? 1
                     : 0;
    pp.off_lb = (int)(((size_t)p.E * sizeof(EdgeMetaL) + 15) & ~(size_t)15);
    pp.off_stage = (pp.off_lb + p.n_cols * H * 4 + 15) & ~15;
    size_t smem = ll_smem_bytes(p, pp.use_tma != 0);
    if (smem < 120 * 1024) smem = 120 * 1024;
    int dev = 0, n_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return LDPC_ERR_CUDA;
    cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    const int threads = ((A * H + 31) / 32) * 32;
    int grid = p.batch < n_sm ? p.batch : n_sm;
    cudaError_t err;
    if (A == 2) {
        err = set_dyn_smem(reinterpret_cast<const void *>(tmem_ll_kernel<2>), smem);
        if (err == cudaSuccess) tmem_ll_kernel<2><<<grid, threads, smem, stream>>>(pp);
    } else {
        err = set_dyn_smem(reinterpret_cast<const void *>(tmem_ll_kernel<4>), smem);
        if (err == cudaSuccess) tmem_ll_kernel<4><<<grid, threads, smem, stream>>>(pp);
    }
    if (err != cudaSuccess) return LDPC_ERR_CUDA;
    count_launch();
    if (cudaGetLastError() != cudaSuccess) return LDPC_ERR_CUDA;
    return LDPC_OK;
}

// ------------------------------------------------------------ work list, low latency

namespace {

__global__ void __launch_bounds__(kThreadsLL, 1)
    list_ll_kernel(const ListItem *__restrict__ items, int n_items, int *counter,
                   int early_stop) {
    list_ll_body(items, n_items, counter, early_stop);
}

}  // namespace

bool list_ll_item_supported(int Z, int E, int n_rows, int max_deg, int slots2) {
    if ((Z & 1) || Z < 2 || Z > kThreadsLL || max_deg < 2 || max_deg > kMaxDeg) return false;
    if (E > kMaxEdgesL || n_rows > kMaxRowsL) return false;
    const int nwarps = (Z + 31) / 32;                // alpha * Z / 2 threads, alpha = 2
    const int depth = (nwarps + 3) / 4;
    return depth * ((slots2 + 1) / 2) <= kTmemColsL;
}

size_t list_ll_smem_bytes(int E, int n_cols, int Z, int n_tx) {
    const size_t off = ((size_t)E * sizeof(EdgeMetaL) + 15) & ~(size_t)15;
    const size_t stage = (off + (size_t)n_cols * (Z / 2) * 4 + 15) & ~(size_t)15;
    return stage + 16 + (size_t)n_tx + 16;
}

ldpc_status launch_list_ll(const ListItem *d_items, int n_items, int *d_counter, size_t smem,
                           int early_stop, cudaStream_t stream, const void *kernel) {
    int dev = 0, n_sm = 0, optin = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return LDPC_ERR_CUDA;
    cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    // at least 120 kB so that one block occupies the SM (its TMEM allocation takes all 512
    // columns; a second block would wait in the allocation)
    if (smem < 120 * 1024) smem = 120 * 1024;
    if (smem > (size_t)optin) return LDPC_ERR_UNSUPPORTED;
    const void *fn = kernel;
    if (!fn || set_dyn_smem(fn, smem) != cudaSuccess) {
        cudaGetLastError();
        fn = reinterpret_cast<const void *>(list_ll_kernel);
        if (set_dyn_smem(fn, smem) != cudaSuccess) return LDPC_ERR_CUDA;
    }
    const int grid = n_items < n_sm ? n_items : n_sm;
    void *args[] = {&d_items, &n_items, &d_counter, &early_stop};
    const cudaError_t e = cudaLaunchKernel(fn, dim3(grid), dim3(kThreadsLL), args, smem, stream);
    count_launch();
    if (e != cudaSuccess || cudaGetLastError() != cudaSuccess) return LDPC_ERR_CUDA;
    return LDPC_OK;
}

}  // namespace ldpc
