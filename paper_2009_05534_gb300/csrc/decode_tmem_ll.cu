// Low-latency decoders of the 8-bit offset min-sum: tmem_ll_kernel (one codeword per
// block, A = 2 or 4 cooperating threads per row pair) and the generic work-list kernel
// list_ll_kernel, with their launches.  The row step and the list kernel's body are in
// ll_kernel.cuh, whose header describes the mapping and the arithmetic.
#include "ldpc_internal.h"
#include "ll_kernel.cuh"

namespace ldpc {
namespace {

// ---------------------------------------------------------------------------- the kernel

template <int A>
__global__ void __launch_bounds__(A * 192, 1) tmem_ll_kernel(const __grid_constant__ LlParams pp) {
    ll_body<A>(pp);
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
    // the kernel compiled for this row sequence, else the generic one
    const void *generic = A == 2 ? reinterpret_cast<const void *>(tmem_ll_kernel<2>)
                                 : reinterpret_cast<const void *>(tmem_ll_kernel<4>);
    const void *fn = ll_jit_kernel(p, A);
    if (!fn || set_dyn_smem(fn, smem) != cudaSuccess) {
        cudaGetLastError();
        fn = generic;
        if (set_dyn_smem(fn, smem) != cudaSuccess) return LDPC_ERR_CUDA;
    }
    void *args[] = {&pp};
    const cudaError_t err = cudaLaunchKernel(fn, dim3(grid), dim3(threads), args, smem, stream);
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
