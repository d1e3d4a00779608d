// Host side of the batch kernel of decode_tmem_pair: the generic kernel (one switch per row
// on the row's degree and first-edge parity) and the launch, which takes the kernel
// compiled at run time for the graph's row sequence when there is one (pair_jit.cu).
// The kernel itself is in pair_kernel.cuh.
#include "ldpc_internal.h"
#include "pair_kernel.cuh"

namespace ldpc {
static_assert(kStatusTimeout == (int)LDPC_ERR_TIMEOUT, "status code of a bounded wait");
namespace {

__global__ void __launch_bounds__(kThreadsQ, 1) pair_kernel(const __grid_constant__ PairParams pp) {
    pair_body(pp);
}

size_t pair_smem_bytes(const DecodeParams &p, bool tma, int *off_meta, int *off_stage,
                       int *stage_bytes) {
    const size_t lb = (size_t)p.n_cols * p.Z * 4;
    const int mt = (int)((lb + 15) & ~(size_t)15);
    const int st = (int)((mt + (size_t)p.E * sizeof(EdgeMetaQ) + 15) & ~(size_t)15);
    const int sb = tma ? ((p.n_tx + 15) & ~15) : 0;
    if (off_meta) *off_meta = mt;
    if (off_stage) *off_stage = st;
    if (stage_bytes) *stage_bytes = sb;
    return (size_t)st + 2 * (size_t)sb;
}

}  // namespace

bool pair_supported(const DecodeParams &p, int llr_type, int max_deg, size_t smem_optin) {
    if (llr_type != LDPC_LLR_INT8 || p.algo != LDPC_OFFSET || p.offset_q != 1) return false;
    if (p.Z < 1 || p.Z > kThreadsQ || max_deg > kMaxDeg || max_deg < 2) return false;
    if (p.E > kMaxEdgesQ || p.n_rows > kMaxRowsQ) return false;
    const int nwarps = (p.Z + 31) / 32;
    const int depth = (nwarps + 3) / 4;
    if (depth * ((p.E + 1) / 2) > kTmemColsQ) return false;
    return pair_smem_bytes(p, true, nullptr, nullptr, nullptr) + 64 <= smem_optin;
}

ldpc_status launch_pair(const DecodeParams &p, cudaStream_t stream) {
    static thread_local PairParams pp;     // ~10 kB: kept off the stack
    pp.p = p;
    for (int r = 0; r <= p.n_rows; ++r) pp.row[r] = p.h_row_ptr[r];
    pp.ncols = (p.E + 1) / 2;
    for (int e = 0; e < p.E; ++e) {
        const uint32_t ed = p.h_edges[e];
        pp.meta[e].s4 = 4 * (int)(ed & 0xffffu);
        pp.meta[e].col4 = 4 * (int)(ed >> 16) * p.Z;
    }
    // bulk copies need 16-byte aligned rows; at least 120 kB of shared memory so that one
    // block occupies the SM (its TMEM allocation takes all 512 columns)
    pp.use_tma = ((reinterpret_cast<uintptr_t>(p.llr) & 15u) == 0 && (p.n_tx % 16) == 0 &&
                  p.n_tx > 0 && p.n_tx < (1 << 20))
                     ? 1
                     : 0;
    size_t smem = pair_smem_bytes(p, pp.use_tma != 0, &pp.off_meta, &pp.off_stage, &pp.stage_bytes);
    if (smem < 120 * 1024) smem = 120 * 1024;
    int dev = 0, n_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return LDPC_ERR_CUDA;
    cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    // the kernel compiled for this row sequence, else the generic one
    const void *fn = pair_jit_kernel(p);
    if (!fn || set_dyn_smem(fn, smem) != cudaSuccess) {
        cudaGetLastError();
        fn = reinterpret_cast<const void *>(pair_kernel);
        if (set_dyn_smem(fn, smem) != cudaSuccess) return LDPC_ERR_CUDA;
    }
    const int threads = ((p.Z + 31) / 32) * 32;
    int grid = (p.batch + 1) / 2;
    if (grid > n_sm) grid = n_sm;
    void *args[] = {&pp};
    const cudaError_t e = cudaLaunchKernel(fn, dim3(grid), dim3(threads), args, smem, stream);
    count_launch();
    if (e != cudaSuccess || cudaGetLastError() != cudaSuccess) return LDPC_ERR_CUDA;
    return LDPC_OK;
}

}  // namespace ldpc
