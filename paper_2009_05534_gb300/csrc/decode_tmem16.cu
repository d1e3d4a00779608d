// Host side of the binary16 decoder: the generic kernels (one switch per row on its
// degree), block shape and shared-memory layout, and the launch, which takes the kernel
// compiled at run time for the row sequence when there is one (t16_jit.cu).  The kernel
// itself is in t16_kernel.cuh, whose header describes the arithmetic and the mapping.
#include "ldpc_internal.h"
#include "t16_kernel.cuh"

namespace ldpc {
namespace {

template <int kCw, bool kHybrid>
__global__ void __launch_bounds__(384, 1) tmem16_kernel(const __grid_constant__ Tmem16Params pp) {
    t16_body<kCw, kHybrid>(pp);
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
    auto generic = sh.cw == 4 ? (hybrid ? tmem16_kernel<4, true> : tmem16_kernel<4, false>)
                 : sh.cw == 2 ? tmem16_kernel<2, false>
                              : (hybrid ? tmem16_kernel<1, true> : tmem16_kernel<1, false>);
    // the kernel compiled for this row sequence and shape, else the generic one; not for
    // the hybrid shape, whose rows each carry both message paths: written out, its layer
    // loop is twice as long and measured slower than the generic kernel (1.97 vs 1.49 ms,
    // BG1-shaped Z=384, batch 1024), while the rate-8/9 shape gains (1.37 vs 1.52 ms)
    const void *kern = hybrid ? nullptr : t16_jit_kernel(p, sh.cw, hybrid);
    if (!kern) kern = reinterpret_cast<const void *>(generic);
    // blocks per SM: as many as shared memory and the 512 TMEM columns allow; the shared
    // memory request is raised so that no more blocks fit than TMEM can hold (a block
    // beyond that would only wait in tcgen05.alloc)
    const int by_tmem = kTmemCols16 / sh.tcols;
    int smem_sm = 0;
    cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    size_t smem = l.total;
    const size_t floor_b = (size_t)smem_sm / (by_tmem + 1) + 1024;
    if (smem < floor_b && floor_b <= (size_t)smem_optin) smem = floor_b;
    if (set_dyn_smem(kern, smem) != cudaSuccess) {
        cudaGetLastError();
        kern = reinterpret_cast<const void *>(generic);
        if (set_dyn_smem(kern, smem) != cudaSuccess) return LDPC_ERR_CUDA;
    }
    const int threads = sh.cw * sh.wpc * 32;
    int per_sm = 0;
    if (blocks_per_sm(&per_sm, kern, threads, smem) != cudaSuccess || per_sm < 1)
        return LDPC_ERR_UNSUPPORTED;
    if (per_sm > by_tmem) per_sm = by_tmem;
    int grid = n_sm * per_sm;
    const int units = (p.batch + sh.cw - 1) / sh.cw;
    if (grid > units) grid = units;
    if (grid < 1) grid = 1;
    void *args[] = {&pp};
    const cudaError_t e = cudaLaunchKernel(kern, dim3(grid), dim3(threads), args, smem, stream);
    count_launch();
    if (e != cudaSuccess || cudaGetLastError() != cudaSuccess) return LDPC_ERR_CUDA;
    return LDPC_OK;
}

}  // namespace ldpc
