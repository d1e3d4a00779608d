// Flooding-schedule decoder, fp32: min-sum with a normalised / offset correction or the
// exact sum-product (tanh) rule (sm_103a).  Paper: Sec. III (check rule with correction,
// the box-plus rule it approximates, posterior = channel LLR + sum of incoming messages),
// Sec. V (the flooding decoders the paper compares its layered decoder against).
//
// Iteration t: every check row of every used base row computes its new messages from the
// posteriors of iteration t-1 (v = L - c_old), then every posterior is recomputed as its
// channel LLR plus its incoming messages, summed in base-row order; after that the syndrome
// of the hard decisions decides the early stop.  All operations are single-rounded binary32
// (min-sum) so the results match the scalar definition operation for operation; the
// sum-product rule evaluates tanh / atanh and the products over the other edges in binary64
// and clamps the product to +-(1 - 1e-15) before atanh.
//
// Mapping: one thread block per codeword (persistent grid-stride loop over the batch); the
// posteriors live in shared memory, the messages ([E][Z] floats per codeword, too large for
// shared memory at Z = 384) in a caller workspace in HBM, read and written coalesced (thread
// i of a check row pass touches message (e, i); thread p of a variable pass touches
// (e, (p - s) mod Z)).  Block barriers separate the check pass, the variable pass and the
// syndrome test.
#include "ldpc_internal.h"

namespace ldpc {
namespace {

constexpr int kMaxEdgesF = 1024;
constexpr int kMaxDegF = 24;

struct FloodParams {
    DecodeParams p;
    float *ws;                   // [batch][E * Z] messages
    int col_ptr[kMaxCols + 1];   // edges of column c: col_edge[col_ptr[c] .. col_ptr[c+1])
    int col_edge[kMaxEdgesF];    // edge indices, in increasing edge (= base row) order
};

__device__ __forceinline__ int fvar(uint32_t edge, int i, int Z) {
    int q = i + (int)(edge & 0xffffu);
    if (q >= Z) q -= Z;
    return (int)(edge >> 16) * Z + q;
}

__device__ __forceinline__ float channel(const DecodeParams &p, int cw, int j) {
    const int t = j - p.punct * p.Z;
    return (t >= 0 && t < p.n_tx) ? reinterpret_cast<const float *>(p.llr)[(size_t)cw * p.n_tx + t]
                                  : 0.0f;
}

// one check row (r, i): new messages from the previous posteriors
__device__ __forceinline__ void check_row(const DecodeParams &p, const uint32_t *s_edge, int e0,
                                          int d, int i, const float *L, float *C) {
    const int Z = p.Z;
    float v[kMaxDegF];
#pragma unroll
    for (int k = 0; k < kMaxDegF; ++k)
        if (k < d) v[k] = __fsub_rn(L[fvar(s_edge[e0 + k], i, Z)], C[(size_t)(e0 + k) * Z + i]);
    if (p.algo == LDPC_SUM_PRODUCT) {
        double tv[kMaxDegF];
#pragma unroll
        for (int k = 0; k < kMaxDegF; ++k)
            if (k < d) tv[k] = tanh(0.5 * (double)v[k]);
#pragma unroll
        for (int k = 0; k < kMaxDegF; ++k) {
            if (k < d) {
                double pr = 1.0;
#pragma unroll
                for (int j = 0; j < kMaxDegF; ++j)
                    if (j < d && j != k) pr *= tv[j];
                if (pr > 1.0 - 1e-15) pr = 1.0 - 1e-15;
                if (pr < -1.0 + 1e-15) pr = -1.0 + 1e-15;
                C[(size_t)(e0 + k) * Z + i] = (float)(2.0 * atanh(pr));
            }
        }
        return;
    }
    float m1 = __int_as_float(0x7f800000), m2 = m1;
    int idx = -1, S = 0;
#pragma unroll
    for (int k = 0; k < kMaxDegF; ++k) {
        if (k < d) {
            const float a = fabsf(v[k]);
            if (a < m1) {
                m2 = m1;
                m1 = a;
                idx = k;
            } else if (a < m2) {
                m2 = a;
            }
            S ^= (v[k] < 0.0f) ? 1 : 0;
        }
    }
    float m1c, m2c;
    if (p.algo == LDPC_NORMALISED) {
        m1c = __fmul_rn(p.alpha, m1);
        m2c = __fmul_rn(p.alpha, m2);
    } else {
        m1c = fmaxf(__fsub_rn(m1, p.offset), 0.0f);
        m2c = fmaxf(__fsub_rn(m2, p.offset), 0.0f);
    }
#pragma unroll
    for (int k = 0; k < kMaxDegF; ++k) {
        if (k < d) {
            const float mag = (k == idx) ? m2c : m1c;
            C[(size_t)(e0 + k) * Z + i] = ((S ^ ((v[k] < 0.0f) ? 1 : 0)) != 0) ? -mag : mag;
        }
    }
}

__global__ void __launch_bounds__(256) flood_kernel(const __grid_constant__ FloodParams fp) {
    const DecodeParams &p = fp.p;
    extern __shared__ __align__(16) unsigned char smem[];
    const int Z = p.Z, E = p.E, n_rows = p.n_rows, N = p.n_cols * Z;
    uint32_t *s_edge = reinterpret_cast<uint32_t *>(smem);
    int *s_row = reinterpret_cast<int *>(s_edge + E);
    float *L = reinterpret_cast<float *>(smem + (((size_t)(E + n_rows + 1) * 4 + 15) & ~(size_t)15));
    const int tid = threadIdx.x, nthr = blockDim.x;
    for (int k = tid; k < E; k += nthr) s_edge[k] = p.edges[k];
    for (int k = tid; k <= n_rows; k += nthr) s_row[k] = p.row_ptr[k];
    const int K = p.K_b * Z;
    const int nbytes = (K + 7) >> 3;
    const int rows_z = n_rows * Z;
    __syncthreads();

    for (int cw = blockIdx.x; cw < p.batch; cw += gridDim.x) {
        float *C = fp.ws + (size_t)cw * E * Z;
        for (int j = tid; j < N; j += nthr) L[j] = channel(p, cw, j);
        for (int k = tid; k < E * Z; k += nthr) C[k] = 0.0f;
        __syncthreads();
        int done = p.max_iter;
        for (int t = 1; t <= p.max_iter; ++t) {
            // check pass: every check row from the posteriors of the previous iteration
            for (int rr = tid; rr < rows_z; rr += nthr) {
                const int r = rr / Z, i = rr - r * Z;
                check_row(p, s_edge, s_row[r], s_row[r + 1] - s_row[r], i, L, C);
            }
            __syncthreads();
            // variable pass: L = L_b + sum of incoming messages in base-row order
            for (int j = tid; j < N; j += nthr) {
                const int c = j / Z, q = j - c * Z;
                float acc = channel(p, cw, j);
                for (int u = fp.col_ptr[c]; u < fp.col_ptr[c + 1]; ++u) {
                    const int e = fp.col_edge[u];
                    int i = q - (int)(s_edge[e] & 0xffffu);
                    if (i < 0) i += Z;
                    acc = __fadd_rn(acc, C[(size_t)e * Z + i]);
                }
                L[j] = acc;
            }
            __syncthreads();
            if (p.early_stop) {
                int bad = 0;
                for (int rr = tid; rr < rows_z && !bad; rr += nthr) {
                    const int r = rr / Z, i = rr - r * Z;
                    int par = 0;
                    for (int e = s_row[r]; e < s_row[r + 1]; ++e)
                        par ^= (L[fvar(s_edge[e], i, Z)] < 0.0f) ? 1 : 0;
                    bad = par;
                }
                if (__syncthreads_or(bad) == 0) {
                    done = t;
                    break;
                }
            }
        }
        for (int b = tid; b < nbytes; b += nthr) {
            unsigned x = 0;
            for (int k = 0; k < 8; ++k) {
                const int j = 8 * b + k;
                if (j < K && L[j] < 0.0f) x |= 1u << k;
            }
            p.bits[(size_t)cw * nbytes + b] = (uint8_t)x;
        }
        if (tid == 0) p.iters[cw] = done;
        if (p.post) {
            float *po = reinterpret_cast<float *>(p.post) + (size_t)cw * N;
            for (int j = tid; j < N; j += nthr) po[j] = L[j];
        }
        __syncthreads();
    }
}

size_t flood_smem(const DecodeParams &p) {
    size_t off = ((size_t)(p.E + p.n_rows + 1) * 4 + 15) & ~(size_t)15;
    return off + (size_t)p.n_cols * p.Z * 4;
}

}  // namespace

size_t flooding_ws_floats_per_cw(int E, int Z) { return (size_t)E * Z; }

ldpc_status launch_flooding(const DecodeParams &p, float *ws, cudaStream_t stream) {
    if (p.E > kMaxEdgesF || p.max_deg > kMaxDegF || p.n_cols > kMaxCols)
        return LDPC_ERR_UNSUPPORTED;
    static thread_local FloodParams fp;    // ~5 kB: kept off the stack
    fp.p = p;
    fp.ws = ws;
    // column edge lists in increasing edge order
    int fill[kMaxCols] = {};
    for (int c = 0; c <= p.n_cols; ++c) fp.col_ptr[c] = 0;
    for (int e = 0; e < p.E; ++e) ++fp.col_ptr[(p.h_edges[e] >> 16) + 1];
    for (int c = 0; c < p.n_cols; ++c) fp.col_ptr[c + 1] += fp.col_ptr[c];
    for (int e = 0; e < p.E; ++e) {
        const int c = (int)(p.h_edges[e] >> 16);
        fp.col_edge[fp.col_ptr[c] + fill[c]++] = e;
    }
    int dev = 0, optin = 0, n_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return LDPC_ERR_CUDA;
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    const size_t smem = flood_smem(p);
    if (smem > (size_t)optin) return LDPC_ERR_UNSUPPORTED;
    if (set_dyn_smem(reinterpret_cast<const void *>(flood_kernel), smem) != cudaSuccess)
        return LDPC_ERR_CUDA;
    const int threads = 256;
    int per_sm = 0;
    if (blocks_per_sm(&per_sm, reinterpret_cast<const void *>(flood_kernel), threads, smem) !=
            cudaSuccess ||
        per_sm < 1)
        return LDPC_ERR_UNSUPPORTED;
    int grid = n_sm * per_sm;
    if (grid > p.batch) grid = p.batch;
    flood_kernel<<<grid, threads, smem, stream>>>(fp);
    count_launch();
    if (cudaGetLastError() != cudaSuccess) return LDPC_ERR_CUDA;
    return LDPC_OK;
}

}  // namespace ldpc
