// Learned normalised-offset min-sum: forward with per-iteration checkpoints and the
// reverse-mode gradient through the unrolled layered decoder (sm_103a).
//
// The paper's min-sum check rule carries one correction factor beta (Sec. III).  The
// learned decoder gives every (iteration t, base row r) its own pair and applies
//     m' = beta[t][r] * max(m - gamma[t][r], 0)
// to the min-sum magnitudes, in IEEE binary32 with every operation rounded once (the same
// arithmetic as the fp32 decode path, so the forward pass is bit-identical to it).
//
// Forward (one thread block per codeword, one thread per check row, posteriors in shared
// memory, messages in the caller's workspace):  before iteration t it stores the
// posteriors as checkpoint P[t]; iteration t reads the messages C[t-1] (zero for t = 0) and
// writes C[t].  Workspace per codeword: P[T][N] | C[T][E*Z] | V[E*Z] | G[E*Z] floats.
//
// Backward: with gL = dLoss/dL (posteriors) and G = dLoss/dC (messages of the iteration
// being undone, zero after the last), for t = T-1 .. 0 the block restores P[t], replays the
// layers of iteration t storing every v = L - c_old in V, then undoes the layers in reverse:
//     for edge e of a row:   g_c = gL[var_e] + G[e]                  (total adjoint of c_new)
//                            c_new = s_e * beta * max(mag_e - gamma, 0)
//                            d beta  += g_c * s_e * max(mag_e - gamma, 0)
//                            d gamma += -g_c * s_e * beta * [mag_e > gamma]
//                            g_v[src_e] += g_c * s_e * beta * [mag_e > gamma] * sgn(v_src)
//     with src_e the edge attaining mag_e (the argmin for e != argmin, the second argmin
//     for e = argmin, lowest index on ties), signs held constant, g_v[e] += gL[var_e];
//     then gL[var_e] = g_v[e] and G[e] = -g_v[e].
// Parameter gradients are reduced deterministically per (codeword, t, r).
//
// Per-iteration outputs: the forward pass can also write the posteriors after every
// iteration (post_iter[t][cw]), and the backward pass then takes one adjoint per iteration
// (grad_post_iter[t][cw]); the adjoint of iteration t < T-1 is added to gL before the
// layers of iteration t are undone, so a loss over every iteration's posteriors
// back-propagates in one sweep.  With `detach` the adjoints are reset at every iteration
// boundary instead (gL = that iteration's own adjoint, G = 0): the parameters of iteration
// t then receive exactly the partial derivative of iteration t's own loss term, the only
// term whose inputs do not depend on them through earlier parameters (the full chain
// grows by orders of magnitude per iteration going backwards).
#include <cuda_fp16.h>

#include "ldpc_internal.h"

namespace ldpc {
namespace {

constexpr int kMaxDegL = 24;

struct LearnedParams {
    const uint32_t *edges;
    const int *row_ptr;
    int n_rows, E, Z, n_cols, punct, n_tx, T, batch;
    const float *params;     // [T][n_rows][2]
    const float *llr;        // [batch][n_tx]
    float *post;             // [batch][N]            (forward)
    const float *grad_post;  // [batch][N]            (backward)
    float *grad_params;      // [batch][T][n_rows][2] (backward)
    float *grad_llr;         // [batch][n_tx] or null (backward)
    float *post_iter;        // [T][batch][N] or null (forward)
    const float *grad_post_iter;  // [T][batch][N] or null (backward, replaces grad_post)
    int detach;              // backward: no adjoint flows between iterations
    float *ws;               // workspace
    size_t ws_per_cw;        // floats per codeword
};

__device__ __forceinline__ int lvar(uint32_t edge, int i, int Z) {
    int p = i + (int)(edge & 0xffffu);
    if (p >= Z) p -= Z;
    return (int)(edge >> 16) * Z + p;
}

// one layer of the forward pass for row i: reads c_old (null = zero), writes c_new and the
// posteriors; optionally stores every v in V
__device__ __forceinline__ void fwd_row(const LearnedParams &p, const uint32_t *s_edge, int e0,
                                        int d, int i, float beta, float gamma, float *L,
                                        const float *c_old, float *c_new, float *V) {
    const int Z = p.Z;
    float v[kMaxDegL];
    int vi[kMaxDegL];
    float m1 = __int_as_float(0x7f800000), m2 = m1;
    int idx = -1, S = 0;
#pragma unroll
    for (int k = 0; k < kMaxDegL; ++k) {
        if (k < d) {
            vi[k] = lvar(s_edge[e0 + k], i, Z);
            const float co = c_old ? c_old[(size_t)(e0 + k) * Z + i] : 0.0f;
            v[k] = __fsub_rn(L[vi[k]], co);
            if (V) V[(size_t)(e0 + k) * Z + i] = v[k];
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
#pragma unroll
    for (int k = 0; k < kMaxDegL; ++k) {
        if (k < d) {
            const float mag = (k == idx) ? m2 : m1;
            const float mc = __fmul_rn(beta, fmaxf(__fsub_rn(mag, gamma), 0.0f));
            const float cv = ((S ^ ((v[k] < 0.0f) ? 1 : 0)) != 0) ? -mc : mc;
            c_new[(size_t)(e0 + k) * Z + i] = cv;
            L[vi[k]] = __fadd_rn(v[k], cv);
        }
    }
}

__global__ void __launch_bounds__(512, 1) learned_fwd_kernel(LearnedParams p) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int Z = p.Z, E = p.E, n_rows = p.n_rows, N = p.n_cols * Z, EZ = E * Z;
    uint32_t *s_edge = reinterpret_cast<uint32_t *>(smem);
    int *s_row = reinterpret_cast<int *>(s_edge + E);
    float *L = reinterpret_cast<float *>(smem + (((size_t)(E + n_rows + 1) * 4 + 15) & ~(size_t)15));
    const int tid = threadIdx.x, nthr = blockDim.x;
    for (int k = tid; k < E; k += nthr) s_edge[k] = p.edges[k];
    for (int k = tid; k <= n_rows; k += nthr) s_row[k] = p.row_ptr[k];
    const int lo = p.punct * Z;
    for (int cw = blockIdx.x; cw < p.batch; cw += gridDim.x) {
        float *P = p.ws + (size_t)cw * p.ws_per_cw;
        float *C = P + (size_t)p.T * N;
        for (int j = tid; j < N; j += nthr) {
            const int t = j - lo;
            L[j] = (t >= 0 && t < p.n_tx) ? p.llr[(size_t)cw * p.n_tx + t] : 0.0f;
        }
        __syncthreads();
        for (int t = 0; t < p.T; ++t) {
            for (int j = tid; j < N; j += nthr) P[(size_t)t * N + j] = L[j];
            const float *c_old = t ? C + (size_t)(t - 1) * EZ : nullptr;
            float *c_new = C + (size_t)t * EZ;
            for (int r = 0; r < n_rows; ++r) {
                const int e0 = s_row[r], d = s_row[r + 1] - e0;
                const float beta = p.params[(t * n_rows + r) * 2 + 0];
                const float gamma = p.params[(t * n_rows + r) * 2 + 1];
                for (int i = tid; i < Z; i += nthr)
                    fwd_row(p, s_edge, e0, d, i, beta, gamma, L, c_old, c_new, nullptr);
                __syncthreads();
            }
            if (p.post_iter) {
                float *o = p.post_iter + ((size_t)t * p.batch + cw) * N;
                for (int j = tid; j < N; j += nthr) o[j] = L[j];
            }
        }
        if (p.post)
            for (int j = tid; j < N; j += nthr) p.post[(size_t)cw * N + j] = L[j];
        __syncthreads();
    }
}

// deterministic block sum of two values; result valid in thread 0
__device__ __forceinline__ float2 block_sum2(float a, float b, float2 *s_part) {
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) s_part[warp] = make_float2(a, b);
    __syncthreads();
    float2 r = make_float2(0.f, 0.f);
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            r.x += s_part[w].x;
            r.y += s_part[w].y;
        }
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(512, 1) learned_bwd_kernel(LearnedParams p) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ float2 s_part[32];
    const int Z = p.Z, E = p.E, n_rows = p.n_rows, N = p.n_cols * Z, EZ = E * Z;
    uint32_t *s_edge = reinterpret_cast<uint32_t *>(smem);
    int *s_row = reinterpret_cast<int *>(s_edge + E);
    float *L = reinterpret_cast<float *>(smem + (((size_t)(E + n_rows + 1) * 4 + 15) & ~(size_t)15));
    float *gL = L + N;
    const int tid = threadIdx.x, nthr = blockDim.x;
    for (int k = tid; k < E; k += nthr) s_edge[k] = p.edges[k];
    for (int k = tid; k <= n_rows; k += nthr) s_row[k] = p.row_ptr[k];
    for (int cw = blockIdx.x; cw < p.batch; cw += gridDim.x) {
        float *P = p.ws + (size_t)cw * p.ws_per_cw;
        float *C = P + (size_t)p.T * N;
        float *V = C + (size_t)p.T * EZ;
        float *G = V + EZ;
        const float *g_last =
            p.grad_post_iter ? p.grad_post_iter + ((size_t)(p.T - 1) * p.batch + cw) * N
                             : p.grad_post + (size_t)cw * N;
        for (int j = tid; j < N; j += nthr) gL[j] = g_last[j];
        for (int k = tid; k < EZ; k += nthr) G[k] = 0.0f;
        __syncthreads();
        for (int t = p.T - 1; t >= 0; --t) {
            // adjoint of this iteration's own output term; replay iteration t from its
            // checkpoint, keeping every v
            const float *g_t = (p.grad_post_iter && t < p.T - 1)
                                   ? p.grad_post_iter + ((size_t)t * p.batch + cw) * N
                                   : nullptr;
            const bool reset = p.detach && t < p.T - 1;
            for (int j = tid; j < N; j += nthr) {
                L[j] = P[(size_t)t * N + j];
                if (reset)
                    gL[j] = g_t ? g_t[j] : 0.0f;
                else if (g_t)
                    gL[j] += g_t[j];
            }
            if (reset)
                for (int k = tid; k < EZ; k += nthr) G[k] = 0.0f;
            __syncthreads();
            const float *c_old = t ? C + (size_t)(t - 1) * EZ : nullptr;
            for (int r = 0; r < n_rows; ++r) {
                const int e0 = s_row[r], d = s_row[r + 1] - e0;
                const float beta = p.params[(t * n_rows + r) * 2 + 0];
                const float gamma = p.params[(t * n_rows + r) * 2 + 1];
                // the replay rewrites C[t] with the values the forward pass stored there
                for (int i = tid; i < Z; i += nthr)
                    fwd_row(p, s_edge, e0, d, i, beta, gamma, L, c_old,
                            C + (size_t)t * EZ, V);
                __syncthreads();
            }
            // undo the layers of iteration t, last first
            for (int r = n_rows - 1; r >= 0; --r) {
                const int e0 = s_row[r], d = s_row[r + 1] - e0;
                const float beta = p.params[(t * n_rows + r) * 2 + 0];
                const float gamma = p.params[(t * n_rows + r) * 2 + 1];
                float gb = 0.f, gg = 0.f;
                for (int i = tid; i < Z; i += nthr) {
                    float v[kMaxDegL], gv[kMaxDegL];
                    int vi[kMaxDegL];
                    float m1 = __int_as_float(0x7f800000), m2 = m1;
                    int idx = -1, idx2 = -1, S = 0;
#pragma unroll
                    for (int k = 0; k < kMaxDegL; ++k) {
                        if (k < d) {
                            v[k] = V[(size_t)(e0 + k) * Z + i];
                            vi[k] = lvar(s_edge[e0 + k], i, Z);
                            gv[k] = gL[vi[k]];
                            const float a = fabsf(v[k]);
                            if (a < m1) {
                                m2 = m1;
                                idx2 = idx;
                                m1 = a;
                                idx = k;
                            } else if (a < m2) {
                                m2 = a;
                                idx2 = k;
                            }
                            S ^= (v[k] < 0.0f) ? 1 : 0;
                        }
                    }
#pragma unroll
                    for (int k = 0; k < kMaxDegL; ++k) {
                        if (k < d) {
                            const float s = ((S ^ ((v[k] < 0.0f) ? 1 : 0)) != 0) ? -1.0f : 1.0f;
                            const float mag = (k == idx) ? m2 : m1;
                            const float gcn = gL[vi[k]] + G[(size_t)(e0 + k) * Z + i];
                            const float rel = mag - gamma;
                            const float act = rel > 0.0f ? 1.0f : 0.0f;
                            gb += gcn * s * (rel > 0.0f ? rel : 0.0f);
                            gg -= gcn * s * beta * act;
                            const float gmag = gcn * s * beta * act;
                            const int src = (k == idx) ? idx2 : idx;
#pragma unroll
                            for (int q = 0; q < kMaxDegL; ++q)
                                if (q < d && q == src) gv[q] += gmag * (v[q] < 0.0f ? -1.0f : 1.0f);
                        }
                    }
#pragma unroll
                    for (int k = 0; k < kMaxDegL; ++k) {
                        if (k < d) {
                            gL[vi[k]] = gv[k];
                            G[(size_t)(e0 + k) * Z + i] = -gv[k];
                        }
                    }
                }
                const float2 sums = block_sum2(gb, gg, s_part);
                if (tid == 0) {
                    float *o = p.grad_params + (((size_t)cw * p.T + t) * n_rows + r) * 2;
                    o[0] = sums.x;
                    o[1] = sums.y;
                }
                __syncthreads();
            }
        }
        if (p.grad_llr)
            for (int j = tid; j < p.n_tx; j += nthr)
                p.grad_llr[(size_t)cw * p.n_tx + j] = gL[p.punct * Z + j];
        __syncthreads();
    }
}

}  // namespace

size_t learned_ws_floats_per_cw(int N, int EZ, int T) {
    return (size_t)T * N + (size_t)T * EZ + 2 * (size_t)EZ;
}

ldpc_status launch_learned(const DecodeParams &dp, int T, const float *params, const float *llr,
                           float *post, const float *grad_post, float *grad_params,
                           float *grad_llr, float *ws, bool backward, cudaStream_t stream,
                           float *post_iter, const float *grad_post_iter, int detach) {
    LearnedParams p;
    p.post_iter = post_iter;
    p.grad_post_iter = grad_post_iter;
    p.detach = detach;
    p.edges = dp.edges;
    p.row_ptr = dp.row_ptr;
    p.n_rows = dp.n_rows;
    p.E = dp.E;
    p.Z = dp.Z;
    p.n_cols = dp.n_cols;
    p.punct = dp.punct;
    p.n_tx = dp.n_tx;
    p.T = T;
    p.batch = dp.batch;
    p.params = params;
    p.llr = llr;
    p.post = post;
    p.grad_post = grad_post;
    p.grad_params = grad_params;
    p.grad_llr = grad_llr;
    p.ws = ws;
    const int N = dp.n_cols * dp.Z;
    p.ws_per_cw = learned_ws_floats_per_cw(N, dp.E * dp.Z, T);
    if (dp.max_deg > kMaxDegL) return LDPC_ERR_UNSUPPORTED;
    const size_t smem = (((size_t)(dp.E + dp.n_rows + 1) * 4 + 15) & ~(size_t)15) +
                        (size_t)N * 4 * (backward ? 2 : 1);
    int dev = 0, n_sm = 0, optin = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return LDPC_ERR_CUDA;
    cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (smem > (size_t)optin) return LDPC_ERR_UNSUPPORTED;
    auto kern = backward ? learned_bwd_kernel : learned_fwd_kernel;
    if (set_dyn_smem(reinterpret_cast<const void *>(kern), smem) !=
        cudaSuccess)
        return LDPC_ERR_CUDA;
    int threads = ((dp.Z + 31) / 32) * 32;
    if (threads > 512) threads = 512;      // rows beyond the block loop
    int per_sm = 0;
    if (blocks_per_sm(&per_sm, reinterpret_cast<const void *>(kern), threads, smem) !=
            cudaSuccess ||
        per_sm < 1)
        return LDPC_ERR_UNSUPPORTED;
    int grid = n_sm * per_sm;
    if (grid > dp.batch) grid = dp.batch;
    kern<<<grid, threads, smem, stream>>>(p);
    count_launch();
    if (cudaGetLastError() != cudaSuccess) return LDPC_ERR_CUDA;
    return LDPC_OK;
}

}  // namespace ldpc
