// Layered min-sum decoder kernels for sm_103a.
//
// Method (paper Sec. III, Sec. IV): for every iteration, base rows ("layers") are processed
// one after another; within a layer the Z check rows are independent.  For check row i of
// layer r and each of its d_r circulants (column c, shift s) the decoder
//   a1 gathers the posterior L_v at c*Z + ((i + s) mod Z),
//   a2 forms the variable-to-check message v = L_v - c2v_old,
//   a3 reduces m1 = min|v|, idx = argmin (lowest edge index on ties), m2 = min over the
//      other edges, S = parity of the negative messages, and corrects the magnitudes,
//   a4 writes c2v_new = (S xor sgn v) * (edge == idx ? m2' : m1') and L_v = v + c2v_new,
// and after a full iteration
//   a5 tests the syndrome of the hard decisions (bit = L_v < 0) for early stop.
//
// Mapping: one thread block decodes one codeword at a time (persistent grid-stride loop
// over the batch); the codeword's posteriors and every check-to-variable message stay in
// shared memory for the whole decode; thread i owns check row i of every layer.  Layers
// are separated by a block barrier.  Within a layer each variable is touched by at most
// one (row, edge) pair — a layer has at most one circulant per column block and a
// circulant is a bijection — so pass 1 stores v in place of L_v and pass 2 rereads it.
#include <cuda_fp16.h>

#include "ldpc_internal.h"

namespace ldpc {
namespace {

// ------------------------------------------------------------------ arithmetic policies

// 8-bit fixed point: L_v, v and c2v saturate to [-127, 127]; offset correction.
struct ArithI8 {
    using T = int8_t;
    using A = int;
    static __device__ __forceinline__ A load(T x) { return x; }
    static __device__ __forceinline__ T store(A x) { return (T)x; }
    static __device__ __forceinline__ A sat(A x) { return max(-127, min(127, x)); }
    static __device__ __forceinline__ A sub(A a, A b) { return sat(a - b); }
    static __device__ __forceinline__ A add(A a, A b) { return sat(a + b); }
    static __device__ __forceinline__ A absv(A a) { return a < 0 ? -a : a; }
    static __device__ __forceinline__ bool neg(A a) { return a < 0; }
    static __device__ __forceinline__ A big() { return 1 << 20; }
    static __device__ __forceinline__ A corr(const DecodeParams &p, A m, float, float) {
        return max(m - p.offset_q, 0);
    }
    static __device__ __forceinline__ A negate(A a) { return -a; }
    static __device__ __forceinline__ A from_llr(const void *llr, size_t k) {
        return ((const int8_t *)llr)[k];
    }
    static __device__ __forceinline__ A zero() { return 0; }
};

// IEEE binary32 with every operation rounded once (no contraction).
struct ArithF32 {
    using T = float;
    using A = float;
    static __device__ __forceinline__ A load(T x) { return x; }
    static __device__ __forceinline__ T store(A x) { return x; }
    static __device__ __forceinline__ A sub(A a, A b) { return __fsub_rn(a, b); }
    static __device__ __forceinline__ A add(A a, A b) { return __fadd_rn(a, b); }
    static __device__ __forceinline__ A absv(A a) { return fabsf(a); }
    static __device__ __forceinline__ bool neg(A a) { return a < 0.0f; }
    static __device__ __forceinline__ A big() { return __int_as_float(0x7f800000); }
    static __device__ __forceinline__ A corr(const DecodeParams &p, A m, float beta,
                                             float gamma) {
        if (p.algo == LDPC_NORMALISED) return __fmul_rn(p.alpha, m);
        if (p.algo == LDPC_OFFSET) return fmaxf(__fsub_rn(m, p.offset), 0.0f);
        return __fmul_rn(beta, fmaxf(__fsub_rn(m, gamma), 0.0f));
    }
    static __device__ __forceinline__ A negate(A a) { return -a; }
    static __device__ __forceinline__ A from_llr(const void *llr, size_t k) {
        return ((const float *)llr)[k];
    }
    static __device__ __forceinline__ A zero() { return 0.0f; }
};

// IEEE binary16 storage and arithmetic: every result rounded to binary16 (to nearest even).
struct ArithF16 {
    using T = __half;
    using A = __half;
    static __device__ __forceinline__ A load(T x) { return x; }
    static __device__ __forceinline__ T store(A x) { return x; }
    static __device__ __forceinline__ A sub(A a, A b) { return __hsub(a, b); }
    static __device__ __forceinline__ A add(A a, A b) { return __hadd(a, b); }
    static __device__ __forceinline__ A absv(A a) { return __habs(a); }
    static __device__ __forceinline__ bool neg(A a) { return __hlt(a, __ushort_as_half(0)); }
    static __device__ __forceinline__ A big() { return __ushort_as_half(0x7c00); }
    static __device__ __forceinline__ A corr(const DecodeParams &p, A m, float beta,
                                             float gamma) {
        const A zero = __ushort_as_half(0);
        if (p.algo == LDPC_NORMALISED) return __hmul(__float2half_rn(p.alpha), m);
        if (p.algo == LDPC_OFFSET) return __hmax(__hsub(m, __float2half_rn(p.offset)), zero);
        return __hmul(__float2half_rn(beta), __hmax(__hsub(m, __float2half_rn(gamma)), zero));
    }
    static __device__ __forceinline__ A negate(A a) { return __hneg(a); }
    static __device__ __forceinline__ A from_llr(const void *llr, size_t k) {
        return ((const __half *)llr)[k];
    }
    static __device__ __forceinline__ A zero() { return __ushort_as_half(0); }
};

template <class Ar>
__device__ __forceinline__ bool less_than(typename Ar::A a, typename Ar::A b) {
    return a < b;
}
template <>
__device__ __forceinline__ bool less_than<ArithF16>(__half a, __half b) {
    return __hlt(a, b);
}

__device__ __forceinline__ int var_index(uint32_t edge, int i, int Z) {
    int p = i + (int)(edge & 0xffffu);
    if (p >= Z) p -= Z;
    return (int)(edge >> 16) * Z + p;
}

// --------------------------------------------------------------------------- the kernel

template <class Ar>
__global__ void __launch_bounds__(1024, 1) layered_kernel(DecodeParams p) {
    using T = typename Ar::T;
    using A = typename Ar::A;
    extern __shared__ __align__(16) unsigned char smem[];
    const int Z = p.Z, E = p.E, n_rows = p.n_rows;
    const int N = p.n_cols * Z;
    uint32_t *s_edge = reinterpret_cast<uint32_t *>(smem);
    int *s_row = reinterpret_cast<int *>(s_edge + E);
    size_t off = (size_t)(E + n_rows + 1) * 4;
    off = (off + 15) & ~(size_t)15;
    T *s_Lv = reinterpret_cast<T *>(smem + off);
    off += (size_t)N * sizeof(T);
    off = (off + 15) & ~(size_t)15;
    T *s_c2v = reinterpret_cast<T *>(smem + off);

    const int tid = threadIdx.x, nthr = blockDim.x;
    for (int k = tid; k < E; k += nthr) s_edge[k] = p.edges[k];
    for (int k = tid; k <= n_rows; k += nthr) s_row[k] = p.row_ptr[k];
    const int K = p.K_b * Z;
    const int nbytes = (K + 7) >> 3;
    const int lo = p.punct * Z, hi = lo + p.n_tx;

    for (int cw = blockIdx.x; cw < p.batch; cw += gridDim.x) {
        // a0: posteriors from the channel LLRs, zero messages
        const size_t base = in_row(p, cw) * p.n_tx;
        for (int j = tid; j < N; j += nthr)
            s_Lv[j] = Ar::store((j >= lo && j < hi) ? Ar::from_llr(p.llr, base + (j - lo))
                                                     : Ar::zero());
        for (int k = tid; k < E * Z; k += nthr) s_c2v[k] = Ar::store(Ar::zero());
        __syncthreads();

        int done = p.max_iter;
        for (int t = 1; t <= p.max_iter; ++t) {
            for (int r = 0; r < n_rows; ++r) {
                const int e0 = s_row[r], e1 = s_row[r + 1];
                float beta = 0.f, gamma = 0.f;
                if (p.algo == LDPC_LEARNED) {
                    beta = p.learned[((t - 1) * n_rows + r) * 2 + 0];
                    gamma = p.learned[((t - 1) * n_rows + r) * 2 + 1];
                }
                for (int i = tid; i < Z; i += nthr) {
                    // a1 + a2 + a3: gather, v = L_v - c2v_old, running min1/min2/argmin/sign
                    A m1 = Ar::big(), m2 = Ar::big();
                    int idx = -1, S = 0;
                    for (int e = e0; e < e1; ++e) {
                        const int vi = var_index(s_edge[e], i, Z);
                        const A v = Ar::sub(Ar::load(s_Lv[vi]), Ar::load(s_c2v[e * Z + i]));
                        s_Lv[vi] = Ar::store(v);
                        const A a = Ar::absv(v);
                        if (less_than<Ar>(a, m1)) {
                            m2 = m1;
                            m1 = a;
                            idx = e;
                        } else if (less_than<Ar>(a, m2)) {
                            m2 = a;
                        }
                        S ^= (int)Ar::neg(v);
                    }
                    const A m1c = Ar::corr(p, m1, beta, gamma);
                    const A m2c = Ar::corr(p, m2, beta, gamma);
                    // a4: new messages and posterior write-back
                    for (int e = e0; e < e1; ++e) {
                        const int vi = var_index(s_edge[e], i, Z);
                        const A v = Ar::load(s_Lv[vi]);
                        const A mag = (e == idx) ? m2c : m1c;
                        const A c = (S ^ (int)Ar::neg(v)) ? Ar::negate(mag) : mag;
                        s_c2v[e * Z + i] = Ar::store(c);
                        s_Lv[vi] = Ar::store(Ar::add(v, c));
                    }
                }
                __syncthreads();
            }
            // a5: syndrome of the hard decisions after a full iteration
            if (p.early_stop) {
                int bad = 0;
                for (int i = tid; i < Z && !bad; i += nthr)
                    for (int r = 0; r < n_rows && !bad; ++r) {
                        int par = 0;
                        for (int e = s_row[r]; e < s_row[r + 1]; ++e)
                            par ^= (int)Ar::neg(Ar::load(s_Lv[var_index(s_edge[e], i, Z)]));
                        bad = par;
                    }
                if (__syncthreads_or(bad) == 0) {
                    done = t;
                    break;
                }
            }
        }

        // a6: outputs
        for (int b = tid; b < nbytes; b += nthr) {
            unsigned x = 0;
            for (int k = 0; k < 8; ++k) {
                const int j = 8 * b + k;
                if (j < K && Ar::neg(Ar::load(s_Lv[j]))) x |= 1u << k;
            }
            p.bits[out_row(p, cw) * nbytes + b] = (uint8_t)x;
        }
        if (tid == 0) p.iters[out_row(p, cw)] = done;
        if (p.post) {
            T *po = reinterpret_cast<T *>(p.post) + (size_t)cw * N;
            for (int j = tid; j < N; j += nthr) po[j] = s_Lv[j];
        }
        if (p.c2v) {
            T *co = reinterpret_cast<T *>(p.c2v) + (size_t)cw * E * Z;
            for (int k = tid; k < E * Z; k += nthr) co[k] = s_c2v[k];
        }
        __syncthreads();
    }
}

template <class Ar>
ldpc_status launch_t(const DecodeParams &p, cudaStream_t stream) {
    using T = typename Ar::T;
    const int N = p.n_cols * p.Z;
    size_t smem = (size_t)(p.E + p.n_rows + 1) * 4;
    smem = (smem + 15) & ~(size_t)15;
    smem += (size_t)N * sizeof(T);
    smem = (smem + 15) & ~(size_t)15;
    smem += (size_t)p.E * p.Z * sizeof(T);
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return LDPC_ERR_CUDA;
    int smem_optin = 0, n_sm = 0;
    cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    if (smem > (size_t)smem_optin) return LDPC_ERR_UNSUPPORTED;
    if (set_dyn_smem(reinterpret_cast<const void *>(layered_kernel<Ar>), smem) != cudaSuccess)
        return LDPC_ERR_CUDA;
    int threads = ((p.Z + 31) / 32) * 32;
    if (threads > 1024) threads = 1024;
    int per_sm = 0;
    if (blocks_per_sm(&per_sm, reinterpret_cast<const void *>(layered_kernel<Ar>), threads,
                      smem) != cudaSuccess ||
        per_sm < 1)
        return LDPC_ERR_UNSUPPORTED;
    int grid = n_sm * per_sm;
    if (grid > p.batch) grid = p.batch;
    layered_kernel<Ar><<<grid, threads, smem, stream>>>(p);
    count_launch();
    if (cudaGetLastError() != cudaSuccess) return LDPC_ERR_CUDA;
    return LDPC_OK;
}

}  // namespace

ldpc_status launch_layered(const DecodeParams &p, int llr_type, cudaStream_t stream) {
    int dev = 0, smem_optin = 0, n_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return LDPC_ERR_CUDA;
    cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    // a cluster of two blocks per codeword when asked for
    if (p.cluster_size == 2) {
        if (!cluster_supported(p, llr_type, p.max_deg, (size_t)smem_optin))
            return LDPC_ERR_UNSUPPORTED;
        return launch_cluster(p, stream);
    }
    // the low-latency strategy (alpha cooperating threads per row pair, one codeword per
    // block) when asked for, or by default when the batch does not fill the SMs.  Compiled
    // for the row sequence it is the fastest for such batches (a lone BG1-shaped Z=384
    // codeword, 10 iterations: 157 us at alpha 2 against 181 us for the compiled batch
    // kernel); while only the batch kernel's compiled form is ready, that one is used
    // instead (the generic alpha-2 kernel takes 230 us)
    int A = p.threads_per_row;
    if (A == 0) {
        A = 1;
        if (p.batch <= n_sm &&
            tmem_ll_supported(p, llr_type, p.max_deg, 2, (size_t)smem_optin)) {
            const bool pair_ok = pair_supported(p, llr_type, p.max_deg, (size_t)smem_optin);
            const bool ll_ready = ll_jit_kernel(p, 2) != nullptr;
            A = (ll_ready || !(pair_ok && pair_jit_kernel(p))) ? 2 : 1;
        }
    }
    if (A > 1) {
        if (!tmem_ll_supported(p, llr_type, p.max_deg, A, (size_t)smem_optin))
            return LDPC_ERR_UNSUPPORTED;
        return launch_tmem_ll(p, A, stream);
    }
    if (pair_supported(p, llr_type, p.max_deg, (size_t)smem_optin))
        return launch_pair(p, stream);
    if (!p.in_rows && !p.out_rows && rowpair_supported(p, llr_type, p.max_deg, (size_t)smem_optin))
        return launch_rowpair(p, p.max_deg, stream);
    if (tmem16_supported(p, llr_type, p.max_deg, (size_t)smem_optin))
        return launch_tmem16(p, stream);
    switch (llr_type) {
    case LDPC_LLR_INT8:
        return launch_t<ArithI8>(p, stream);
    case LDPC_LLR_FP16:
        return launch_t<ArithF16>(p, stream);
    case LDPC_LLR_FP32:
        return launch_t<ArithF32>(p, stream);
    default:
        return LDPC_ERR_INVALID_ARG;
    }
}

}  // namespace ldpc
