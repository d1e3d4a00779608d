// DecodeParams: everything a decode kernel needs, passed by value.  Device-side code only
// (no host headers), so that the runtime compiler of the per-graph batch kernel can take
// it as it is (pair_kernel.cuh).
#pragma once

#ifndef __CUDACC_RTC__
#include <cstddef>
#include <cstdint>
#endif

namespace ldpc {

// LDPC_ERR_TIMEOUT of ldpc.h, for kernels compiled without the public header (checked
// against it in decode_tmem_pair.cu)
constexpr int kStatusTimeout = 5;

struct DecodeParams {
    const uint32_t *edges;    // device [E]
    const int *row_ptr;       // device [n_rows + 1]
    const uint32_t *h_edges;  // host copies of the same tables
    const int *h_row_ptr;
    int n_rows, E, Z, n_cols, K_b;
    int max_deg;              // largest row degree among the used rows
    int punct, n_tx, max_iter, early_stop, batch;
    int algo;
    float alpha, offset;
    int offset_q;
    const float *learned;     // [max_iter][n_rows][2] or null
    const void *llr;          // [batch][n_tx]
    uint8_t *bits;            // [batch][ceil(K/8)]
    int32_t *iters;           // [batch]
    void *post;               // [batch][n_cols * Z] or null
    void *c2v;                // [batch][E * Z] or null
    int *status;              // device status word
    const int32_t *in_rows;   // [batch] LLR row of codeword b, or null (row b)
    const int32_t *out_rows;  // [batch] output row of codeword b, or null (row b)
    int threads_per_row;      // cooperating threads per row pair (0 = automatic)
    int cluster_size;         // 1, or 2: one codeword per cluster of two blocks
    int *queue;               // device [2] work counters of the launch's stream, or null
};

// source and destination rows of codeword b of a batch (identity without row maps)
__host__ __device__ __forceinline__ size_t in_row(const DecodeParams &p, int b) {
    return (size_t)(p.in_rows ? p.in_rows[b] : b);
}
__host__ __device__ __forceinline__ size_t out_row(const DecodeParams &p, int b) {
    return (size_t)(p.out_rows ? p.out_rows[b] : b);
}

// One codeword of a work list (device side; built by ldpc_decode_list).
struct ListItem {
    const uint32_t *edges;    // graph edge table
    const int *row_ptr;       // graph row pointers
    const int8_t *llr;        // [n_tx]
    uint8_t *bits;            // [ceil(K/8)]
    int32_t *iters;           // [1]
    int Z, K_b, n_rows, n_cols;
    int E, n_tx, punct, max_iter;
    int seq;                  // its row sequence in a compiled list kernel, or -1
};

}  // namespace ldpc
