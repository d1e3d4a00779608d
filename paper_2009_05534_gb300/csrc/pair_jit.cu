// Per-graph batch kernels compiled at run time.  The batch kernel (pair_kernel.cuh) walks
// the layers of an iteration with one indirect branch per row on the row's degree and the
// parity of its first edge; compiled with the graph's row sequence written out
// (LDPC_PAIR_ROWS), the same kernel runs the layers as straight-line code (measured 19 %
// less time per headline launch, bit-identical results).  The row sequence depends only on
// the degrees of the rows a decode uses, so one module serves every graph and lifting size
// with that degree sequence: the shifts and columns stay in the kernel's parameter table.
//
// Modules are built with NVRTC from the kernel headers embedded at build time and kept in
// the registry of jit_common.cu: compiling takes a few seconds of host time, so by default
// it runs on a background thread and the generic kernel serves the degree sequence until
// the module is ready; in the blocking mode the launch that meets a new sequence compiles
// and loads it itself.  A compile or load that fails leaves the sequence on the generic
// kernel.
#include <string>
#include <vector>

#include "f16x2.h"
#include "ldpc_internal.h"

namespace ldpc {
namespace {

// The source of one module: the prelude, the row sequence and the kernel header.  A block
// of up to 4 rows repeated back to back (same degrees, same first-edge parities) becomes a
// loop over its repetitions, the block that saves the most edges of code first: the
// straight-line layer loop is about 22 instructions per edge, its instruction fetch grows
// with its length, and the loops shorten it by a quarter on the BG1-shaped table (3 % less
// time per headline launch, measured).
std::string module_source(const std::vector<int> &deg) {
    std::string s(jit_prelude());
    s += "#define LDPC_PAIR_ROWS";
    const int n = (int)deg.size();
    std::vector<int> e0s(n + 1, 0);
    for (int r = 0; r < n; ++r) e0s[r + 1] = e0s[r] + deg[r];
    auto same = [&](int a, int b, int L) {
        for (int t = 0; t < L; ++t)
            if (a + t >= n || b + t >= n || deg[a + t] != deg[b + t] ||
                ((e0s[a + t] ^ e0s[b + t]) & 1))
                return false;
        return true;
    };
    int r = 0;
    while (r < n) {
        int bestL = 0, bestK = 0, bestSave = 0;
        for (int L = 1; L <= 4 && r + 2 * L <= n; ++L) {
            int k = 1;
            while (r + (k + 1) * L <= n && same(r, r + k * L, L)) ++k;
            const int save = (k - 1) * (e0s[r + L] - e0s[r]);
            if (k >= 2 && save > bestSave) {
                bestL = L;
                bestK = k;
                bestSave = save;
            }
        }
        if (bestK >= 2) {
            const int S = e0s[r + bestL] - e0s[r];
            s += " _Pragma(\"unroll 1\") for (int u_ = 0; u_ < " + std::to_string(bestK) +
                 "; ++u_) {";
            for (int t = 0; t < bestL; ++t)
                s += " LDPC_PQ(" + std::to_string(deg[r + t]) + ", " +
                     std::to_string(e0s[r + t] & 1) + ", (" + std::to_string(e0s[r + t]) +
                     " + u_ * " + std::to_string(S) + "))";
            s += " }";
            r += bestL * bestK;
        } else {
            s += " LDPC_PQ(" + std::to_string(deg[r]) + ", " + std::to_string(e0s[r] & 1) +
                 ", " + std::to_string(e0s[r]) + ")";
            ++r;
        }
    }
    s += "\n#include \"pair_kernel.cuh\"\n";
    return s;
}

std::string degree_key(const std::vector<int> &deg) {
    std::string key = "pair:";
    for (const int d : deg) {
        key += std::to_string(d);
        key += ',';
    }
    return key;
}

}  // namespace

const void *pair_jit_kernel(const DecodeParams &p) {
    if (jit_mode() == 0) return nullptr;
    std::vector<int> deg((size_t)p.n_rows);
    for (int r = 0; r < p.n_rows; ++r) deg[(size_t)r] = p.h_row_ptr[r + 1] - p.h_row_ptr[r];
    return jit_kernel(degree_key(deg), [&deg] { return module_source(deg); },
                      "ldpc_pair_rows.cu", "pair_kernel");
}

}  // namespace ldpc

extern "C" int ldpc_pair_jit(int mode) { return ldpc::jit_set_mode(mode); }

extern "C" ldpc_status ldpc_pair_jit_prepare(const int *row_degrees, int n_rows) {
    if (!row_degrees || n_rows < 1 || n_rows > ldpc::kMaxRows) return LDPC_ERR_INVALID_ARG;
    std::vector<int> deg((size_t)n_rows);
    int E = 0;
    for (int r = 0; r < n_rows; ++r) {
        deg[(size_t)r] = row_degrees[r];
        if (row_degrees[r] < 2 || row_degrees[r] > ldpc::h2::kMaxDeg)
            return LDPC_ERR_INVALID_ARG;
        E += row_degrees[r];
    }
    if (E > ldpc::kMaxEdges) return LDPC_ERR_INVALID_ARG;
    // the batch kernel and the low-latency kernel at both alphas
    const bool ok = ldpc::jit_prepare(ldpc::degree_key(deg),
                                      [&deg] { return ldpc::module_source(deg); },
                                      "ldpc_pair_rows.cu");
    const bool ok2 = ldpc::ll_jit_prepare(deg, 2);
    const bool ok4 = ldpc::ll_jit_prepare(deg, 4);
    return ok && ok2 && ok4 ? LDPC_OK : LDPC_ERR_UNSUPPORTED;
}
