// The binary16 decoder compiled at run time for a row sequence.  tmem16_kernel
// (t16_kernel.cuh) dispatches once per row on the row's degree; compiled with the sequence
// written out (LDPC_T16_ROWS) for the block shape of the launch (codewords per block,
// messages partly in shared memory or not), a layer is straight-line code.  The learned
// correction's (beta, gamma) table stays a run-time input, so one module serves every
// table, correction and lifting size with that degree sequence and shape.  Modules go
// through the registry of jit_common.cu (background compile by default, the generic kernel
// meanwhile); ldpc_pair_jit's mode applies.  The launch does not use it for the hybrid
// shape (decode_tmem16.cu says why).
#include <string>
#include <vector>

#include "ldpc_internal.h"

namespace ldpc {
namespace {

// Blocks of up to four rows repeated back to back (same degrees) become loops over their
// repetitions (one TMEM column per edge, so the degrees alone fix a row's code).
std::string t16_source(const std::vector<int> &deg, int cw, bool hybrid) {
    std::string s(jit_prelude());
    s += "#define LDPC_T16_CW " + std::to_string(cw) + "\n";
    s += std::string("#define LDPC_T16_HYB ") + (hybrid ? "true" : "false") + "\n";
    s += "#define LDPC_T16_ROWS";
    const int n = (int)deg.size();
    std::vector<int> e0(n + 1, 0);
    for (int r = 0; r < n; ++r) e0[r + 1] = e0[r] + deg[r];
    auto same = [&](int a, int b, int L) {
        for (int t = 0; t < L; ++t)
            if (a + t >= n || b + t >= n || deg[a + t] != deg[b + t]) return false;
        return true;
    };
    int r = 0;
    while (r < n) {
        int bestL = 0, bestK = 0, bestSave = 0;
        for (int L = 1; L <= 4 && r + 2 * L <= n; ++L) {
            int k = 1;
            while (r + (k + 1) * L <= n && same(r, r + k * L, L)) ++k;
            const int save = (k - 1) * (e0[r + L] - e0[r]);
            if (k >= 2 && save > bestSave) {
                bestL = L;
                bestK = k;
                bestSave = save;
            }
        }
        if (bestK >= 2) {
            const int S = e0[r + bestL] - e0[r];
            s += " _Pragma(\"unroll 1\") for (int u_ = 0; u_ < " + std::to_string(bestK) +
                 "; ++u_) {";
            for (int t = 0; t < bestL; ++t)
                s += " LDPC_T16Q(" + std::to_string(deg[r + t]) + ", (" +
                     std::to_string(e0[r + t]) + " + u_ * " + std::to_string(S) + "), (" +
                     std::to_string(r + t) + " + u_ * " + std::to_string(bestL) + "))";
            s += " }";
            r += bestL * bestK;
        } else {
            s += " LDPC_T16Q(" + std::to_string(deg[r]) + ", " + std::to_string(e0[r]) + ", " +
                 std::to_string(r) + ")";
            ++r;
        }
    }
    s += "\n#include \"t16_kernel.cuh\"\n";
    return s;
}

}  // namespace

const void *t16_jit_kernel(const DecodeParams &p, int cw, bool hybrid) {
    if (jit_mode() == 0) return nullptr;
    std::vector<int> deg((size_t)p.n_rows);
    std::string key = "t16:" + std::to_string(cw) + (hybrid ? "h:" : ":");
    for (int r = 0; r < p.n_rows; ++r) {
        deg[(size_t)r] = p.h_row_ptr[r + 1] - p.h_row_ptr[r];
        key += std::to_string(deg[(size_t)r]);
        key += ',';
    }
    return jit_kernel(key, [&deg, cw, hybrid] { return t16_source(deg, cw, hybrid); },
                      "ldpc_t16_rows.cu", "tmem16_kernel");
}

}  // namespace ldpc
