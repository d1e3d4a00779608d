// Self-test of the bounded device waits (failure handling without a GPU fault).
//
// The decode kernels wait on shared-memory barriers for their channel-LLR bulk copies; every
// such wait polls at most a fixed number of times and, when it gives up, records
// LDPC_ERR_TIMEOUT in the graph's status word and lets the kernel return.  This kernel
// exercises that path on purpose: it arms a barrier for a transfer that is never issued, so
// the wait must run out, and reports what the wait returned.  Nothing is left in flight (no
// copy was started), so the context stays usable.
#include "ldpc_internal.h"
#include "tmem.h"

namespace ldpc {
namespace {

__global__ void wait_timeout_kernel(uint32_t limit, int *status, unsigned long long *cycles) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x != 0) return;
    tm::mbar_init(&bar);
    // expect 16 bytes that no copy will deliver: phase 0 never completes
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(
                     tm::smem_addr(&bar)),
                 "r"(16u)
                 : "memory");
    const unsigned long long t0 = clock64();
    const bool ok = tm::mbar_wait(&bar, 0u, limit);
    *cycles = clock64() - t0;
    *status = ok ? (int)LDPC_OK : (int)LDPC_ERR_TIMEOUT;
}

}  // namespace
}  // namespace ldpc

extern "C" ldpc_status ldpc_selftest_wait_timeout(unsigned int spin_limit, ldpc_stream_t stream,
                                                  unsigned long long *cycles_out) {
    if (spin_limit == 0 || spin_limit > ldpc::tm::kSpinLimit) return LDPC_ERR_INVALID_ARG;
    int *d_status = nullptr;
    unsigned long long *d_cycles = nullptr;
    if (ldpc::dev_alloc((void **)&d_status, sizeof(int)) != cudaSuccess) return LDPC_ERR_OUT_OF_MEMORY;
    if (ldpc::dev_alloc((void **)&d_cycles, sizeof(unsigned long long)) != cudaSuccess) {
        cudaFree(d_status);
        return LDPC_ERR_OUT_OF_MEMORY;
    }
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    ldpc::wait_timeout_kernel<<<1, 32, 0, s>>>(spin_limit, d_status, d_cycles);
    ldpc::count_launch();
    int status = (int)LDPC_ERR_CUDA;
    unsigned long long cycles = 0;
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpyAsync(&status, d_status, sizeof(int), cudaMemcpyDeviceToHost, s) !=
            cudaSuccess ||
        cudaMemcpyAsync(&cycles, d_cycles, sizeof(cycles), cudaMemcpyDeviceToHost, s) !=
            cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        status = (int)LDPC_ERR_CUDA;
    cudaFree(d_status);
    cudaFree(d_cycles);
    if (cycles_out) *cycles_out = cycles;
    return (ldpc_status)status;
}
