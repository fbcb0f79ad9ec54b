// Self-test of the bounded device waits: a kernel whose wait can never be
// satisfied gives up after a time limit and reports it through a status
// word, the way the library's waiting kernels do (the SetEq look-back, the
// FRI copy pipeline).  No fault, trap or unbounded loop is involved.
#include <cuda_runtime.h>

#include "../../include/v3c.h"
#include "ctx.h"
#include "gl.cuh"
#include "internal.h"
#include "mbar.cuh"

namespace v3c {

// One thread.  kind 0: an mbarrier phase that expects two arrivals and gets
// one; kind 1: a device word that nothing sets, polled with short sleeps.
// *status = 1 when the wait gave up after limit_ns, 0 if it was satisfied.
__global__ void k_wait_selftest(u32 kind, u64 limit_ns, const u32* flag, u32* status)
{
    __shared__ u64 bar;
    if (threadIdx.x != 0) return;
    bool ok = false;
    if (kind == 0) {
        mbar_init(&bar, 2);
        mbar_init_fence();
        mbar_arrive(&bar);
        ok = mbar_wait(&bar, 0, limit_ns);
    } else {
        const u64 t0 = global_timer_ns();
        for (;;) {
            if (*(volatile const u32*)flag) {
                ok = true;
                break;
            }
            if (global_timer_ns() - t0 > limit_ns) break;
            __nanosleep(256);
        }
    }
    *status = ok ? 0u : 1u;
}

}  // namespace v3c

using namespace v3c::detail;

extern "C" v3c_status v3c_wait_selftest(v3c_ctx* ctx, uint32_t kind, uint32_t limit_us, void* stream)
{
    if (!ctx) return V3C_EINVAL;
    if (kind > 1 || limit_us == 0 || limit_us > 2000000)
        return fail(ctx, V3C_EINVAL, "v3c_wait_selftest: kind %u, limit %u us", kind, limit_us);
    v3c_status r = use_device(ctx);
    if (r) return r;
    cudaStream_t s = (cudaStream_t)stream;
    std::lock_guard<std::mutex> g(ctx->mu);
    v3c::u32* d = nullptr;
    CK(cudaMallocAsync((void**)&d, 8, s));
    v3c::u32 st = 0;
    cudaError_t e = cudaMemsetAsync(d, 0, 8, s);
    if (e == cudaSuccess) {
        v3c::k_wait_selftest<<<1, 32, 0, s>>>(kind, (v3c::u64)limit_us * 1000, d, d + 1);
        e = cudaGetLastError();
        ctx->launches++;
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&st, d + 1, 4, cudaMemcpyDeviceToHost, s);
    cudaFreeAsync(d, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail(ctx, V3C_ECUDA, "v3c_wait_selftest: %s", cudaGetErrorString(e));
    if (st) return fail(ctx, V3C_ETIMEDOUT, "v3c_wait_selftest: the wait gave up after %u us", limit_us);
    return V3C_OK;
}
