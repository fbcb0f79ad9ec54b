// v3c_lde_noalloc: the coset LDE with its scratch in a fixed device array.
//
// Some callers cannot allocate device memory.  One example is a host process
// that runs next to an inference server whose caching allocator has already
// reserved the GPU's HBM.  Another is a latency-critical audit path that
// must not take the device-wide synchronisation a cudaMalloc/cudaFree may
// imply.  For them this entry point runs the same three LDE stages as
// v3c_lde without any allocation.  The work space lives in the file-scope
// array below, which every GPU that loads the library holds until the
// process exits.  It holds:
//   words [0, 64)          the job descriptor and the stage item lists,
//   words [64, 64 + T)     the twiddle and coset tables of the shape,
//   then Y (c*n words) and Z (c*N words) when the shape needs them.
// Everything in it is written before it is read on every call, so nothing
// has to start at zero.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <mutex>

#include "../../include/v3c.h"
#include "gl.cuh"
#include "internal.h"

namespace v3c {
namespace {

constexpr size_t kHeaderWords = 64;

static __device__ __align__(256) u64 g_noalloc_scratch[V3C_NOALLOC_SCRATCH_BYTES / 8];

// Device address of g_noalloc_scratch per device.  In host code the array's
// name is only a host-side stand-in, so it is looked up once per device with
// that device current.  The modules of this library load lazily: the first
// lookup on a device loads this file's module and so reserves the array
// there.  The cached address belongs to the device's primary context and
// goes stale after cudaDeviceReset.
constexpr int kMaxDevices = 64;
std::mutex g_mu;
u64* g_addr[kMaxDevices] = {nullptr};

v3c_status scratch_address(int dev, u64** out)
{
    if (dev < 0 || dev >= kMaxDevices) return V3C_EINVAL;
    std::lock_guard<std::mutex> g(g_mu);
    if (!g_addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            // Loading the module reserves the array; with the HBM already
            // taken by another allocator that reservation is what fails.
            return e == cudaErrorMemoryAllocation ? V3C_ENOMEM : V3C_ECUDA;
        }
        g_addr[dev] = (u64*)p;
    }
    *out = g_addr[dev];
    return V3C_OK;
}

// Writes the job descriptor and the item lists of stages A, B, C.
__global__ void k_noalloc_header(LdeJob job, u32 na, u32 nb, u32 nc, u64* dst)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    *reinterpret_cast<LdeJob*>(dst) = job;
    u32* lists = reinterpret_cast<u32*>(dst + 32);
    lists[0] = 0;
    lists[1] = na;
    lists[2] = 0;
    lists[3] = nb;
    lists[4] = 0;
    lists[5] = nc;
}

}  // namespace
}  // namespace v3c

using namespace v3c;

extern "C" v3c_status v3c_lde_noalloc(const uint64_t* d_cols, uint32_t c, uint32_t log_n, uint32_t rate_bits,
                                      uint64_t* d_lde, uint32_t ld, void* stream)
{
    static_assert(sizeof(LdeJob) <= 32 * sizeof(u64), "job descriptor must fit the header words");
    if (!d_cols || !d_lde || c < 1 || ld < c || log_n > V3C_MAX_LOG_N || rate_bits > V3C_MAX_RATE_BITS ||
        log_n + rate_bits > V3C_MAX_LOG_LDE)
        return V3C_EINVAL;
    u32 l1, l2;
    plan_split(log_n, rate_bits, l1, l2);
    size_t n = (size_t)1 << log_n, N = n << rate_bits;
    size_t table_words = plan_table_words(log_n, rate_bits);
    size_t work_words = l1 ? (size_t)c * (n + N) : 0;
    if (kHeaderWords + table_words + work_words > V3C_NOALLOC_SCRATCH_BYTES / 8) return V3C_EINVAL;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return V3C_ECUDA;
    }
    u64* base = nullptr;
    v3c_status st = scratch_address(dev, &base);
    if (st) return st;
    cudaStream_t s = (cudaStream_t)stream;

    LdeJob j;
    memset(&j, 0, sizeof j);
    j.plan.log_n = log_n;
    j.plan.r = rate_bits;
    j.plan.gshift = 1;
    j.plan.sfac = gl::h_inv(n % gl::P);
    if (build_plan_tables(j.plan, base + kHeaderWords, s) != cudaSuccess) return V3C_ECUDA;
    j.x = d_cols;
    j.c = c;
    j.ld = ld;
    j.wcols = ld;
    j.lde = d_lde;
    j.vec_ok = ((uintptr_t)d_lde % 16 == 0) && (ld % 2 == 0);
    if (l1) {
        j.Y = base + kHeaderWords + table_words;
        j.Z = j.Y + (size_t)c * n;
    }
    lde_job_tiles(j);  // same tile rules as the allocating path

    Tiles t = default_tiles();
    u32 na = stage_a_items(j, t), nb = stage_b_items(j), nc = stage_c_items(j, t);
    k_noalloc_header<<<1, 32, 0, s>>>(j, na, nb, nc, base);
    if (cudaGetLastError() != cudaSuccess) return V3C_ECUDA;
    const LdeJob* dj = reinterpret_cast<const LdeJob*>(base);
    const u32* lists = reinterpret_cast<const u32*>(base + 32);
    u32 done_cols = c + (c & 1);
    if (ld > done_cols &&
        cudaMemset2DAsync(d_lde + done_cols, (size_t)ld * 8, 0, (size_t)(ld - done_cols) * 8, N, s) != cudaSuccess)
        return V3C_ECUDA;
    StageList la{lists, 1, na}, lb{lists + 2, 1, nb}, lc{lists + 4, 1, nc};
    if (na && launch_stage_a(dj, la, stage_a_smem(j, t), t, 0, s) != cudaSuccess) return V3C_ECUDA;
    const bool spec = lde_job_spec(j);
    if (nb && launch_stage_b(dj, lb, stage_b_smem(j), t, 0, s, spec) != cudaSuccess) return V3C_ECUDA;
    if (nc && launch_stage_c(dj, lc, stage_c_smem(j, t), t, 0, s) != cudaSuccess) return V3C_ECUDA;
    return V3C_OK;
}
