// lc_monitor_noalloc: the steady-state monitor reduction for callers that
// cannot allocate device memory.
//
// Some callers cannot call cudaMalloc: a host framework that owns every byte
// of device memory through its own pool, code running while a CUDA graph is
// being captured (where allocation is not allowed), or a process whose
// memory budget is fixed up front.  This entry point computes the same three
// monitors as lc_monitor on state arrays the caller already holds, and keeps
// its only scratch (one partial result per grid row and a block counter) in
// a fixed file-scope device array instead of allocating it.
//
// The array is 3 * (LC_NOALLOC_MAX_N + 1) doubles plus a counter, about
// 192 KiB; every GPU that loads the library holds it until the process
// exits.  All calls share it, so calls whose work overlaps on the GPU (on two
// streams, or from two threads) race and give wrong results; calls issued in
// order on one stream are safe.  The counter is cleared at the start of
// every call; the partials are fully rewritten by each call before they are
// read.
#include "../../include/lc.h"
#include "lc_internal.h"

#include <cuda_runtime.h>

#include <cmath>
#include <mutex>
#include <string>

namespace {

struct NoAllocScratch {
    double part[3 * (LC_NOALLOC_MAX_N + 1)];
    unsigned int counter;
};

static __device__ __align__(256) NoAllocScratch g_noalloc_scratch;

constexpr int kThreads = 256;
constexpr int kMaxDevices = 64;

std::mutex g_mu;
NoAllocScratch *g_dev_ptr[kMaxDevices];  // device address of g_noalloc_scratch, per device

__device__ __forceinline__ void reduce3(double &mx, double &s1, double &s2, double (*sh)[kThreads / 32]) {
    for (int o = 16; o > 0; o >>= 1) {
        mx = fmax(mx, __shfl_down_sync(0xffffffffu, mx, o));
        s1 += __shfl_down_sync(0xffffffffu, s1, o);
        s2 += __shfl_down_sync(0xffffffffu, s2, o);
    }
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) {
        sh[0][warp] = mx;
        sh[1][warp] = s1;
        sh[2][warp] = s2;
    }
    __syncthreads();
    if (warp == 0) {
        mx = lane < kThreads / 32 ? sh[0][lane] : 0.0;
        s1 = lane < kThreads / 32 ? sh[1][lane] : 0.0;
        s2 = lane < kThreads / 32 ? sh[2][lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) {
            mx = fmax(mx, __shfl_down_sync(0xffffffffu, mx, o));
            s1 += __shfl_down_sync(0xffffffffu, s1, o);
            s2 += __shfl_down_sync(0xffffffffu, s2, o);
        }
    }
}

// One block per grid row j: max |d omega|, sum |d psi|, sum |d omega| over the
// row into the scratch partials; the last block to finish reduces the rows in
// order 0..N and writes out[0] = max / dt, out[1] = RES_psi, out[2] = RES_omega.
__global__ void __launch_bounds__(kThreads)
    k_monitor_rows(const double *__restrict__ p0, const double *__restrict__ p1, const double *__restrict__ w0,
                   const double *__restrict__ w1, int N, size_t pitch, double dt, double *__restrict__ out,
                   NoAllocScratch *scr) {
    __shared__ double sh[3][kThreads / 32];
    __shared__ bool last;
    int j = blockIdx.x;
    double mx = 0.0, sp = 0.0, sw = 0.0;
    for (int i = threadIdx.x; i <= N; i += kThreads) {
        size_t c = (size_t)j * pitch + i;
        double dw = fabs(w1[c] - w0[c]);
        mx = fmax(mx, dw);
        sw += dw;
        sp += fabs(p1[c] - p0[c]);
    }
    reduce3(mx, sp, sw, sh);
    if (threadIdx.x == 0) {
        scr->part[3 * j] = mx;
        scr->part[3 * j + 1] = sp;
        scr->part[3 * j + 2] = sw;
        __threadfence();
        last = atomicAdd(&scr->counter, 1u) == (unsigned)N;  // N + 1 rows
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    const volatile double *part = scr->part;
    mx = 0.0;
    sp = 0.0;
    sw = 0.0;
    for (int r = threadIdx.x; r <= N; r += kThreads) {
        mx = fmax(mx, part[3 * r]);
        sp += part[3 * r + 1];
        sw += part[3 * r + 2];
    }
    reduce3(mx, sp, sw, sh);
    if (threadIdx.x == 0) {
        out[0] = mx / dt;
        out[1] = sp / (N + 1);
        out[2] = sw / (N + 1);
    }
}

int noalloc_fail(int code, const std::string &msg) {
    lcx::set_last_error(msg.c_str());
    return code;
}

}  // namespace

extern "C" int lc_monitor_noalloc(int N, const double *psi0, const double *psi1, const double *omega0,
                                  const double *omega1, size_t pitch, double dt, double *out, void *cuda_stream) {
    if (!psi0 || !psi1 || !omega0 || !omega1 || !out) return noalloc_fail(LC_ERR_ARG, "NULL array");
    if (N < 1) return noalloc_fail(LC_ERR_ARG, "N must be >= 1");
    if (N > LC_NOALLOC_MAX_N)
        return noalloc_fail(LC_ERR_SIZE, "N exceeds LC_NOALLOC_MAX_N (" + std::to_string(LC_NOALLOC_MAX_N) +
                                             "), the size of the fixed scratch array");
    if (pitch < (size_t)N + 1) return noalloc_fail(LC_ERR_ARG, "pitch must be >= N + 1");
    if (!(dt > 0.0) || !std::isfinite(dt)) return noalloc_fail(LC_ERR_ARG, "dt must be positive and finite");

    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return noalloc_fail(LC_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return noalloc_fail(LC_ERR_CUDA, "device ordinal out of range");
    NoAllocScratch *scr;
    {
        // one-time set-up per device, with that device current: the host-side
        // name of the array is not a device address, so look the address up
        std::lock_guard<std::mutex> lk(g_mu);
        if (!g_dev_ptr[dev]) {
            void *p = nullptr;
            e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess)
                return noalloc_fail(LC_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
            g_dev_ptr[dev] = static_cast<NoAllocScratch *>(p);
        }
        scr = g_dev_ptr[dev];
    }
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    e = cudaMemsetAsync(&scr->counter, 0, sizeof(unsigned int), s);
    if (e != cudaSuccess) return noalloc_fail(LC_ERR_CUDA, std::string("cudaMemsetAsync: ") + cudaGetErrorString(e));
    k_monitor_rows<<<N + 1, kThreads, 0, s>>>(psi0, psi1, omega0, omega1, N, pitch, dt, out, scr);
    e = cudaGetLastError();
    if (e != cudaSuccess) return noalloc_fail(LC_ERR_CUDA, std::string("launch: ") + cudaGetErrorString(e));
    return LC_OK;
}
