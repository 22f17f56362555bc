// tvolap_process_signal_static: the offline path with its scratch in a fixed
// device array instead of a workspace the library allocates.
//
// Who needs it: callers that must not allocate device memory once they are
// running, for example a real-time audio callback whose deadline leaves no room
// for an allocation that may synchronise the device or take unbounded time, or
// a host process that runs under a fixed device-memory budget set at start-up.
// tvolap_process_signal grows its workspace with cudaMalloc; this variant uses
// the file-scope array below, which every GPU that loads the library holds
// until the process exits.
#include <mutex>

#include "internal.h"
#include "trace.h"

using namespace tvolap;

namespace {

// Forward spectra X then output spectra Y of one call.
static __device__ __align__(256) unsigned char g_static_scratch[TVOLAP_STATIC_SCRATCH_BYTES];

constexpr int MAX_DEVICES = 64;

// Device address of g_static_scratch on the plan's device, looked up once per
// device (host code cannot use the symbol itself: on the host it is only a
// stand-in). The plan's device is its stream's; the lookup resolves the symbol
// on the current device, so the two must be the same (TVOLAP_ERR_ARG if not:
// the kernels would otherwise run on the plan's device against another GPU's
// copy of the array).
void *scratch_address(cudaStream_t stream, int &status)
{
    static std::mutex mu;
    static void *addr[MAX_DEVICES] = {};
    int dev = 0, plan_dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaStreamGetDevice(stream, &plan_dev);
    if (e != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) {
        cudaGetLastError();
        status = TVOLAP_ERR_CUDA;
        return nullptr;
    }
    if (plan_dev != dev) {
        status = TVOLAP_ERR_ARG;
        return nullptr;
    }
    std::lock_guard<std::mutex> lock(mu);
    if (!addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            status = TVOLAP_ERR_CUDA;
            return nullptr;
        }
        addr[dev] = p;
    }
    status = TVOLAP_OK;
    return addr[dev];
}

}  // namespace

extern "C" int tvolap_process_signal_static(tvolap_t h, const float *x_dev, int64_t N,
                                            int64_t x_stride, const int32_t *sched_a,
                                            const int32_t *sched_b, const float *sched_alpha,
                                            int64_t sched_stride, float *y_dev, int64_t out_len,
                                            int64_t y_stride)
{
    TVOLAP_TRACE();
    if (!h) return TVOLAP_ERR_STATE;
    if (N < 0 || out_len < 0 || x_stride < N || y_stride < out_len) return TVOLAP_ERR_ARG;
    if (out_len == 0) return TVOLAP_OK;
    if ((N > 0 && !x_dev) || !y_dev || !sched_a) return TVOLAP_ERR_ARG;
    const int64_t nb = (out_len - 1) / h->L + 2;
    if (nb > (int64_t)0x7fffffff / 2 || sched_stride < nb) return TVOLAP_ERR_ARG;
    const int64_t bytes = (int64_t)sizeof(float2) * h->P * nb * (h->n_in + h->n_out);
    if (bytes > (int64_t)TVOLAP_STATIC_SCRATCH_BYTES) return TVOLAP_ERR_CAPACITY;
    int st = TVOLAP_OK;
    float2 *X = reinterpret_cast<float2 *>(scratch_address(h->stream, st));
    if (st != TVOLAP_OK) return st;
    float2 *Y = X + (int64_t)h->n_in * nb * h->P;
    // every element of X and Y is written before it is read: nothing to clear
    cudaError_t e = launch_forward_signal(h, x_dev, N, x_stride, (int)nb, X);
    if (e == cudaSuccess)
        e = launch_mac_signal_lsu(h, X, (int)nb, sched_a, sched_b, sched_alpha, sched_stride, Y);
    if (e == cudaSuccess) e = launch_inverse_ola(h, Y, (int)nb, y_dev, out_len, y_stride);
    if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? TVOLAP_ERR_OOM : TVOLAP_ERR_CUDA;
    return TVOLAP_OK;
}
