// ts_norm_noalloc: the norm reduction for callers that cannot allocate
// device memory.
//
// The regular ts_norm keeps its per-block partial sums in the grid's slab.
// This entry point instead uses one fixed scratch array that lives in the
// library's own device image, so the call itself allocates nothing: no
// cudaMalloc, no cudaFree, no torch or other allocating routine.
//
// The array is a file-scope __device__ variable.  Host code cannot use its
// name as a device address (on the host the name is only a stand-in); the
// device address is looked up once per device with cudaGetSymbolAddress, with
// that device current, and passed to the kernels.
#include <cstdint>
#include <cstdio>
#include <mutex>

#include "../../include/trotter.h"
#include "internal.h"

namespace {

constexpr int kMaxDevices = 64;
constexpr size_t kScratchDoubles = (size_t)ts::OBS_MAX_BLOCKS * ts::OBS_Q;   // 56 KiB

// One array per device that loads the library, kept until the process exits.
static __device__ __align__(256) double g_norm_scratch[kScratchDoubles];

std::mutex g_mu;
double *g_scratch_addr[kMaxDevices] = {};

}  // namespace

extern "C" size_t ts_norm_noalloc_scratch_bytes(void)
{
    return kScratchDoubles * sizeof(double);
}

extern "C" ts_status ts_norm_noalloc(const void *re, const void *im, ts_dtype dtype, int64_t nx,
                                     int64_t ny, int64_t pitch, double *out, void *stream)
{
    if (!re || !im || !out)
        return (ts_status)ts::set_error(TS_ERR_ARG, "ts_norm_noalloc: null argument");
    if (dtype != TS_F32 && dtype != TS_F64)
        return (ts_status)ts::set_error(TS_ERR_ARG, "ts_norm_noalloc: unknown dtype %d", (int)dtype);
    // The reduction runs a grid-stride loop over at most OBS_MAX_BLOCKS blocks,
    // so the fixed scratch holds every partial for any grid inside these limits.
    if (nx < 1 || ny < 1 || nx > (int64_t(1) << 20) || ny > (int64_t(1) << 20))
        return (ts_status)ts::set_error(
            TS_ERR_ARG, "ts_norm_noalloc: sides must be in [1, 2^20] for its fixed %zu-byte "
            "scratch, got %lld x %lld", kScratchDoubles * sizeof(double), (long long)nx,
            (long long)ny);
    if (pitch < nx || pitch > (int64_t(1) << 31))
        return (ts_status)ts::set_error(TS_ERR_ARG, "ts_norm_noalloc: pitch %lld must be in "
                                        "[nx, 2^31]", (long long)pitch);
    // The FP32 reduction reads 4 sites at a time with 16-byte loads from
    // re + y*pitch + x0 (x0 a multiple of 4), so the planes must be 16-byte
    // aligned and the pitch a multiple of 4 floats; then a row's last load
    // stays inside that row's pitch.  The FP64 reduction loads single doubles.
    const uintptr_t align = dtype == TS_F32 ? 16 : 8;
    if ((uintptr_t)re % align != 0 || (uintptr_t)im % align != 0)
        return (ts_status)ts::set_error(TS_ERR_ARG, "ts_norm_noalloc: re and im must be %d-byte "
                                        "aligned for this dtype", (int)align);
    if (dtype == TS_F32 && pitch % 4 != 0)
        return (ts_status)ts::set_error(TS_ERR_ARG, "ts_norm_noalloc: an FP32 pitch must be a "
                                        "multiple of 4, got %lld", (long long)pitch);
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return (ts_status)ts::set_error(TS_ERR_CUDA, "ts_norm_noalloc: no usable current device");
    double *scratch = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        if (!g_scratch_addr[dev]) {
            void *p = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&p, g_norm_scratch);
            if (e != cudaSuccess || !p)
                return (ts_status)ts::set_error(TS_ERR_CUDA, "ts_norm_noalloc: "
                                                "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
            g_scratch_addr[dev] = (double *)p;
        }
        scratch = g_scratch_addr[dev];
    }
    // Every partial the final pass reads is written by the first pass of the
    // same call, so the array needs no clearing between calls.
    cudaError_t e = ts::launch_observe(re, im, nullptr, dtype == TS_F64, (int)nx, (int)ny, pitch,
                                       0.0, true, scratch, out, (cudaStream_t)stream);
    if (e != cudaSuccess)
        return (ts_status)ts::set_error(TS_ERR_CUDA, "ts_norm_noalloc: launch: %s",
                                        cudaGetErrorString(e));
    return TS_OK;
}
