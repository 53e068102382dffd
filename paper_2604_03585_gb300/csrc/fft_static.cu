// sar_fft_lines_static: the line FFT of sar_fft_lines without any device
// memory allocation.
//
// sar_fft_lines keeps its twiddle tables in device memory that the library
// allocates with cudaMalloc the first time each line length is used on a
// device.  Some callers cannot let a library allocate device memory behind
// their back: real-time or on-board radar processors that fix their whole
// device-memory footprint at start-up and forbid any later allocation, and
// applications whose device memory belongs to a pool allocator that a hidden
// cudaMalloc could fail against or fragment.  This entry point serves them:
// its twiddle table lives
// in a fixed file-scope device array that exists once the CUDA module holding
// it is loaded (with CUDA's lazy module loading, the default, that happens on
// first use, not when the library is opened), and it calls no cudaMalloc,
// cudaFree or allocating library routine.
//
// Limits and sharing rules:
//   * the array holds kStaticTwiddleElems = 32768 complex64 values (256 KiB);
//     every GPU that loads the library keeps it until the process exits.  The
//     largest table any supported line length needs is 17,408 values
//     (N = 16384), so every N in [256, 16384] fits; a length whose table
//     would not fit is refused with SAR_ERR_UNSUPPORTED.
//   * every call rewrites the table for its own N on the caller's stream,
//     before its FFT; nothing in the array has to start at zero.  All calls,
//     from every stream and thread, share this one array: two calls that can
//     run at the same time on the GPU (different streams without an ordering
//     event between them) race on it and may compute with the wrong table.
//     Order such calls on one stream, or with events.
//   * the first call on each device looks up the array's device address once
//     (cudaGetSymbolAddress) with that device current; the first call at each
//     line length on a device loads that length's kernels (lazy loading) and
//     sets their shared-memory limits, once, so it does more host work than
//     the calls after it.
#include <mutex>

#include "../../include/sar.h"
#include "registry.h"
#include "tables.h"

namespace sar {
sar_status report_error(sar_status st, const char *msg);
sar_status validate_device_ptr(const void *p, const char *what);
sar_status validate_length(int64_t n, const char *what);
}  // namespace sar

namespace {

constexpr int kStaticTwiddleElems = 32768;

__device__ __align__(256) float2 g_static_twiddles[kStaticTwiddleElems];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
float2 *g_twiddle_addr[kMaxDevices] = {};   // device address of the array, per device
// schedules whose kernel attributes are set, per device (a schedule is one
// compiled kernel set: its descriptor's address identifies it)
constexpr int kMaxPrepared = 64;
const sar::SchedDesc *g_prepared[kMaxDevices][kMaxPrepared] = {};

// Once per device, with that device current: find where the array lives in
// this device's memory (the host-side name g_static_twiddles is only a
// stand-in, not a device address).
sar_status static_twiddles(const sar::SchedDesc &d, float2 **out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return sar::report_error(SAR_ERR_CUDA, "cudaGetDevice failed");
    if (dev < 0 || dev >= kMaxDevices) return sar::report_error(SAR_ERR_UNSUPPORTED, "device index out of range");
    std::lock_guard<std::mutex> lk(g_setup_mu);
    if (!g_twiddle_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_static_twiddles);
        if (e != cudaSuccess || p == nullptr) {
            cudaGetLastError();
            return sar::report_error(SAR_ERR_CUDA, "cudaGetSymbolAddress of the static twiddle array failed");
        }
        g_twiddle_addr[dev] = (float2 *)p;
    }
    // shared-memory limit of the kernels (an attribute, not an allocation),
    // once per device and schedule
    bool done = false;
    int slot = -1;
    for (int i = 0; i < kMaxPrepared && !done; ++i) {
        if (g_prepared[dev][i] == &d) done = true;
        else if (!g_prepared[dev][i] && slot < 0) slot = i;
    }
    if (!done) {
        e = d.prepare();
        if (e != cudaSuccess) return sar::report_error(SAR_ERR_CUDA, "cudaFuncSetAttribute failed");
        if (slot >= 0) g_prepared[dev][slot] = &d;
    }
    *out = g_twiddle_addr[dev];
    return SAR_OK;
}

}  // namespace

extern "C" sar_status sar_fft_lines_static(int64_t n, int64_t n_lines, const void *in, void *out, int inverse,
                                           sar_stream stream) {
    sar_status st;
    if ((st = sar::validate_length(n, "n")) != SAR_OK) return st;
    const sar::SchedDesc *d = sar::default_schedule((int)n);
    if (!d) return sar::report_error(SAR_ERR_UNSUPPORTED, "no compiled schedule for this length");
    if (d->tw_elems > kStaticTwiddleElems)
        return sar::report_error(SAR_ERR_UNSUPPORTED,
                                 "this length needs a twiddle table larger than the static 32768-entry array");
    if (n_lines < 0) return sar::report_error(SAR_ERR_INVALID_ARG, "n_lines < 0");
    if (n_lines == 0) return SAR_OK;
    if ((st = sar::validate_device_ptr(in, "in")) != SAR_OK) return st;
    if ((st = sar::validate_device_ptr(out, "out")) != SAR_OK) return st;
    const size_t bytes = sizeof(float2) * (size_t)n * (size_t)n_lines;
    const char *a = (const char *)in, *b = (const char *)out;
    if (a != b && a < b + bytes && b < a + bytes)
        return sar::report_error(SAR_ERR_INVALID_ARG, "in and out partially overlap");
    float2 *tw = nullptr;
    if ((st = static_twiddles(*d, &tw)) != SAR_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = sar::build_twiddles(*d, tw, s);
    if (e != cudaSuccess) return sar::report_error(SAR_ERR_CUDA, "twiddle table launch failed");
    e = d->dft((const float2 *)in, (float2 *)out, n_lines, n, (int)n, tw, inverse ? 1 : 0, s);
    if (e != cudaSuccess) return sar::report_error(SAR_ERR_CUDA, "fft launch failed");
    return SAR_OK;
}
