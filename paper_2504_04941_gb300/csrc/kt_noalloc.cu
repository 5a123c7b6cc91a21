// kt_noalloc.cu -- kt_integrate_noalloc: the integrate call for callers that must not
// allocate device memory.
//
// Some hosts cannot call cudaMalloc at the point where they integrate: a solver step
// that runs inside a host framework's own memory pool, code that runs while another
// component owns every allocation, or a context where allocating would break a
// real-time budget.  For them this entry point reuses the ordinary kernels with every
// piece of memory they need beyond the caller's inputs and outputs -- the work-queue
// counter, the device error word and the network tables -- placed in one file-scope
// static device array of fixed size (kNoAllocBytes per device, held by every device
// that loads the library until the process exits).
#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <mutex>

#include "kt_internal.h"

namespace {

constexpr size_t kNoAllocBytes = 64 * 1024;   // static scratch per device
constexpr size_t kTablesOffset = 256;          // scratch words first, then the tables
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

std::mutex g_mu;
unsigned char *g_addr[kMaxDevices] = {};       // device address of g_noalloc_scratch per device

// Set-up, once per device with that device current: the device address of the static
// array (its name in host code is only a stand-in for the symbol).
int scratch_address(unsigned char **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        kt::set_error("kt_integrate_noalloc: no usable current device");
        return KT_ECUDA;
    }
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            char msg[256];
            std::snprintf(msg, sizeof msg, "kt_integrate_noalloc: cudaGetSymbolAddress failed: %s",
                          cudaGetErrorString(e));
            kt::set_error(msg);
            return KT_ECUDA;
        }
        g_addr[dev] = static_cast<unsigned char *>(p);
    }
    *out = g_addr[dev];
    return KT_OK;
}

}  // namespace

extern "C" KT_API int kt_integrate_noalloc(const kt_network *net, int64_t ncells, const double *y_in,
                                           const double *T_in, const double *rho, double dt,
                                           const kt_options *opts, double *y_out, double *T_out,
                                           int32_t *status, int32_t *n_substeps, int32_t *n_newton,
                                           void *cuda_stream)
{
    // the per-cell status is this call's only report of a device-side failure (the error
    // word sits in the internal array, which the caller cannot read), so it is required
    if (!status) {
        kt::set_error("kt_integrate_noalloc: status must not be NULL (it is the only error report)");
        return KT_EINVAL;
    }
    kt::LaunchArgs a{};
    kt::LaunchCfg c{};
    const unsigned char *host_tables = nullptr;
    int rc = kt::prepare_launch(net, ncells, y_in, T_in, rho, dt, opts, y_out, T_out, status, n_substeps,
                                n_newton, &a, &c, &host_tables);
    if (rc) return rc;
    const size_t need = kTablesOffset + static_cast<size_t>(a.nv.bytes_total);
    if (need > kNoAllocBytes) {
        char msg[256];
        std::snprintf(msg, sizeof msg,
                      "kt_integrate_noalloc: the network tables need %zu bytes of scratch, the static area "
                      "holds %zu; use kt_integrate_ptrs for this network",
                      need, kNoAllocBytes);
        kt::set_error(msg);
        return KT_EINVAL;
    }
    if (ncells == 0) return KT_OK;
    unsigned char *area = nullptr;
    rc = scratch_address(&area);
    if (rc) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    // the area keeps the previous call's contents: reset the queue counter and the error
    // word, refresh the tables; -1 marks cells a kernel did not reach (a device error)
    cudaError_t e = cudaMemsetAsync(area, 0, sizeof(kt::Scratch), s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(area + kTablesOffset, host_tables, static_cast<size_t>(a.nv.bytes_total),
                            cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(status, 0xff, static_cast<size_t>(ncells) * sizeof(int32_t), s);
    if (e != cudaSuccess) {
        char msg[256];
        std::snprintf(msg, sizeof msg, "kt_integrate_noalloc: %s", cudaGetErrorString(e));
        kt::set_error(msg);
        return KT_ECUDA;
    }
    a.blob = area + kTablesOffset;
    a.scratch = reinterpret_cast<kt::Scratch *>(area);
    const int ce = c.cells_per_warp == 32 ? kt::launch_lane(a, c, cuda_stream) : kt::launch_warp(a, c, cuda_stream);
    if (ce != 0) {
        char msg[256];
        std::snprintf(msg, sizeof msg, "kt_integrate_noalloc: kernel launch: %s",
                      cudaGetErrorString(static_cast<cudaError_t>(ce)));
        kt::set_error(msg);
        return KT_ECUDA;
    }
    return KT_OK;
}
