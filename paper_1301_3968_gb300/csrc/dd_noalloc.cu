// Boxcar S/N without device allocation.
//
// dd_boxcar_snr keeps its normaliser tables in workspace that the plan allocates on
// first use.  Some callers may not allocate device memory once they are running: a
// real-time detection pipeline that fixes its device-memory footprint at start-up
// (a late cudaMalloc can stall the pipeline or fail once the memory is committed), or
// a host that gives the library a fixed device-memory budget.  dd_boxcar_snr_noalloc
// computes the same result with its scratch in a fixed-size array in device global
// memory that is part of the library image, so it allocates nothing.
//
// CUDA loads a module's code and its __device__ arrays onto a device lazily, at first
// use.  So that this entry point's first call is not that use, the array and the boxcar
// kernels are loaded when a plan's tables are first put on a device (noalloc_preload,
// from upload_tables), which the entry point requires anyway.
#include <mutex>

#include "dd_internal.h"
#include "dd_trace.h"

namespace {

// Scratch for the normaliser tables of one call: per-trial offsets (fp64), the
// normaliser means and inverse deviations ([ndm][nw] fp32 each) and the width list.
// Every GPU on which a plan's tables have been uploaded holds these 8 MiB until the
// process exits.
constexpr size_t kScratchBytes = (size_t)8 << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
void* g_scratch_addr[kMaxDevices];  // device address of the array, per device

size_t align256(size_t n) { return (n + 255) & ~(size_t)255; }

// The array's device address on the current device.  In host code the array's name
// is only a stand-in, so the address is looked up once per device (with that device
// current) and cached.  The first lookup on a device also loads the array and the
// boxcar kernels there.
dd_status scratch_address(void** out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return dd::cuda_status(e);
    if (dev < 0 || dev >= kMaxDevices) return DD_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return dd::cuda_status(e);
        const dd_status st = dd::preload_boxcar_kernels();
        if (st != DD_OK) return st;
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return DD_OK;
}

}  // namespace

namespace dd {
dd_status noalloc_preload() {
    void* p = nullptr;
    return scratch_address(&p);
}
}  // namespace dd

extern "C" dd_status dd_boxcar_snr_noalloc(dd_plan_t p, const void* x, int64_t ld, int64_t t_len,
                                           const int32_t* widths, int32_t nw, const double* mean,
                                           const double* sd, float* peak, int32_t* arg,
                                           float thresh, dd_candidate* cands, int32_t cap,
                                           int32_t* ncands, void* stream) {
    DD_TRACE("dd_boxcar_snr_noalloc");
    if (!p || !x || !widths || nw < 1 || !mean || !sd || !peak || !arg) return DD_ERR_ARG;
    if (t_len < 1 || ld < t_len || t_len > INT32_MAX) return DD_ERR_ARG;
    if (cands && (!ncands || cap < 0)) return DD_ERR_ARG;
    for (int i = 0; i < nw; ++i) {
        if (widths[i] < 1 || widths[i] > t_len) return DD_ERR_ARG;
        if (i && widths[i] <= widths[i - 1]) return DD_ERR_ARG;
    }
    const size_t b_off = align256((size_t)p->ndm * sizeof(double));
    const size_t b_tab = align256((size_t)p->ndm * nw * sizeof(float));
    const size_t b_w = align256((size_t)nw * sizeof(int32_t));
    if (b_off + 2 * b_tab + b_w > kScratchBytes) return DD_ERR_CAPACITY;
    // the plan's tables must already be on this device: uploading them would allocate
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return dd::cuda_status(e);
    if (p->dev_dirty || p->dev.device != dev) return DD_ERR_STATE;
    void* base = nullptr;
    dd_status st = scratch_address(&base);
    if (st != DD_OK) return st;
    unsigned char* s = (unsigned char*)base;
    double* off = (double*)s;
    float* mu = (float*)(s + b_off);
    float* isd = (float*)(s + b_off + b_tab);
    int32_t* wdev = (int32_t*)(s + b_off + 2 * b_tab);
    // every scratch value this call reads is written earlier in the same call, so
    // nothing needs clearing; the widths travel by a stream-ordered copy (from pageable
    // memory the copy has read them when it returns; from pinned memory only once the
    // stream reaches it)
    e = cudaMemcpyAsync(wdev, widths, (size_t)nw * sizeof(int32_t), cudaMemcpyHostToDevice,
                        (cudaStream_t)stream);
    if (e != cudaSuccess) return dd::cuda_status(e);
    return dd::launch_boxcar_scratch(p, x, ld, t_len, widths, nw, wdev, mean, sd, off, mu, isd,
                                     peak, arg, thresh, cands, cap, ncands, (cudaStream_t)stream);
}
