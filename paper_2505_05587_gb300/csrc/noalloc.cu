// Allocation-free variant of sgs_densify_split.
//
// Some callers cannot hand the library a workspace: code that runs where a
// cudaMalloc is not allowed or not wanted (inside a host callback, in a
// real-time loop where an allocation would synchronise the device, or in a
// plugin whose host owns every device allocation and exposes only the
// input/output buffers).  For them this entry point takes its scratch from a
// fixed array that lives in the library's device image instead of from a
// caller workspace.  The array is reserved on every GPU that loads the
// library, for as long as the process runs.
#include <mutex>

#include "common.cuh"

namespace sgs {

// Scratch for sgs_densify_split_noalloc: split flags, their prefix sum, the
// eigenvalue and the (up to 7-component) eigenvector when the caller passes no
// output for them, and the budget's tie flags -- 4 + 4 + 4 + 28 + 4 = 44 bytes
// per Gaussian -- plus the scan's block partials and 256-byte alignment of
// each region: about 44 MB at SGS_NOALLOC_MAX_GAUSSIANS.  Every call checks
// that the largest allowed n still fits, so a change of the workspace layout
// cannot silently shrink the documented limit.
static __device__ __align__(256) unsigned char g_densify_scratch[SGS_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
static void* g_scratch_addr[kMaxDevices];
static std::mutex g_scratch_mu;

// Device address of the scratch array on the calling thread's current device.
// Host code cannot use the array's name as a device address, so the address is
// looked up once per device (with that device current) and cached for the life
// of the process: a device reset (cudaDeviceReset) reloads the library's device
// image elsewhere, after which the cached address is stale.
static int scratch_address(void** out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return (int)e;
    if (dev < 0 || dev >= kMaxDevices) return (int)cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (g_scratch_addr[dev] == nullptr) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_densify_scratch);
        if (e != cudaSuccess) return (int)e;
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return 0;
}

}  // namespace sgs

using namespace sgs;

extern "C" int sgs_densify_split_noalloc(const sgs_gaussians* in, const float* S_accum, const float* S_po_accum,
                                         const float* S_ls_accum, float inv_T_split, float eps_split, float step_scale,
                                         const float* grad_norm, float eps_grad, int64_t max_splits,
                                         const sgs_gaussians_mut* out, int64_t capacity, int32_t* d_n_out,
                                         int32_t* parent_index, float* lam_min_out, float* v_min_out,
                                         void* stream) {
    SGS_NVTX_RANGE();
    if (densify_ws_bytes(SGS_NOALLOC_MAX_GAUSSIANS) > (size_t)SGS_NOALLOC_SCRATCH_BYTES) return SGS_ERR_WORKSPACE;
    if (!in || in->n < 0 || in->n > SGS_NOALLOC_MAX_GAUSSIANS) return SGS_ERR_INVALID_ARG;
    if (densify_ws_bytes(in->n) > (size_t)SGS_NOALLOC_SCRATCH_BYTES) return SGS_ERR_WORKSPACE;
    void* ws = nullptr;
    int ce = scratch_address(&ws);
    if (ce != 0) return record_cuda_error((cudaError_t)ce);
    return sgs_densify_split(in, S_accum, S_po_accum, S_ls_accum, inv_T_split, eps_split, step_scale, grad_norm,
                             eps_grad,
                             max_splits, out, capacity, d_n_out, parent_index, lam_min_out, v_min_out, ws,
                             (size_t)SGS_NOALLOC_SCRATCH_BYTES, stream);
}
