// Internal declarations shared by the CUDA translation units of libsteepgs.
// Not part of the public ABI (include/steepgs.h is).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <utility>

#include <nvtx3/nvToolsExt.h>

#include "steepgs.h"

namespace sgs {

constexpr int kMaxShDegree = 3;

// ---------------------------------------------------------------------------
// IEEE float32 operations that the compiler never contracts into FMA.  The
// integer stage (depth key, tile rect) is written with these so that every
// build produces the same bits.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float sub_rn(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float div_rn(float a, float b) { return __fdiv_rn(a, b); }
__device__ __forceinline__ float sqrt_rn(float a) { return __fsqrt_rn(a); }
// a*b + c with two roundings
__device__ __forceinline__ float mad_rn(float a, float b, float c) { return __fadd_rn(__fmul_rn(a, b), c); }

// Float32 state of one Gaussian in one view, produced by the integer stage.
struct Stage {
    bool culled;
    float tx, ty, tz;      // camera-space mean
    float ux, uy;          // clamped tx/tz, ty/tz
    bool clx, cly;         // clamp active
    float T[6];            // P = J W (2x3)
    float Rq[9];           // rotation of the unit quaternion
    float qn;              // |q|
    float s[3];            // exp(log_scale)
    float V[6];            // P Rq diag(s)
    float a, b, c;         // Sigma2D with dilation
    int x_lo, x_hi, y_lo, y_hi;
};

struct CamDev {
    float R[9];
    float t[3];
    float fx, fy, cx, cy;
    int width, height;
    float near_z;
    float limx, limy;       // Jacobian clamp limits
    float cc[3];            // camera centre -R^T t
    int gx, gy;             // tiles
};

// Up to kMaxViews views of one scene processed together.  Single-view calls
// use nv = 1.  Rows of the concatenated per-view projection buffers are
// v * n + i; global tile id = tile_off[v] + local tile id; pixel p of view v is
// pix_off[v] + p.  Passed by value as a kernel parameter.
constexpr int kMaxViews = 16;
struct ViewsDev {
    int nv;
    int T_total;
    long long P_total;
    int tile_off[kMaxViews + 1];
    long long pix_off[kMaxViews + 1];
    int row_off[kMaxViews + 1];     // projection rows of view v: [row_off[v], row_off[v+1])
    CamDev cam[kMaxViews];
};

// Gaussian arrays of each view's scene (all equal when the views share one).
struct ScenesDev {
    const float* means[kMaxViews];
    const float* log_scales[kMaxViews];
    const float* quats[kMaxViews];
    const float* opacity_logit[kMaxViews];
    const float* sh[kMaxViews];
};

__device__ __forceinline__ int view_of_row(const ViewsDev& vd, long long r) {
    int v = 0;
    while (v + 1 < vd.nv && r >= vd.row_off[v + 1]) ++v;
    return v;
}

__device__ __forceinline__ int view_of_tile(const ViewsDev& vd, int t) {
    int v = 0;
    while (v + 1 < vd.nv && t >= vd.tile_off[v + 1]) ++v;
    return v;
}

__device__ __forceinline__ int view_of_pixel(const ViewsDev& vd, long long p) {
    int v = 0;
    while (v + 1 < vd.nv && p >= vd.pix_off[v + 1]) ++v;
    return v;
}

struct SetDev {
    int tile_w, tile_h;
    float alpha_min, alpha_max, T_min, radius_sigma, dilation, fov_clamp;
    float bg[3];
};

__device__ Stage integer_stage(const float* __restrict__ means, const float* __restrict__ log_scales,
                               const float* __restrict__ quats, int i, const CamDev& cam,
                               const SetDev& st);

// NVTX range named after the entry point, for the duration of the host call:
// a profiler's timeline shows each call's launches under it.  Without a tool
// attached, push and pop are a pointer check each.
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};
#define SGS_NVTX_RANGE() ::sgs::NvtxRange sgs_nvtx_range_(__func__)

// Host helpers (defined in api.cu)
// Counts kernel launches issued by the library (for measurement reports).
void note_launch(int k = 1);

// Programmatic dependent launch: the kernel may be scheduled while the
// previous kernel on the stream drains; it waits for that kernel's completion
// (and memory) in pdl_wait_and_trigger before touching any data.
// launch_pdl_if(false, ...) launches the same kernel with ordinary stream
// order (its wait then returns at once).
template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl_if(bool pdl, void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem,
                                 cudaStream_t s, Args&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...);
}
template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                              Args&&... args) {
    return launch_pdl_if(true, kern, grid, block, smem, s, std::forward<Args>(args)...);
}
__device__ __forceinline__ void pdl_wait_and_trigger() {
    asm volatile("griddepcontrol.wait;\n" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;\n" :::);
}
// Keeps `e` for sgs_get_last_cuda_error() and returns SGS_ERR_CUDA.
int record_cuda_error(cudaError_t e);
CamDev make_cam(const sgs_camera& c, const sgs_settings& s);
ViewsDev make_views(const sgs_camera* cams, int nv, const sgs_settings& s, const int* rows_per_view = nullptr,
                    int rows_each = 0);
ScenesDev make_scenes(const sgs_gaussians* g, int nv, bool per_view);
SetDev make_set(const sgs_settings& s);
bool tile_supported(int tw, int th);

// Flags of the projection adjoint (the backward entry points' `flags`).
constexpr int kBwdAccumulateGrads = SGS_BWD_ACCUMULATE_GRADS;
constexpr int kBwdResetS = SGS_BWD_RESET_S;

// Launchers (host functions, enqueue on `stream`).
cudaError_t launch_project(const ScenesDev& sc, int sh_degree, const ViewsDev& vd, const SetDev& st,
                           const sgs_proj& out, cudaStream_t stream);
cudaError_t launch_project_bwd(const sgs_gaussians& g, const sgs_proj& proj, const ViewsDev& vd, const float* g2d,
                               const float* g2d_hi, int flags, const sgs_grads& grads, float* S_accum,
                               float* S_po_accum, float* S_ls_accum, cudaStream_t stream);

size_t bin_sort_ws_bytes(int n, int64_t capacity, int num_tiles);
cudaError_t launch_bin_sort(const sgs_proj& proj, const ViewsDev& vd, const SetDev& st, const sgs_bins& out, void* ws,
                            cudaStream_t stream);

// target != null: the L1 loss is fused into the epilogue (dL overwritten, loss +=).
cudaError_t launch_render_fwd(const sgs_proj& proj, const sgs_bins& bins, const CamDev& cam,
                              const SetDev& st, float* image, float* final_T, uint32_t* n_contrib,
                              const float* target, int n_views, float* dL, float* loss, cudaStream_t stream);
// Zeroes the 16-float accumulator rows (and the higher-moment rows when
// g2d_hi is not null) of the Gaussians with tiles_touched > 0.
cudaError_t launch_zero_reached_rows(const uint32_t* tiles, int n, float* g2d, float* g2d_hi, cudaStream_t stream);
cudaError_t launch_render_bwd(const sgs_proj& proj, const sgs_bins& bins, const CamDev& cam,
                              const SetDev& st, const float* final_T, const uint32_t* n_contrib,
                              const float* dL_dimage, float* g2d, float* g2d_hi, cudaStream_t stream);

// Walk lists of a multi-view pass (all null: none; the kernels then cull
// every list entry themselves): walk [cap] u32, count [T_total * warps per tile].
struct WalkLists {
    uint32_t* walk;
    uint32_t* count;
    long long cap;
};
cudaError_t launch_render_fwd_views(const ViewsDev& vd, const sgs_proj& proj, const uint32_t* ranges,
                                    const uint32_t* gids, const SetDev& st, int batch, float* images,
                                    float* final_T, uint32_t* n_contrib, uint32_t* counter, const uint32_t* order,
                                    const WalkLists& wl, cudaStream_t stream);
cudaError_t launch_render_bwd_views(const ViewsDev& vd, const sgs_proj& proj, const uint32_t* ranges,
                                    const uint32_t* gids, const SetDev& st, int batch, const float* final_T,
                                    const uint32_t* n_contrib, const float* dL, float* g2d, uint32_t* counter,
                                    const uint32_t* order, const WalkLists& wl, cudaStream_t stream);

size_t ssim_ws_bytes(int H, int W);
cudaError_t launch_ssim_l1(const float* image, const float* target, int H, int W, int n_views, float lam, float* dL,
                           float* loss, void* ws, cudaStream_t stream);
cudaError_t launch_fma_probe(float* out, int blocks, int iters, cudaStream_t stream);
cudaError_t launch_render_stats(const sgs_proj& proj, const sgs_bins& bins, const CamDev& cam,
                                const SetDev& st, uint32_t* counts, uint32_t* warp_union, cudaStream_t stream);

cudaError_t launch_l1_views(const float* image, const float* target, const ViewsDev& vd, float* dL, float* loss,
                            cudaStream_t stream);
cudaError_t launch_l1(const float* image, const float* target, int H, int W, int n_views,
                      float* dL, float* loss, cudaStream_t stream);

cudaError_t launch_adam(float* p, const float* g, float* m, float* v, int64_t count, float lr, float b1, float b2,
                        float eps, int step, const int32_t* d_step, float* G, cudaStream_t stream);

size_t densify_ws_bytes(int n);
cudaError_t launch_densify(const sgs_gaussians& in, const float* S, const float* S_po, const float* S_ls, float inv_T,
                           float eps_split,
                           float step_scale, const float* grad_norm, float eps_grad, int64_t max_splits,
                           const sgs_gaussians_mut& out, int64_t capacity, int32_t* d_n_out,
                           int32_t* parent, float* lam_out, float* v_out, void* ws,
                           cudaStream_t stream);

// Generic device-side primitives (sort.cu)
// Exclusive scan of n uint32 values (n read from *d_n when d_n != nullptr,
// else n_host), writing out[i] and *d_total.  `tmp` needs scan_tmp_bytes(n_max).
size_t scan_tmp_bytes(int64_t n_max);
cudaError_t launch_exclusive_scan(const uint32_t* in, uint32_t* out, uint32_t* d_total,
                                  int64_t n_max, const int32_t* d_n, void* tmp, cudaStream_t stream);
// The same scan of n values whose producer already wrote the sum of every
// 256-value block (bcount[b] = sum of in[256 b, 256 b + 256)), so that no
// reduction pass over `in` is needed.
cudaError_t launch_exclusive_scan_counted(const uint32_t* in, uint32_t* out, uint32_t* d_total, int64_t n,
                                          const uint32_t* bcount, void* tmp, cudaStream_t stream);

constexpr size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Carves aligned sub-buffers out of one workspace.
struct Carver {
    char* base;
    size_t off;
    template <class T>
    T* take(size_t count) {
        off = align_up(off, 256);
        T* p = reinterpret_cast<T*>(base + off);
        off += sizeof(T) * count;
        return p;
    }
};

}  // namespace sgs
