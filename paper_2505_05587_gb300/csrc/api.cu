// C ABI of libsteepgs (declarations and contracts: include/steepgs.h).
// Host-side argument checks, workspace carving and kernel launches only.
#include <math.h>
#include <string.h>

#include <atomic>

#include "common.cuh"

namespace sgs {

bool tile_supported(int tw, int th) {
    return (tw == 16 && th == 16) || (tw == 16 && th == 8) || (tw == 8 && th == 8) || (tw == 32 && th == 8);
}

CamDev make_cam(const sgs_camera& c, const sgs_settings& s) {
    CamDev d;
    memcpy(d.R, c.R, sizeof(d.R));
    memcpy(d.t, c.t, sizeof(d.t));
    d.fx = c.fx; d.fy = c.fy; d.cx = c.cx; d.cy = c.cy;
    d.width = c.width; d.height = c.height;
    d.near_z = c.near_z;
    d.limx = (s.fov_clamp * (0.5f * (float)c.width)) / c.fx;
    d.limy = (s.fov_clamp * (0.5f * (float)c.height)) / c.fy;
    for (int k = 0; k < 3; ++k) {
        double v = -((double)c.R[k] * c.t[0] + (double)c.R[3 + k] * c.t[1] + (double)c.R[6 + k] * c.t[2]);
        d.cc[k] = (float)v;
    }
    d.gx = (c.width + s.tile_w - 1) / s.tile_w;
    d.gy = (c.height + s.tile_h - 1) / s.tile_h;
    return d;
}

ViewsDev make_views(const sgs_camera* cams, int nv, const sgs_settings& s, const int* rows_per_view, int rows_each) {
    ViewsDev vd;
    memset(&vd, 0, sizeof(vd));
    vd.nv = nv;
    int t = 0, r = 0;
    long long p = 0;
    for (int v = 0; v < nv; ++v) {
        vd.cam[v] = make_cam(cams[v], s);
        vd.tile_off[v] = t;
        vd.pix_off[v] = p;
        vd.row_off[v] = r;
        t += vd.cam[v].gx * vd.cam[v].gy;
        p += (long long)cams[v].width * cams[v].height;
        r += rows_per_view ? rows_per_view[v] : rows_each;
    }
    vd.tile_off[nv] = t;
    vd.pix_off[nv] = p;
    vd.row_off[nv] = r;
    vd.T_total = t;
    vd.P_total = p;
    return vd;
}

ScenesDev make_scenes(const sgs_gaussians* g, int nv, bool per_view) {
    ScenesDev sc;
    memset(&sc, 0, sizeof(sc));
    for (int v = 0; v < nv; ++v) {
        const sgs_gaussians& gv = per_view ? g[v] : g[0];
        sc.means[v] = gv.means;
        sc.log_scales[v] = gv.log_scales;
        sc.quats[v] = gv.quats;
        sc.opacity_logit[v] = gv.opacity_logit;
        sc.sh[v] = gv.sh;
    }
    return sc;
}

SetDev make_set(const sgs_settings& s) {
    SetDev d;
    d.tile_w = s.tile_w; d.tile_h = s.tile_h;
    d.alpha_min = s.alpha_min; d.alpha_max = s.alpha_max; d.T_min = s.T_min;
    d.radius_sigma = s.radius_sigma; d.dilation = s.dilation; d.fov_clamp = s.fov_clamp;
    d.bg[0] = s.bg[0]; d.bg[1] = s.bg[1]; d.bg[2] = s.bg[2];
    return d;
}

static thread_local int g_last_cuda = 0;
static std::atomic<unsigned long long> g_launches{0};

void note_launch(int k) { g_launches.fetch_add((unsigned long long)k, std::memory_order_relaxed); }

int record_cuda_error(cudaError_t e) {
    g_last_cuda = (int)e;
    return SGS_ERR_CUDA;
}

static int cuda_status(cudaError_t e) {
    if (e == cudaSuccess) return SGS_OK;
    return record_cuda_error(e);
}

static bool valid_cam(const sgs_camera* c) {
    return c && c->width > 0 && c->height > 0 && c->width <= 32767 * 8 && c->height <= 32767 * 8 &&
           isfinite(c->fx) && isfinite(c->fy) && c->fx > 0.0f && c->fy > 0.0f;
}

static bool valid_settings(const sgs_settings* s) {
    return s && tile_supported(s->tile_w, s->tile_h) && s->alpha_max > 0.0f && s->alpha_max <= 1.0f &&
           s->alpha_min >= 0.0f && s->T_min >= 0.0f && s->radius_sigma > 0.0f && s->dilation >= 0.0f &&
           s->fov_clamp > 0.0f;
}

static bool valid_gaussians(const sgs_gaussians* g) {
    if (!g || g->n < 0 || g->sh_degree < 0 || g->sh_degree > kMaxShDegree) return false;
    if (g->n == 0) return true;
    return g->means && g->log_scales && g->quats && g->opacity_logit && g->sh;
}

static bool tiles_fit(const sgs_camera* c, const sgs_settings* s) {
    int64_t gx = (c->width + s->tile_w - 1) / s->tile_w;
    int64_t gy = (c->height + s->tile_h - 1) / s->tile_h;
    return gx <= 32767 && gy <= 32767 && gx * gy < (int64_t)1 << 31;
}

}  // namespace sgs

using namespace sgs;

extern "C" {

const char* sgs_error_string(int status) {
    switch (status) {
        case SGS_OK: return "ok";
        case SGS_ERR_INVALID_ARG: return "invalid argument";
        case SGS_ERR_WORKSPACE: return "workspace too small";
        case SGS_ERR_CAPACITY: return "capacity exceeded";
        case SGS_ERR_CUDA: return "CUDA error";
        case SGS_ERR_TIMEOUT: return "timeout";
        case SGS_ERR_UNSUPPORTED: return "unsupported";
        default: return "unknown status";
    }
}

int sgs_get_last_cuda_error(void) { return g_last_cuda; }

int sgs_version(void) { return 100; }

uint64_t sgs_kernel_launches(void) { return (uint64_t)g_launches.load(std::memory_order_relaxed); }

int sgs_clear(void* dst, size_t bytes, void* stream) {
    SGS_NVTX_RANGE();
    if (bytes == 0) return SGS_OK;
    if (!dst) return SGS_ERR_INVALID_ARG;
    return cuda_status(cudaMemsetAsync(dst, 0, bytes, (cudaStream_t)stream));
}

int sgs_project(const sgs_gaussians* g, const sgs_camera* cam, const sgs_settings* st, const sgs_proj* out,
                void* stream) {
    SGS_NVTX_RANGE();
    if (!valid_gaussians(g) || !valid_cam(cam) || !valid_settings(st) || !out || !tiles_fit(cam, st))
        return SGS_ERR_INVALID_ARG;
    if (g->n > 0 && (!out->xy || !out->conic_opac || !out->rgb || !out->depth || !out->rect || !out->tiles_touched))
        return SGS_ERR_INVALID_ARG;
    return cuda_status(launch_project(make_scenes(g, 1, false), g->sh_degree, make_views(cam, 1, *st, nullptr, g->n),
                                      make_set(*st), *out, (cudaStream_t)stream));
}

int sgs_bin_sort_workspace_size(int32_t n, int64_t capacity, int32_t num_tiles, size_t* bytes) {
    if (n < 0 || capacity < 0 || num_tiles <= 0 || !bytes || capacity > ((int64_t)1 << 31) - 1)
        return SGS_ERR_INVALID_ARG;
    *bytes = bin_sort_ws_bytes(n, capacity, num_tiles);
    return SGS_OK;
}

int sgs_bin_sort(const sgs_proj* proj, int32_t n, const sgs_camera* cam, const sgs_settings* st,
                 const sgs_bins* out, void* ws, size_t ws_bytes, void* stream) {
    SGS_NVTX_RANGE();
    if (!proj || n < 0 || !valid_cam(cam) || !valid_settings(st) || !out || !tiles_fit(cam, st))
        return SGS_ERR_INVALID_ARG;
    if (!out->ranges || !out->count || out->capacity < 0 || out->capacity > ((int64_t)1 << 31) - 1)
        return SGS_ERR_INVALID_ARG;
    if (out->capacity > 0 && !out->gids) return SGS_ERR_INVALID_ARG;
    if (n > 0 && (!proj->depth || !proj->rect || !proj->tiles_touched)) return SGS_ERR_INVALID_ARG;
    ViewsDev vd = make_views(cam, 1, *st, nullptr, n);
    if (!ws || ws_bytes < bin_sort_ws_bytes(n, out->capacity, vd.T_total)) return SGS_ERR_WORKSPACE;
    return cuda_status(launch_bin_sort(*proj, vd, make_set(*st), *out, ws, (cudaStream_t)stream));
}

// Walk lists come as a pair (both given or both NULL), with a capacity whose
// rows (warps per tile x capacity) fit a 64-bit index.
static bool walk_ok(const sgs_bins* b) {
    if ((b->walk == nullptr) != (b->walk_count == nullptr)) return false;
    return b->walk == nullptr || (b->capacity >= 0 && b->capacity <= ((int64_t)1 << 31) - 1);
}

int sgs_render_fwd(const sgs_proj* proj, const sgs_bins* bins, const sgs_camera* cam, const sgs_settings* st,
                   float* image, float* final_T, uint32_t* n_contrib, void* stream) {
    SGS_NVTX_RANGE();
    if (!proj || !bins || !valid_cam(cam) || !valid_settings(st) || !image || !final_T || !n_contrib ||
        !tiles_fit(cam, st) || !bins->ranges || !walk_ok(bins))
        return SGS_ERR_INVALID_ARG;
    return cuda_status(launch_render_fwd(*proj, *bins, make_cam(*cam, *st), make_set(*st), image, final_T,
                                         n_contrib, nullptr, 1, nullptr, nullptr, (cudaStream_t)stream));
}

int sgs_render_fwd_l1(const sgs_proj* proj, const sgs_bins* bins, const sgs_camera* cam, const sgs_settings* st,
                      const float* target, int32_t n_views, float* image, float* final_T, uint32_t* n_contrib,
                      float* dL_dimage, float* loss, void* stream) {
    SGS_NVTX_RANGE();
    if (!proj || !bins || !valid_cam(cam) || !valid_settings(st) || !image || !final_T || !n_contrib ||
        !tiles_fit(cam, st) || !bins->ranges || !walk_ok(bins) || !target || n_views <= 0 || !dL_dimage || !loss)
        return SGS_ERR_INVALID_ARG;
    return cuda_status(launch_render_fwd(*proj, *bins, make_cam(*cam, *st), make_set(*st), image, final_T,
                                         n_contrib, target, n_views, dL_dimage, loss, (cudaStream_t)stream));
}

int sgs_render_stats(const sgs_proj* proj, const sgs_bins* bins, const sgs_camera* cam, const sgs_settings* st,
                     uint32_t* counts, uint32_t* warp_union, void* stream) {
    SGS_NVTX_RANGE();
    if (!proj || !bins || !valid_cam(cam) || !valid_settings(st) || !counts || !tiles_fit(cam, st) ||
        !bins->ranges)
        return SGS_ERR_INVALID_ARG;
    return cuda_status(launch_render_stats(*proj, *bins, make_cam(*cam, *st), make_set(*st), counts, warp_union,
                                           (cudaStream_t)stream));
}

int sgs_ssim_l1_workspace_size(int32_t height, int32_t width, size_t* bytes) {
    if (height < 0 || width < 0 || !bytes) return SGS_ERR_INVALID_ARG;
    *bytes = ssim_ws_bytes(height, width);
    return SGS_OK;
}

int sgs_ssim_l1_loss_grad(const float* image, const float* target, int32_t height, int32_t width, int32_t n_views,
                          float lambda_dssim, float* dL_dimage, float* loss, void* ws, size_t ws_bytes,
                          void* stream) {
    SGS_NVTX_RANGE();
    if (!image || !target || height <= 0 || width <= 0 || n_views <= 0 || !dL_dimage || !loss ||
        !(lambda_dssim >= 0.0f && lambda_dssim <= 1.0f))
        return SGS_ERR_INVALID_ARG;
    if (!ws || ws_bytes < ssim_ws_bytes(height, width)) return SGS_ERR_WORKSPACE;
    return cuda_status(launch_ssim_l1(image, target, height, width, n_views, lambda_dssim, dL_dimage, loss, ws,
                                      (cudaStream_t)stream));
}

int sgs_fma_probe(float* out, int32_t blocks, int32_t iters, void* stream) {
    SGS_NVTX_RANGE();
    if (!out || blocks <= 0 || iters <= 0) return SGS_ERR_INVALID_ARG;
    return cuda_status(launch_fma_probe(out, blocks, iters, (cudaStream_t)stream));
}

int sgs_l1_loss_grad(const float* image, const float* target, int32_t height, int32_t width, int32_t n_views,
                     float* dL_dimage, float* loss, void* stream) {
    SGS_NVTX_RANGE();
    if (!image || !target || height <= 0 || width <= 0 || n_views <= 0 || !dL_dimage || !loss)
        return SGS_ERR_INVALID_ARG;
    return cuda_status(launch_l1(image, target, height, width, n_views, dL_dimage, loss, (cudaStream_t)stream));
}

// Backward workspace: per Gaussian a 16-float accumulator row, and a second
// one for the higher moments of the log-scale blocks (used when S_ls_accum is
// given).
int sgs_render_bwd_workspace_size(int32_t n, size_t* bytes) {
    if (n < 0 || !bytes) return SGS_ERR_INVALID_ARG;
    *bytes = sizeof(float) * 32 * (size_t)(n > 0 ? n : 1) + 256;
    return SGS_OK;
}

int sgs_render_bwd_with_splitting(const sgs_gaussians* g, const sgs_proj* proj, const sgs_bins* bins,
                                  const sgs_camera* cam, const sgs_settings* st, const float* final_T,
                                  const uint32_t* n_contrib, const float* dL_dimage, const sgs_grads* grads,
                                  int32_t flags, float* S_accum, float* S_po_accum, float* S_ls_accum,
                                  void* ws, size_t ws_bytes, void* stream) {
    SGS_NVTX_RANGE();
    if (flags & ~(SGS_BWD_ACCUMULATE_GRADS | SGS_BWD_RESET_S)) return SGS_ERR_INVALID_ARG;
    if (!valid_gaussians(g) || !proj || !bins || !valid_cam(cam) || !valid_settings(st) || !final_T ||
        !n_contrib || !dL_dimage || !grads || !tiles_fit(cam, st) || !bins->ranges || !walk_ok(bins))
        return SGS_ERR_INVALID_ARG;
    if (S_ls_accum && !S_po_accum) return SGS_ERR_INVALID_ARG;      // theta = (p, l, o) includes o
    if (g->n > 0 && (!grads->means || !grads->log_scales || !grads->quats || !grads->opacity_logit ||
                     !grads->sh || !S_accum))
        return SGS_ERR_INVALID_ARG;
    size_t need = 0;
    sgs_render_bwd_workspace_size(g->n, &need);
    if (!ws || ws_bytes < need) return SGS_ERR_WORKSPACE;
    if (g->n == 0) return SGS_OK;
    cudaStream_t s = (cudaStream_t)stream;
    float* g2d = reinterpret_cast<float*>(align_up(reinterpret_cast<uintptr_t>(ws), 256));
    if ((char*)g2d + sizeof(float) * 32 * (size_t)g->n > (char*)ws + ws_bytes) return SGS_ERR_WORKSPACE;
    float* g2d_hi = S_ls_accum ? g2d + 16 * (size_t)g->n : nullptr;
    CamDev cd = make_cam(*cam, *st);
    SetDev sd = make_set(*st);
    cudaError_t e = launch_zero_reached_rows(proj->tiles_touched, g->n, g2d, g2d_hi, s);
    if (e == cudaSuccess)
        e = launch_render_bwd(*proj, *bins, cd, sd, final_T, n_contrib, dL_dimage, g2d, g2d_hi, s);
    if (e == cudaSuccess)
        e = launch_project_bwd(*g, *proj, make_views(cam, 1, *st, nullptr, g->n), g2d, g2d_hi, flags, *grads,
                               S_accum, S_po_accum, S_ls_accum, s);
    return cuda_status(e);
}

int sgs_adam_step(float* param, const float* grad, float* m, float* v, int64_t count, float lr, float beta1,
                  float beta2, float eps, int32_t step, float* grad_accum, void* stream) {
    SGS_NVTX_RANGE();
    if (count < 0 || step < 1 || !(lr >= 0.0f) || !(beta1 >= 0.0f && beta1 < 1.0f) ||
        !(beta2 >= 0.0f && beta2 < 1.0f) || !(eps > 0.0f))
        return SGS_ERR_INVALID_ARG;
    if (count > 0 && (!param || !grad || !m || !v)) return SGS_ERR_INVALID_ARG;
    return cuda_status(launch_adam(param, grad, m, v, count, lr, beta1, beta2, eps, step, nullptr, grad_accum,
                                   (cudaStream_t)stream));
}

int sgs_adam_step_dev(float* param, const float* grad, float* m, float* v, int64_t count, float lr, float beta1,
                      float beta2, float eps, const int32_t* d_step, float* grad_accum, void* stream) {
    SGS_NVTX_RANGE();
    if (count < 0 || !d_step || !(lr >= 0.0f) || !(beta1 >= 0.0f && beta1 < 1.0f) ||
        !(beta2 >= 0.0f && beta2 < 1.0f) || !(eps > 0.0f))
        return SGS_ERR_INVALID_ARG;
    if (count > 0 && (!param || !grad || !m || !v)) return SGS_ERR_INVALID_ARG;
    return cuda_status(launch_adam(param, grad, m, v, count, lr, beta1, beta2, eps, 1, d_step, grad_accum,
                                   (cudaStream_t)stream));
}

// ---------------------------------------------------------------------------
// Several views in one pass
// ---------------------------------------------------------------------------
struct ViewsWs {
    sgs_proj proj;
    sgs_bins bins;
    void* sort_ws;
    size_t sort_bytes;
    float* final_T;
    uint32_t* n_contrib;
    float* dL;
    float* g2d;
    uint32_t* counters;
    WalkLists wl;
    size_t bytes;
};

// The workspace of a multi-view pass.  With the backward it also holds the
// forward's walk lists (warps per tile x capacity entries, and a count per
// warp of every tile), which the backward then follows.
static ViewsWs carve_views_ws(void* base, const ViewsDev& vd, int64_t capacity, bool with_backward, int nw = 8) {
    Carver c{reinterpret_cast<char*>(base), 0};
    ViewsWs w{};
    const size_t rows = (size_t)(vd.row_off[vd.nv] > 0 ? vd.row_off[vd.nv] : 1);
    const size_t P = (size_t)(vd.P_total > 0 ? vd.P_total : 1);
    const size_t cap = (size_t)(capacity > 0 ? capacity : 1);
    w.proj.xy = c.take<float>(4 * rows);
    w.proj.conic_opac = c.take<float>(4 * rows);
    w.proj.rgb = c.take<float>(4 * rows);
    w.proj.depth = c.take<float>(rows);
    w.proj.rect = c.take<int16_t>(4 * rows);
    w.proj.tiles_touched = c.take<uint32_t>(rows);
    w.bins.gids = c.take<uint32_t>(cap);
    w.bins.keys = nullptr;
    w.bins.ranges = c.take<uint32_t>(2 * (size_t)vd.T_total);
    w.bins.count = nullptr;
    w.bins.capacity = capacity;
    w.bins.order = c.take<uint32_t>((size_t)(vd.T_total > 0 ? vd.T_total : 1));
    w.sort_bytes = bin_sort_ws_bytes((int)rows, capacity, vd.T_total);
    w.sort_ws = c.take<char>(w.sort_bytes);
    w.final_T = c.take<float>(P);
    w.n_contrib = c.take<uint32_t>(P);
    w.dL = with_backward ? c.take<float>(3 * P) : nullptr;
    w.g2d = with_backward ? c.take<float>(16 * rows) : nullptr;
    w.counters = c.take<uint32_t>(2);
    if (with_backward) {
        w.wl.cap = (long long)nw * (long long)cap;
        w.wl.walk = c.take<uint32_t>((size_t)w.wl.cap);
        w.wl.count = c.take<uint32_t>((size_t)nw * (size_t)(vd.T_total > 0 ? vd.T_total : 1));
    }
    w.bytes = c.off + 256;
    return w;
}

static bool valid_views(const sgs_camera* cams, int32_t n_views, const sgs_settings* st) {
    if (!cams || n_views < 1 || n_views > kMaxViews || !valid_settings(st)) return false;
    long long tiles = 0;
    for (int v = 0; v < n_views; ++v) {
        if (!valid_cam(&cams[v]) || !tiles_fit(&cams[v], st)) return false;
        tiles += (long long)((cams[v].width + st->tile_w - 1) / st->tile_w) *
                 ((cams[v].height + st->tile_h - 1) / st->tile_h);
    }
    return tiles < ((long long)1 << 31);
}

int sgs_render_views_workspace_size(int32_t n, const sgs_camera* cams, int32_t n_views, const sgs_settings* st,
                                    int64_t capacity, size_t* bytes) {
    if (n < 0 || capacity < 0 || capacity > ((int64_t)1 << 31) - 1 || !bytes || !valid_views(cams, n_views, st) ||
        (long long)n * n_views > ((long long)1 << 31) - 1)
        return SGS_ERR_INVALID_ARG;
    ViewsDev vd = make_views(cams, n_views, *st, nullptr, n);
    *bytes = carve_views_ws(nullptr, vd, capacity, true, st->tile_w * st->tile_h / 32).bytes;
    return SGS_OK;
}

int sgs_render_views_bins(int32_t n, const sgs_camera* cams, int32_t n_views, const sgs_settings* st,
                          int64_t capacity, void* ws, size_t ws_bytes, sgs_bins* out) {
    if (n < 0 || capacity < 0 || capacity > ((int64_t)1 << 31) - 1 || !out || !valid_views(cams, n_views, st) ||
        (long long)n * n_views > ((long long)1 << 31) - 1)
        return SGS_ERR_INVALID_ARG;
    ViewsDev vd = make_views(cams, n_views, *st, nullptr, n);
    const int nw = st->tile_w * st->tile_h / 32;
    ViewsWs w = carve_views_ws(nullptr, vd, capacity, true, nw);
    if (!ws || ws_bytes < w.bytes) return SGS_ERR_WORKSPACE;
    w = carve_views_ws(ws, vd, capacity, true, nw);
    *out = w.bins;
    return SGS_OK;
}

int sgs_render_views_with_splitting(const sgs_gaussians* g, const sgs_camera* cams, int32_t n_views,
                                    const sgs_settings* st, int32_t batch, const float* targets, float* images,
                                    float* loss, const sgs_grads* grads, int32_t flags, float* S_accum,
                                    float* S_po_accum,
                                    int32_t* d_count, int64_t capacity, void* ws, size_t ws_bytes, void* stream) {
    SGS_NVTX_RANGE();
    if (flags & ~(SGS_BWD_ACCUMULATE_GRADS | SGS_BWD_RESET_S)) return SGS_ERR_INVALID_ARG;
    if (!valid_gaussians(g) || !valid_views(cams, n_views, st) || !targets || !images || !loss || !grads ||
        !d_count || capacity < 0 || capacity > ((int64_t)1 << 31) - 1 ||
        (long long)g->n * n_views > ((long long)1 << 31) - 1)
        return SGS_ERR_INVALID_ARG;
    if (batch == 0) batch = st->tile_w * st->tile_h > 256 ? 256 : st->tile_w * st->tile_h;
    if (batch != 64 && batch != 128 && batch != 256) return SGS_ERR_INVALID_ARG;
    if (g->n > 0 && (!grads->means || !grads->log_scales || !grads->quats || !grads->opacity_logit || !grads->sh ||
                     !S_accum))
        return SGS_ERR_INVALID_ARG;
    ViewsDev vd = make_views(cams, n_views, *st, nullptr, g->n);
    const int nw = st->tile_w * st->tile_h / 32;
    ViewsWs w = carve_views_ws(nullptr, vd, capacity, true, nw);
    if (!ws || ws_bytes < w.bytes) return SGS_ERR_WORKSPACE;
    w = carve_views_ws(ws, vd, capacity, true, nw);
    w.bins.count = d_count;
    const SetDev sd = make_set(*st);
    cudaStream_t s = (cudaStream_t)stream;
    const size_t rows = (size_t)g->n * n_views;
    cudaError_t e = launch_project(make_scenes(g, n_views, false), g->sh_degree, vd, sd, w.proj, s);
    if (e == cudaSuccess) e = launch_bin_sort(w.proj, vd, sd, w.bins, w.sort_ws, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(w.counters, 0, 2 * sizeof(uint32_t), s);
    if (e == cudaSuccess)
        e = launch_render_fwd_views(vd, w.proj, w.bins.ranges, w.bins.gids, sd, batch, images, w.final_T,
                                    w.n_contrib, w.counters, w.bins.order, w.wl, s);
    if (e == cudaSuccess) e = launch_l1_views(images, targets, vd, w.dL, loss, s);
    // the backward adds into the accumulator rows of reached (view, Gaussian)
    // pairs only, and the adjoint reads only those: clear just them
    if (e == cudaSuccess) e = launch_zero_reached_rows(w.proj.tiles_touched, (int)rows, w.g2d, nullptr, s);
    if (e == cudaSuccess)
        e = launch_render_bwd_views(vd, w.proj, w.bins.ranges, w.bins.gids, sd, batch, w.final_T, w.n_contrib,
                                    w.dL, w.g2d, w.counters + 1, w.bins.order, w.wl, s);
    if (e == cudaSuccess)
        e = launch_project_bwd(*g, w.proj, vd, w.g2d, nullptr, flags, *grads, S_accum, S_po_accum, nullptr, s);
    return cuda_status(e);
}

// Forward-only batch of views whose scenes may differ (render serving).
static bool valid_batch(const sgs_gaussians* scenes, const sgs_camera* cams, int32_t n_views,
                        const sgs_settings* st, int rows[kMaxViews]) {
    if (!scenes || !valid_views(cams, n_views, st)) return false;
    long long total = 0;
    for (int v = 0; v < n_views; ++v) {
        if (!valid_gaussians(&scenes[v]) || scenes[v].sh_degree != scenes[0].sh_degree) return false;
        rows[v] = scenes[v].n;
        total += scenes[v].n;
    }
    return total < ((long long)1 << 31);
}

int sgs_render_batch_workspace_size(const sgs_gaussians* scenes, const sgs_camera* cams, int32_t n_views,
                                    const sgs_settings* st, int64_t capacity, size_t* bytes) {
    int rows[kMaxViews];
    if (!bytes || capacity < 0 || capacity > ((int64_t)1 << 31) - 1 || !valid_batch(scenes, cams, n_views, st, rows))
        return SGS_ERR_INVALID_ARG;
    ViewsDev vd = make_views(cams, n_views, *st, rows, 0);
    *bytes = carve_views_ws(nullptr, vd, capacity, false).bytes;
    return SGS_OK;
}

int sgs_render_batch_fwd(const sgs_gaussians* scenes, const sgs_camera* cams, int32_t n_views, const sgs_settings* st,
                         int32_t batch, float* images, int32_t* d_count, int64_t capacity, void* ws, size_t ws_bytes,
                         void* stream) {
    SGS_NVTX_RANGE();
    int rows[kMaxViews];
    if (!images || !d_count || capacity < 0 || capacity > ((int64_t)1 << 31) - 1 ||
        !valid_batch(scenes, cams, n_views, st, rows))
        return SGS_ERR_INVALID_ARG;
    if (batch == 0) batch = st->tile_w * st->tile_h > 256 ? 256 : st->tile_w * st->tile_h;
    if (batch != 64 && batch != 128 && batch != 256) return SGS_ERR_INVALID_ARG;
    ViewsDev vd = make_views(cams, n_views, *st, rows, 0);
    ViewsWs w = carve_views_ws(nullptr, vd, capacity, false);
    if (!ws || ws_bytes < w.bytes) return SGS_ERR_WORKSPACE;
    w = carve_views_ws(ws, vd, capacity, false);
    w.bins.count = d_count;
    const SetDev sd = make_set(*st);
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = launch_project(make_scenes(scenes, n_views, true), scenes[0].sh_degree, vd, sd, w.proj, s);
    if (e == cudaSuccess) e = launch_bin_sort(w.proj, vd, sd, w.bins, w.sort_ws, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(w.counters, 0, sizeof(uint32_t), s);
    if (e == cudaSuccess)
        e = launch_render_fwd_views(vd, w.proj, w.bins.ranges, w.bins.gids, sd, batch, images, w.final_T,
                                    w.n_contrib, w.counters, w.bins.order, WalkLists{nullptr, nullptr, 0}, s);
    return cuda_status(e);
}

int sgs_densify_split_workspace_size(int32_t n, size_t* bytes) {
    if (n < 0 || !bytes) return SGS_ERR_INVALID_ARG;
    *bytes = densify_ws_bytes(n);
    return SGS_OK;
}

int sgs_densify_split(const sgs_gaussians* in, const float* S_accum, const float* S_po_accum,
                      const float* S_ls_accum, float inv_T_split, float eps_split, float step_scale,
                      const float* grad_norm, float eps_grad, int64_t max_splits,
                      const sgs_gaussians_mut* out, int64_t capacity, int32_t* d_n_out, int32_t* parent_index,
                      float* lam_min_out, float* v_min_out, void* ws, size_t ws_bytes, void* stream) {
    SGS_NVTX_RANGE();
    if (!valid_gaussians(in) || !out || !d_n_out || capacity < in->n || !isfinite(inv_T_split) ||
        !isfinite(step_scale))
        return SGS_ERR_INVALID_ARG;
    if (in->n > 0 && (!S_accum || !out->means || !out->log_scales || !out->quats || !out->opacity_logit ||
                      !out->sh))
        return SGS_ERR_INVALID_ARG;
    if (in->n > 0 && (out->means == in->means || out->sh == in->sh || out->opacity_logit == in->opacity_logit))
        return SGS_ERR_INVALID_ARG;
    if (S_ls_accum && !S_po_accum) return SGS_ERR_INVALID_ARG;
    if (!ws || ws_bytes < densify_ws_bytes(in->n)) return SGS_ERR_WORKSPACE;
    return cuda_status(launch_densify(*in, S_accum, S_po_accum, S_ls_accum, inv_T_split, eps_split, step_scale, grad_norm,
                                      eps_grad, max_splits, *out, capacity, d_n_out, parent_index, lam_min_out,
                                      v_min_out, ws, (cudaStream_t)stream));
}

}  // extern "C"
