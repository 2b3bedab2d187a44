// Tile rasteriser: forward front-to-back compositing and its back-to-front
// adjoint fused with the splitting-matrix accumulation.
//
// Paper: Section 3, Eq. alpha_blend (C = sum_i c_i T_i sigma_i, T_i =
// prod_{j<i} (1 - sigma_j)) and Eq. sigma_2D; Section 4.4 / Algorithm 1 (the
// splitting matrix S = E[dl/dsigma Hess_p sigma] accumulated during
// back-propagation); Appendix "Deriving Hessian of Gaussian".
//
// One CTA per tile of TW x TH pixels, one thread per pixel.  Gaussian records
// of the tile's depth-sorted list are staged in shared memory in batches of
// TW*TH (one coalesced 16-byte load per field per thread).
#include "common.cuh"

namespace sgs {

// Row of the per-Gaussian 2-D accumulator buffer (16 floats, 4 float4 atomics):
//  0 dL/dmu_x   1 dL/dmu_y   2 dL/dQ00   3 dL/dQ01 (shared off-diagonal)
//  4 dL/dQ11    5 dL/do      6..8 dL/drgb
//  9 a0 = sum w   10..12 A2 = sum w u u^T (xx, xy, yy)   13..15 unused
constexpr int kG2dStride = 16;

template <int TW, int TH>
__global__ void __launch_bounds__(TW * TH) render_fwd_kernel(
    const uint2* __restrict__ ranges, const uint32_t* __restrict__ gids, const float4* __restrict__ xy,
    const float4* __restrict__ conic_opac, const float4* __restrict__ rgb, int W, int H, int gx, SetDev st,
    float* __restrict__ image, float* __restrict__ final_T, uint32_t* __restrict__ n_contrib) {
    constexpr int BS = TW * TH;
    __shared__ float4 s_xy[BS];
    __shared__ float4 s_co[BS];
    __shared__ float4 s_rgb[BS];
    const int tile = blockIdx.x;
    const int px = (tile % gx) * TW + (int)(threadIdx.x % TW);
    const int py = (tile / gx) * TH + (int)(threadIdx.x / TW);
    const bool inside = px < W && py < H;
    const float fpx = (float)px, fpy = (float)py;
    const uint2 rg = ranges[tile];
    const int n = (int)(rg.y - rg.x);
    bool done = !inside;
    float T = 1.0f, C0 = 0.0f, C1 = 0.0f, C2 = 0.0f;
    uint32_t last = 0;
    for (int base = 0; base < n; base += BS) {
        if (__syncthreads_count(done) == BS) break;
        const int k = base + (int)threadIdx.x;
        if (k < n) {
            const uint32_t g = gids[rg.x + k];
            s_xy[threadIdx.x] = xy[g];
            s_co[threadIdx.x] = conic_opac[g];
            s_rgb[threadIdx.x] = rgb[g];
        }
        __syncthreads();
        const int cnt = min(BS, n - base);
        for (int j = 0; !done && j < cnt; ++j) {
            const float4 m = s_xy[j];
            const float4 co = s_co[j];
            const float dx = (fpx - m.x) - m.z;
            const float dy = (fpy - m.y) - m.w;
            const float power = -0.5f * (co.x * dx * dx + co.z * dy * dy) - co.y * dx * dy;
            const float alpha = fminf(st.alpha_max, co.w * __expf(power));
            if (alpha < st.alpha_min) continue;
            const float Tn = T * (1.0f - alpha);
            if (Tn < st.T_min) {
                done = true;
                break;
            }
            const float4 c = s_rgb[j];
            const float wgt = alpha * T;
            C0 += c.x * wgt;
            C1 += c.y * wgt;
            C2 += c.z * wgt;
            T = Tn;
            last = (uint32_t)(base + j + 1);
        }
    }
    if (inside) {
        const int pix = py * W + px;
        image[3 * pix] = C0 + T * st.bg[0];
        image[3 * pix + 1] = C1 + T * st.bg[1];
        image[3 * pix + 2] = C2 + T * st.bg[2];
        final_T[pix] = T;
        n_contrib[pix] = last;
    }
}

// Pair counts of the forward walk, per pixel: (pairs evaluated, pairs
// composited).  A measurement aid; it replays the walk without colour.
template <int TW, int TH>
__global__ void __launch_bounds__(TW * TH) render_stats_kernel(
    const uint2* __restrict__ ranges, const uint32_t* __restrict__ gids, const float4* __restrict__ xy,
    const float4* __restrict__ conic_opac, int W, int H, int gx, SetDev st, uint2* __restrict__ counts) {
    const int tile = blockIdx.x;
    const int px = (tile % gx) * TW + (int)(threadIdx.x % TW);
    const int py = (tile / gx) * TH + (int)(threadIdx.x / TW);
    if (px >= W || py >= H) return;
    const uint2 rg = ranges[tile];
    float T = 1.0f;
    uint32_t ev = 0, comp = 0;
    for (uint32_t k = rg.x; k < rg.y; ++k) {
        const uint32_t g = gids[k];
        const float4 m = xy[g];
        const float4 co = conic_opac[g];
        const float dx = ((float)px - m.x) - m.z;
        const float dy = ((float)py - m.y) - m.w;
        const float power = -0.5f * (co.x * dx * dx + co.z * dy * dy) - co.y * dx * dy;
        const float alpha = fminf(st.alpha_max, co.w * __expf(power));
        ++ev;
        if (alpha < st.alpha_min) continue;
        const float Tn = T * (1.0f - alpha);
        if (Tn < st.T_min) break;
        ++comp;
        T = Tn;
    }
    counts[py * W + px] = make_uint2(ev, comp);
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

template <int TW, int TH>
__global__ void __launch_bounds__(TW * TH) render_bwd_kernel(
    const uint2* __restrict__ ranges, const uint32_t* __restrict__ gids, const float4* __restrict__ xy,
    const float4* __restrict__ conic_opac, const float4* __restrict__ rgb, int W, int H, int gx, SetDev st,
    const float* __restrict__ final_T, const uint32_t* __restrict__ n_contrib,
    const float* __restrict__ dL_dimage, float* __restrict__ g2d) {
    constexpr int BS = TW * TH;
    __shared__ uint32_t s_gid[BS];
    __shared__ float4 s_xy[BS];
    __shared__ float4 s_co[BS];
    __shared__ float4 s_rgb[BS];
    __shared__ uint32_t s_max;
    const int tile = blockIdx.x;
    const int px = (tile % gx) * TW + (int)(threadIdx.x % TW);
    const int py = (tile / gx) * TH + (int)(threadIdx.x / TW);
    const bool inside = px < W && py < H;
    const float fpx = (float)px, fpy = (float)py;
    const int pix = py * W + px;
    const uint2 rg = ranges[tile];
    const int lane = threadIdx.x & 31;

    float T = inside ? final_T[pix] : 1.0f;
    const uint32_t last = inside ? n_contrib[pix] : 0u;
    const float g0 = inside ? dL_dimage[3 * pix] : 0.0f;
    const float g1 = inside ? dL_dimage[3 * pix + 1] : 0.0f;
    const float g2 = inside ? dL_dimage[3 * pix + 2] : 0.0f;
    float acc0 = st.bg[0], acc1 = st.bg[1], acc2 = st.bg[2];

    if (threadIdx.x == 0) s_max = 0u;
    __syncthreads();
    {
        uint32_t m = __reduce_max_sync(0xffffffffu, last);
        if (lane == 0) atomicMax(&s_max, m);
    }
    __syncthreads();
    const int maxl = min((int)s_max, (int)(rg.y - rg.x));

    for (int end = maxl; end > 0; end -= BS) {
        const int start = max(0, end - BS);
        __syncthreads();
        const int k = start + (int)threadIdx.x;
        if (k < end) {
            const uint32_t g = gids[rg.x + k];
            s_gid[threadIdx.x] = g;
            s_xy[threadIdx.x] = xy[g];
            s_co[threadIdx.x] = conic_opac[g];
            s_rgb[threadIdx.x] = rgb[g];
        }
        __syncthreads();
        for (int j = end - 1; j >= start; --j) {
            const int jj = j - start;
            bool valid = inside && (uint32_t)j < last;
            float v0 = 0.f, v1 = 0.f, v2 = 0.f, v3 = 0.f, v4 = 0.f, v5 = 0.f, v6 = 0.f, v7 = 0.f;
            float v8 = 0.f, v9 = 0.f, v10 = 0.f, v11 = 0.f, v12 = 0.f;
            if (valid) {
                const float4 m = s_xy[jj];
                const float4 co = s_co[jj];
                const float dx = (fpx - m.x) - m.z;
                const float dy = (fpy - m.y) - m.w;
                const float power = -0.5f * (co.x * dx * dx + co.z * dy * dy) - co.y * dx * dy;
                const float G = __expf(power);
                const float araw = co.w * G;
                const bool clamped = !(araw < st.alpha_max);
                const float alpha = clamped ? st.alpha_max : araw;
                if (alpha < st.alpha_min) {
                    valid = false;
                } else {
                    const float4 c = s_rgb[jj];
                    const float one_m = 1.0f - alpha;
                    T = __fdividef(T, one_m);            // transmittance in front of this Gaussian
                    const float dLda = T * (g0 * (c.x - acc0) + g1 * (c.y - acc1) + g2 * (c.z - acc2));
                    acc0 = alpha * c.x + one_m * acc0;
                    acc1 = alpha * c.y + one_m * acc1;
                    acc2 = alpha * c.z + one_m * acc2;
                    const float aT = alpha * T;
                    v6 = g0 * aT;
                    v7 = g1 * aT;
                    v8 = g2 * aT;
                    if (!clamped) {
                        const float w = dLda * alpha;          // dL/dsigma * sigma
                        const float ux = co.x * dx + co.y * dy;  // u = Q (x - mu)
                        const float uy = co.y * dx + co.z * dy;
                        v0 = w * ux;
                        v1 = w * uy;
                        v2 = -0.5f * w * dx * dx;
                        v3 = -w * dx * dy;
                        v4 = -0.5f * w * dy * dy;
                        v5 = dLda * G;
                        v9 = w;
                        v10 = w * ux * ux;
                        v11 = w * ux * uy;
                        v12 = w * uy * uy;
                    }
                }
            }
            if (__any_sync(0xffffffffu, valid)) {
                v0 = warp_sum(v0); v1 = warp_sum(v1); v2 = warp_sum(v2); v3 = warp_sum(v3);
                v4 = warp_sum(v4); v5 = warp_sum(v5); v6 = warp_sum(v6); v7 = warp_sum(v7);
                v8 = warp_sum(v8); v9 = warp_sum(v9); v10 = warp_sum(v10); v11 = warp_sum(v11);
                v12 = warp_sum(v12);
                if (lane == 0) {
                    float4* row = reinterpret_cast<float4*>(g2d + (size_t)s_gid[jj] * kG2dStride);
                    atomicAdd(row, make_float4(v0, v1, v2, v3));
                    atomicAdd(row + 1, make_float4(v4, v5, v6, v7));
                    atomicAdd(row + 2, make_float4(v8, v9, v10, v11));
                    atomicAdd(row + 3, make_float4(v12, 0.f, 0.f, 0.f));
                }
            }
        }
    }
}

template <int TW, int TH>
static cudaError_t stats_tmpl(const sgs_proj& proj, const sgs_bins& bins, const CamDev& cam, const SetDev& st,
                              uint32_t* counts, cudaStream_t stream) {
    const int T = cam.gx * cam.gy;
    render_stats_kernel<TW, TH><<<T, TW * TH, 0, stream>>>(
        reinterpret_cast<const uint2*>(bins.ranges), bins.gids, reinterpret_cast<const float4*>(proj.xy),
        reinterpret_cast<const float4*>(proj.conic_opac), cam.width, cam.height, cam.gx, st,
        reinterpret_cast<uint2*>(counts));
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_render_stats(const sgs_proj& proj, const sgs_bins& bins, const CamDev& cam, const SetDev& st,
                                uint32_t* counts, cudaStream_t stream) {
    if (st.tile_w == 16 && st.tile_h == 16) return stats_tmpl<16, 16>(proj, bins, cam, st, counts, stream);
    if (st.tile_w == 16 && st.tile_h == 8) return stats_tmpl<16, 8>(proj, bins, cam, st, counts, stream);
    if (st.tile_w == 8 && st.tile_h == 8) return stats_tmpl<8, 8>(proj, bins, cam, st, counts, stream);
    if (st.tile_w == 32 && st.tile_h == 8) return stats_tmpl<32, 8>(proj, bins, cam, st, counts, stream);
    return cudaErrorInvalidValue;
}

template <int TW, int TH>
static cudaError_t fwd_tmpl(const sgs_proj& proj, const sgs_bins& bins, const CamDev& cam, const SetDev& st,
                            float* image, float* final_T, uint32_t* n_contrib, cudaStream_t stream) {
    const int T = cam.gx * cam.gy;
    render_fwd_kernel<TW, TH><<<T, TW * TH, 0, stream>>>(
        reinterpret_cast<const uint2*>(bins.ranges), bins.gids, reinterpret_cast<const float4*>(proj.xy),
        reinterpret_cast<const float4*>(proj.conic_opac), reinterpret_cast<const float4*>(proj.rgb),
        cam.width, cam.height, cam.gx, st, image, final_T, n_contrib);
    note_launch();
    return cudaGetLastError();
}

template <int TW, int TH>
static cudaError_t bwd_tmpl(const sgs_proj& proj, const sgs_bins& bins, const CamDev& cam, const SetDev& st,
                            const float* final_T, const uint32_t* n_contrib, const float* dL, float* g2d,
                            cudaStream_t stream) {
    const int T = cam.gx * cam.gy;
    render_bwd_kernel<TW, TH><<<T, TW * TH, 0, stream>>>(
        reinterpret_cast<const uint2*>(bins.ranges), bins.gids, reinterpret_cast<const float4*>(proj.xy),
        reinterpret_cast<const float4*>(proj.conic_opac), reinterpret_cast<const float4*>(proj.rgb),
        cam.width, cam.height, cam.gx, st, final_T, n_contrib, dL, g2d);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_render_fwd(const sgs_proj& proj, const sgs_bins& bins, const CamDev& cam, const SetDev& st,
                              float* image, float* final_T, uint32_t* n_contrib, cudaStream_t stream) {
    if (st.tile_w == 16 && st.tile_h == 16) return fwd_tmpl<16, 16>(proj, bins, cam, st, image, final_T, n_contrib, stream);
    if (st.tile_w == 16 && st.tile_h == 8) return fwd_tmpl<16, 8>(proj, bins, cam, st, image, final_T, n_contrib, stream);
    if (st.tile_w == 8 && st.tile_h == 8) return fwd_tmpl<8, 8>(proj, bins, cam, st, image, final_T, n_contrib, stream);
    if (st.tile_w == 32 && st.tile_h == 8) return fwd_tmpl<32, 8>(proj, bins, cam, st, image, final_T, n_contrib, stream);
    return cudaErrorInvalidValue;
}

cudaError_t launch_render_bwd(const sgs_proj& proj, const sgs_bins& bins, const CamDev& cam, const SetDev& st,
                              const float* final_T, const uint32_t* n_contrib, const float* dL, float* g2d,
                              cudaStream_t stream) {
    if (st.tile_w == 16 && st.tile_h == 16) return bwd_tmpl<16, 16>(proj, bins, cam, st, final_T, n_contrib, dL, g2d, stream);
    if (st.tile_w == 16 && st.tile_h == 8) return bwd_tmpl<16, 8>(proj, bins, cam, st, final_T, n_contrib, dL, g2d, stream);
    if (st.tile_w == 8 && st.tile_h == 8) return bwd_tmpl<8, 8>(proj, bins, cam, st, final_T, n_contrib, dL, g2d, stream);
    if (st.tile_w == 32 && st.tile_h == 8) return bwd_tmpl<32, 8>(proj, bins, cam, st, final_T, n_contrib, dL, g2d, stream);
    return cudaErrorInvalidValue;
}

}  // namespace sgs
