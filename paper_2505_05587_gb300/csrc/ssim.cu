// SSIM term of the photometric loss (Section 3, Eq. loss: 3D Gaussian
// Splatting trains on (1 - lambda) L1 + lambda (1 - SSIM); the paper's
// analysis keeps only L1).  SSIM per channel after Wang et al. (2004): local
// means, variances and covariance under an 11x11 Gaussian window (sigma 1.5,
// zero padding), C1 = 0.01^2, C2 = 0.03^2, averaged over pixels and channels.
//
// Two kernels over 32x8 pixel blocks with a 5-pixel halo staged in shared
// memory; the separable window is applied as a horizontal then a vertical
// 11-tap pass.
//  1. moments: the five filtered moments per channel -> SSIM map S; the loss
//     terms (sum |x - y|, sum S) and three coefficient maps, the derivatives
//     of S with respect to the filtered x, x^2 and x y:
//        a = S (2 mu_y / A1 - 2 mu_x / B1) + (S / B2)(2 mu_x) - (2 S / A2) mu_y
//        b = -S / B2,   c = 2 S / A2
//  2. gradient: the window is symmetric and zero padded, hence its own
//     adjoint:  d mean(S) / dx = (F a + 2 x F b + y F c) / (3 H W); combined
//     with the L1 sign term and the view normalisation.
#include "common.cuh"

namespace sgs {

constexpr int SS_W = 32, SS_H = 8, SS_R = 5, SS_TAPS = 2 * SS_R + 1;
constexpr int SS_RW = SS_W + 2 * SS_R, SS_RH = SS_H + 2 * SS_R;   // 42 x 18 staged region
constexpr float SS_C1 = 0.01f * 0.01f, SS_C2 = 0.03f * 0.03f;

// Normalised taps of the 1-D Gaussian (sigma 1.5), computed by each block.
__device__ __forceinline__ void ssim_taps(float* taps) {
    if (threadIdx.x < SS_TAPS) {
        const float r = (float)((int)threadIdx.x - SS_R);
        taps[threadIdx.x] = expf(-r * r / (2.0f * 1.5f * 1.5f));
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        float s = 0.0f;
        for (int k = 0; k < SS_TAPS; ++k) s += taps[k];
        for (int k = 0; k < SS_TAPS; ++k) taps[k] /= s;
    }
    __syncthreads();
}

__device__ __forceinline__ float block_sum(float v, float* s_part) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) s_part[threadIdx.x >> 5] = v;
    __syncthreads();
    float s = 0.0f;
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += s_part[w];
    __syncthreads();
    return s;
}

__global__ void __launch_bounds__(SS_W * SS_H) ssim_moments_kernel(const float* __restrict__ image,
                                                                   const float* __restrict__ target, int H, int W,
                                                                   float lam, float inv_views,
                                                                   float* __restrict__ coef, float* __restrict__ loss) {
    pdl_wait_and_trigger();
    __shared__ float taps[SS_TAPS];
    __shared__ float sx[3][SS_RH][SS_RW];
    __shared__ float sy[3][SS_RH][SS_RW];
    __shared__ float hor[5][SS_RH][SS_W];
    __shared__ float s_part[8];
    ssim_taps(taps);
    const int bx = blockIdx.x * SS_W, by = blockIdx.y * SS_H;
    for (int k = threadIdx.x; k < SS_RH * SS_RW; k += SS_W * SS_H) {
        const int ry = k / SS_RW, rx = k - ry * SS_RW;
        const int gy = by - SS_R + ry, gx = bx - SS_R + rx;
        const bool in = gy >= 0 && gy < H && gx >= 0 && gx < W;
        const size_t p = in ? 3 * ((size_t)gy * W + gx) : 0;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            sx[c][ry][rx] = in ? image[p + c] : 0.0f;
            sy[c][ry][rx] = in ? target[p + c] : 0.0f;
        }
    }
    __syncthreads();
    const int tx = threadIdx.x % SS_W, ty = threadIdx.x / SS_W;
    const int px = bx + tx, py = by + ty;
    const bool inside = px < W && py < H;
    const size_t P = (size_t)H * W;
    float l1 = 0.0f, ssum = 0.0f;
    for (int c = 0; c < 3; ++c) {
        for (int k = threadIdx.x; k < SS_RH * SS_W; k += SS_W * SS_H) {
            const int ry = k / SS_W, cx = k - ry * SS_W;
            float m0 = 0.f, m1 = 0.f, m2 = 0.f, m3 = 0.f, m4 = 0.f;
#pragma unroll
            for (int t = 0; t < SS_TAPS; ++t) {
                const float a = sx[c][ry][cx + t], b = sy[c][ry][cx + t], w = taps[t];
                m0 += w * a;
                m1 += w * b;
                m2 += w * a * a;
                m3 += w * b * b;
                m4 += w * a * b;
            }
            hor[0][ry][cx] = m0;
            hor[1][ry][cx] = m1;
            hor[2][ry][cx] = m2;
            hor[3][ry][cx] = m3;
            hor[4][ry][cx] = m4;
        }
        __syncthreads();
        float mx = 0.f, my = 0.f, exx = 0.f, eyy = 0.f, exy = 0.f;
#pragma unroll
        for (int t = 0; t < SS_TAPS; ++t) {
            const float w = taps[t];
            mx += w * hor[0][ty + t][tx];
            my += w * hor[1][ty + t][tx];
            exx += w * hor[2][ty + t][tx];
            eyy += w * hor[3][ty + t][tx];
            exy += w * hor[4][ty + t][tx];
        }
        if (inside) {
            const float sxx = exx - mx * mx, syy = eyy - my * my, sxy = exy - mx * my;
            const float A1 = 2.0f * mx * my + SS_C1, A2 = 2.0f * sxy + SS_C2;
            const float B1 = mx * mx + my * my + SS_C1, B2 = sxx + syy + SS_C2;
            const float S = (A1 * A2) / (B1 * B2);
            const float b = -S / B2, cc = 2.0f * S / A2;
            const float a = S * (2.0f * my / A1 - 2.0f * mx / B1) - 2.0f * mx * b - my * cc;
            const size_t pix = (size_t)py * W + px;
            coef[(size_t)(3 * c + 0) * P + pix] = a;
            coef[(size_t)(3 * c + 1) * P + pix] = b;
            coef[(size_t)(3 * c + 2) * P + pix] = cc;
            ssum += S;
            l1 += fabsf(sx[c][ty + SS_R][tx + SS_R] - sy[c][ty + SS_R][tx + SS_R]);
        }
        __syncthreads();                             // hor is reused by the next channel
    }
    const float norm = 1.0f / (3.0f * (float)P);
    const float bl1 = block_sum(l1, s_part);
    const float bs = block_sum(ssum, s_part);
    if (threadIdx.x == 0) {
        float add = ((1.0f - lam) * bl1 * norm - lam * bs * norm) * inv_views;
        if (blockIdx.x == 0 && blockIdx.y == 0) add += lam * inv_views;     // the constant of 1 - SSIM
        atomicAdd(loss, add);
    }
}

__global__ void __launch_bounds__(SS_W * SS_H) ssim_grad_kernel(const float* __restrict__ image,
                                                                const float* __restrict__ target, int H, int W,
                                                                float lam, float inv_views,
                                                                const float* __restrict__ coef,
                                                                float* __restrict__ dL) {
    pdl_wait_and_trigger();
    __shared__ float taps[SS_TAPS];
    __shared__ float sm[3][SS_RH][SS_RW];
    __shared__ float hor[3][SS_RH][SS_W];
    ssim_taps(taps);
    const int bx = blockIdx.x * SS_W, by = blockIdx.y * SS_H;
    const int tx = threadIdx.x % SS_W, ty = threadIdx.x / SS_W;
    const int px = bx + tx, py = by + ty;
    const bool inside = px < W && py < H;
    const size_t P = (size_t)H * W;
    const float norm = 1.0f / (3.0f * (float)P);
    for (int c = 0; c < 3; ++c) {
        for (int k = threadIdx.x; k < SS_RH * SS_RW; k += SS_W * SS_H) {
            const int ry = k / SS_RW, rx = k - ry * SS_RW;
            const int gy = by - SS_R + ry, gx = bx - SS_R + rx;
            const bool in = gy >= 0 && gy < H && gx >= 0 && gx < W;
            const size_t pix = in ? (size_t)gy * W + gx : 0;
#pragma unroll
            for (int q = 0; q < 3; ++q) sm[q][ry][rx] = in ? coef[(size_t)(3 * c + q) * P + pix] : 0.0f;
        }
        __syncthreads();
        for (int k = threadIdx.x; k < SS_RH * SS_W; k += SS_W * SS_H) {
            const int ry = k / SS_W, cx = k - ry * SS_W;
            float h0 = 0.f, h1 = 0.f, h2 = 0.f;
#pragma unroll
            for (int t = 0; t < SS_TAPS; ++t) {
                const float w = taps[t];
                h0 += w * sm[0][ry][cx + t];
                h1 += w * sm[1][ry][cx + t];
                h2 += w * sm[2][ry][cx + t];
            }
            hor[0][ry][cx] = h0;
            hor[1][ry][cx] = h1;
            hor[2][ry][cx] = h2;
        }
        __syncthreads();
        if (inside) {
            float fa = 0.f, fb = 0.f, fc = 0.f;
#pragma unroll
            for (int t = 0; t < SS_TAPS; ++t) {
                const float w = taps[t];
                fa += w * hor[0][ty + t][tx];
                fb += w * hor[1][ty + t][tx];
                fc += w * hor[2][ty + t][tx];
            }
            const size_t k = 3 * ((size_t)py * W + px) + c;
            const float x = image[k], y = target[k];
            const float dssim = (fa + 2.0f * x * fb + y * fc) * norm;
            const float r = x - y;
            const float sg = r > 0.0f ? 1.0f : (r < 0.0f ? -1.0f : 0.0f);
            dL[k] = ((1.0f - lam) * sg * norm - lam * dssim) * inv_views;
        }
        __syncthreads();                             // sm / hor are reused by the next channel
    }
}

size_t ssim_ws_bytes(int H, int W) { return sizeof(float) * 9 * (size_t)H * (size_t)W + 256; }

cudaError_t launch_ssim_l1(const float* image, const float* target, int H, int W, int n_views, float lam, float* dL,
                           float* loss, void* ws, cudaStream_t stream) {
    if (H == 0 || W == 0) return cudaSuccess;
    float* coef = reinterpret_cast<float*>(ws);
    const dim3 grid((W + SS_W - 1) / SS_W, (H + SS_H - 1) / SS_H);
    const float inv_views = 1.0f / (float)n_views;
    (void)launch_pdl(ssim_moments_kernel, dim3(grid), dim3(SS_W * SS_H), 0, stream, image, target, H, W, lam,
                     inv_views, coef, loss);
    note_launch();
    (void)launch_pdl(ssim_grad_kernel, dim3(grid), dim3(SS_W * SS_H), 0, stream, image, target, H, W, lam, inv_views,
                     coef, dL);
    note_launch();
    return cudaGetLastError();
}

}  // namespace sgs
