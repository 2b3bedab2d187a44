// Tile rasteriser: forward front-to-back compositing and its back-to-front
// adjoint fused with the splitting-matrix accumulation.
//
// Paper: Section 3, Eq. alpha_blend (C = sum_i c_i T_i sigma_i, T_i =
// prod_{j<i} (1 - sigma_j)) and Eq. sigma_2D; Section 4.4 / Algorithm 1 (the
// splitting matrix S = E[dl/dsigma Hess_p sigma] accumulated during
// back-propagation); Appendix "Deriving Hessian of Gaussian".
//
// A CTA renders a tile of TW x TH pixels, one thread per pixel, warps on 8x4
// pixel blocks.  Gaussian records of the tile's depth-sorted list are staged in
// shared memory in batches of BATCH (coalesced 16-byte loads per field); each
// warp then walks only the batch entries whose alpha support meets its block
// (an exact skip: outside that support alpha < alpha_min).  Single-view
// kernels launch one CTA per tile; the multi-view kernels are persistent and
// pull global tiles of all views from an atomic counter.  Both take their
// tiles in the schedule bin_sort writes (longest lists first), so that the
// heaviest tiles do not run alone at the end of a launch.  The forward can
// carry the L1 loss in its epilogue.
#include "common.cuh"

namespace sgs {

// Row of the per-Gaussian 2-D accumulator buffer (16 floats, slots 9..15
// unused; one 9-lane vector of atomics per warp and Gaussian).  With
// w = dL/dalpha * alpha for unclamped composited pairs (0 otherwise) and
// d = x - mu:
//  0..1 sum w d            (dL/dmu = Q sum w d)
//  2..4 D = sum w d d^T    (xx, xy, yy): dL/dQ = -D/2, and the splitting
//                          accumulator sum w u u^T = Q D Q with u = Q d
//  5    a0 = sum w         (dL/do = a0 / o)
//  6..8 dL/drgb = sum g alpha T
constexpr int kG2dStride = 16;

// Staged conic in base-2 exponent form: G = 2^(dx (A dx + B dy) + C dy^2)
// with (A, B, C) = -log2(e) (Q00/2, Q01, Q11/2); w = opacity.
__device__ __forceinline__ float4 conic_exp2(float4 co) {
    constexpr float L2E = 1.4426950408889634f;
    return make_float4(-0.5f * L2E * co.x, -L2E * co.y, -0.5f * L2E * co.z, co.w);
}

__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// 2-D Gaussian value at offset (dx, dy) from the staged exponent form.  The
// operations are spelled out so that the forward and backward kernels compute
// the same bits (their skip and clamp decisions must agree).
__device__ __forceinline__ float gauss2(float4 cp, float dx, float dy) {
    const float t = __fmaf_rn(cp.y, dy, __fmul_rn(cp.x, dx));
    return ex2_approx(__fmaf_rn(dx, t, __fmul_rn(__fmul_rn(cp.z, dy), dy)));
}

// Pixel of a thread: warps cover 8x4 pixel blocks of the tile (lane -> 8
// columns x 4 rows), so that a warp can skip, as a whole, every Gaussian whose
// alpha support misses its block.
template <int TW>
__device__ __forceinline__ void warp_block_origin(int tile, int gx, int TH_, int* bx, int* by) {
    const int warp = threadIdx.x >> 5;
    *bx = (tile % gx) * TW + (warp % (TW / 8)) * 8;
    *by = (tile / gx) * TH_ + (warp / (TW / 8)) * 4;
}

// Per column strip of a tile (the 8 pixel-centre columns of one column of
// warp blocks, NS = TW / 8 strips), the rows where alpha = o G can reach
// alpha_min.  That region is the ellipse d^T Q d <= M, M = 2 ln(o /
// alpha_min); its part inside a strip is convex, so its rows form one
// interval and a warp's 8x4 block meets the region iff the block's rows meet
// its strip's interval (an exact test, where an axis-aligned box of the whole
// ellipse also passes blocks in the box's empty corners).  On the ellipse's
// boundary at column offset u, dy = (-b u +- sqrt(c M - det u^2)) / c; the
// upper branch (concave) peaks at the ellipse's top, u_t = -b e_y / a with
// e_y = sqrt(M a / det), the lower branch (convex) bottoms out at -u_t, so
// the interval's ends are the branches at u_t and -u_t clamped into the
// strip.  Conservative against float32 rounding, including that of the
// compositing kernels' own evaluation of d^T Q d at a pixel (cancellation
// there is at most about 16 eps (a + c)^2 / det of M near the boundary): M
// is widened by that term and 1e-3 relative, the strips and intervals by
// 0.01 pixel, and det = ac - b^2 is taken with the rounding error of b^2
// compensated.  Empty intervals when o < alpha_min; whole columns when
// alpha_min = 0 or the conic is not positive definite.  yr[s * stride] gets
// strip s's interval (lo, hi) in view rows.
template <int NS>
__device__ __forceinline__ void alpha_support_strips(float4 m, float4 co, float alpha_min, float ox, float2* yr,
                                                     int stride) {
    const float o = co.w;
    const float a = co.x, b = co.y, c = co.z;
    const float bb = b * b;
    const float det = __fmaf_rn(a, c, -bb) - __fmaf_rn(b, b, -bb);
    if (!(o >= alpha_min)) {
#pragma unroll
        for (int s = 0; s < NS; ++s) yr[s * stride] = make_float2(1e30f, -1e30f);
        return;
    }
    if (!(alpha_min > 0.0f) || !(det > 0.0f) || !(a > 0.0f) || !(c > 0.0f)) {
#pragma unroll
        for (int s = 0; s < NS; ++s) yr[s * stride] = make_float2(-1e30f, 1e30f);
        return;
    }
    const float sa = a + c;
    const float M = 2.0f * logf(o / alpha_min) * (1.001f + 1e-6f * (sa * sa / det)) + 1e-3f;
    const float cM = c * M, ic = 1.0f / c;
    const float ex = sqrtf(cM / det);
    const float ut = -b * sqrtf(M * a / det) / a;
    const float cx = m.x + m.z, cy = m.y + m.w;
#pragma unroll
    for (int s = 0; s < NS; ++s) {
        const float xa = (ox + (float)(8 * s)) - cx - 0.01f, xb = xa + 7.02f;
        float2 r = make_float2(1e30f, -1e30f);
        if (xb >= -ex && xa <= ex) {
            const float u = fminf(fmaxf(ut, xa), xb);
            const float v = fminf(fmaxf(-ut, xa), xb);
            const float hi = (sqrtf(fmaxf(0.0f, cM - det * u * u)) - b * u) * ic;
            const float lo = (-sqrtf(fmaxf(0.0f, cM - det * v * v)) - b * v) * ic;
            r = make_float2(cy + lo - 0.01f, cy + hi + 0.01f);
        }
        yr[s * stride] = r;
    }
}

// Order-preserving list of the batch entries [0, cnt) whose support meets the
// warp's pixel rows [by, by+3] within its strip (s_yr: the strip's intervals).
// Returns the list length.
__device__ __forceinline__ int build_warp_list(const float2* s_yr, int cnt, float by, uint8_t* list) {
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    int nl = 0;
    for (int c = 0; c < cnt; c += 32) {
        const int e = c + lane;
        bool hit = false;
        if (e < cnt) {
            const float2 r = s_yr[e];
            hit = r.y >= by && r.x <= by + 3.0f;
        }
        const unsigned m = __ballot_sync(0xffffffffu, hit);
        if (hit) list[nl + __popc(m & lt)] = (uint8_t)e;
        nl += __popc(m);
    }
    __syncwarp();
    return nl;
}


template <int BATCH, int NW, int NS>
struct FwdSmem {
    float2 xy[BATCH];      // mean relative to the tile origin
    float4 co[BATCH];
    float4 rgb[BATCH];
    float2 yr[NS][BATCH];  // per column strip: rows of the alpha support
    uint8_t list[NW][BATCH];
    uint8_t hit[NW][BATCH];  // walk recording: list slot composited by some pixel of the warp
    float l1_part[NW];
};

// L1 loss fused into the forward epilogue: dL = sign(C - target) norm,
// loss += norm sum |C - target|, norm = 1 / (3 H W n_views).
struct L1Out {
    const float* target;
    float* dL;
    float* loss;
    float norm;
};

// Per-warp transposed reduction buffer of the backward pass: 18 rows of the
// warp's 32 per-pixel values (9 per entry, two entries per flush; or the 18
// values of one entry with the higher moments), each row padded to 36 floats
// so that the writes (one row per value, a lane per column) and the 16-byte
// reads of the summing lanes (a row per lane) are free of bank conflicts.
constexpr int kRedRows = 18;
constexpr int kRedStride = 36;
// Half rows of the walk backward: after one shuffle exchange between lanes
// 16 apart, each of the nine values of an entry is carried by 16 lanes; rows
// of 16 floats on a 20-float stride keep both the writes (rows j and j + 4
// from the two lane halves at once) and the 16-byte row reads conflict-free.
constexpr int kHalfStride = 20;

template <int BATCH, int NW, int NS>
struct BwdSmem {
    uint32_t gid[BATCH];
    float2 xy[BATCH];      // mean relative to the tile origin
    float4 co[BATCH];
    float4 rgb[BATCH];
    float2 yr[NS][BATCH];  // per column strip: rows of the alpha support
    uint8_t list[NW][BATCH];
    uint32_t maxl;
    alignas(16) float red[NW][kRedRows * kRedStride];
};

// Forward compositing of one tile (local tile id `tile` in a gx-wide grid of a
// W x H view); outputs are the view's own image / final_T / n_contrib arrays.
// Walk lists written by the forward pass (REC): for warp w of a tile with list
// [start, end), entries NW*start + w*(end - start) on of `walk` hold the list
// positions it composited in some pixel, front to back; walk_count[tile*NW + w]
// their number.
struct WalkOut {
    uint32_t* walk;
    uint32_t* count;
    long long cap;          // entries of walk
};

template <int TW, int TH, int BATCH, bool REC = false>
__device__ __forceinline__ void fwd_tile(int tile, int gx, int W, int H, uint2 rg, const uint32_t* __restrict__ gids,
                                         const float4* __restrict__ xy, const float4* __restrict__ conic_opac,
                                         const float4* __restrict__ rgb, const SetDev& st, float* __restrict__ image,
                                         float* __restrict__ final_T, uint32_t* __restrict__ n_contrib,
                                         FwdSmem<BATCH, TW * TH / 32, TW / 8>& sm, const L1Out* l1 = nullptr,
                                         WalkOut wo = WalkOut{nullptr, nullptr, 0}) {
    constexpr int NW = TW * TH / 32;
    constexpr int BS = TW * TH;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int bx, by;
    warp_block_origin<TW>(tile, gx, TH, &bx, &by);
    const int px = bx + (lane & 7);
    const int py = by + (lane >> 3);
    const bool inside = px < W && py < H;
    // offsets from the tile origin: the staged mean is tile-local, so a pair's
    // offset is one subtraction (same bits in the forward and the backward)
    const int ox = (tile % gx) * TW, oy = (tile / gx) * TH;
    const float lx = (float)(px - ox), ly = (float)(py - oy);
    const int n = (int)(rg.y - rg.x);
    bool done = !inside;
    float T = 1.0f, C0 = 0.0f, C1 = 0.0f, C2 = 0.0f;
    uint32_t last = 0;
    uint32_t* wp = nullptr;                         // this warp's list
    uint32_t wroom = 0;                             // rows left in `walk` from wp on
    uint32_t wcnt = 0;                              // entries recorded by this warp
    if constexpr (REC) {
        const long long wbase = (long long)NW * rg.x + (long long)warp * n;
        wp = wo.walk + wbase;
        wroom = (uint32_t)max(0LL, min(wo.cap - wbase, (long long)n));
        for (int k = threadIdx.x; k < NW * BATCH; k += BS) (&sm.hit[0][0])[k] = 0;   // read after a barrier
    }
    for (int base = 0; base < n; base += BATCH) {
        if (__syncthreads_count(done) == BS) break;
        const int cnt = min(BATCH, n - base);
        for (int k = threadIdx.x; k < cnt; k += BS) {
            const uint32_t g = gids[rg.x + base + k];
            const float4 m = xy[g];
            const float4 co = conic_opac[g];
            sm.xy[k] = make_float2((m.x - (float)ox) + m.z, (m.y - (float)oy) + m.w);
            sm.co[k] = conic_exp2(co);
            sm.rgb[k] = rgb[g];
            alpha_support_strips<TW / 8>(m, co, st.alpha_min, (float)ox, &sm.yr[0][k], BATCH);
        }
        __syncthreads();
        if (__all_sync(0xffffffffu, done)) continue;
        const int nl = build_warp_list(sm.yr[warp % (TW / 8)], cnt, (float)by, sm.list[warp]);
        for (int k = 0; k < nl && !done; ++k) {
            const int j = sm.list[warp][k];
            const float2 m = sm.xy[j];
            const float4 cp = sm.co[j];
            const float dx = lx - m.x;
            const float dy = ly - m.y;
            const float alpha = fminf(st.alpha_max, __fmul_rn(cp.w, gauss2(cp, dx, dy)));
            if (alpha < st.alpha_min) continue;
            const float Tn = T * (1.0f - alpha);
            if (Tn < st.T_min) {
                done = true;
                break;
            }
            const float4 c = sm.rgb[j];
            const float wgt = alpha * T;
            C0 += c.x * wgt;
            C1 += c.y * wgt;
            C2 += c.z * wgt;
            T = Tn;
            last = (uint32_t)(base + j + 1);
            if constexpr (REC) sm.hit[warp][k] = 1;  // lanes at one k store the same byte
        }
        if constexpr (REC) {                        // append the composited slots, in list order
            __syncwarp();
            const unsigned lt = (1u << lane) - 1u;
            for (int c = 0; c < nl; c += 32) {
                const int k = c + lane;
                const bool h = k < nl && sm.hit[warp][k] != 0;
                const unsigned m = __ballot_sync(0xffffffffu, h);
                if (h) {
                    sm.hit[warp][k] = 0;
                    const uint32_t at = wcnt + __popc(m & lt);
                    if (at < wroom) wp[at] = (uint32_t)(base + sm.list[warp][k]);
                }
                wcnt += __popc(m);
            }
            __syncwarp();
        }
    }
    if constexpr (REC) {
        if (lane == 0) wo.count[(long long)tile * NW + warp] = wcnt;
    }
    float l1_sum = 0.0f;
    if (inside) {
        const int pix = py * W + px;
        const float c[3] = {C0 + T * st.bg[0], C1 + T * st.bg[1], C2 + T * st.bg[2]};
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) image[3 * pix + ch] = c[ch];
        final_T[pix] = T;
        n_contrib[pix] = last;
        if (l1) {                                   // the L1 loss and its gradient at this pixel
#pragma unroll
            for (int ch = 0; ch < 3; ++ch) {
                const float r = c[ch] - l1->target[3 * pix + ch];
                l1_sum += fabsf(r);
                l1->dL[3 * pix + ch] = r > 0.0f ? l1->norm : (r < 0.0f ? -l1->norm : 0.0f);
            }
        }
    }
    if (l1) {                                       // one atomic per tile for the loss
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) l1_sum += __shfl_xor_sync(0xffffffffu, l1_sum, o);
        if (lane == 0) sm.l1_part[warp] = l1_sum;
        __syncthreads();
        if (threadIdx.x == 0) {
            float t = 0.0f;
            for (int w = 0; w < BS / 32; ++w) t += sm.l1_part[w];
            if (t != 0.0f) atomicAdd(l1->loss, t * l1->norm);
        }
    }
    __syncthreads();        // shared memory is reused by the next tile
}

// Sum of the 32 floats of one 16-byte aligned row: eight 16-byte loads and a
// tree of packed two-lane float32 additions (add.rn.f32x2).
__device__ __forceinline__ unsigned long long add_f32x2(unsigned long long a, unsigned long long b) {
    unsigned long long d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

// Sum of the 16 floats of one 16-byte aligned row (four 16-byte loads).
__device__ __forceinline__ float row_sum16(const float* row) {
    const ulonglong2* r = reinterpret_cast<const ulonglong2*>(row);
    const ulonglong2 a = r[0], b = r[1], c = r[2], d = r[3];
    unsigned long long s0 = add_f32x2(add_f32x2(a.x, b.x), add_f32x2(c.x, d.x));
    const unsigned long long s1 = add_f32x2(add_f32x2(a.y, b.y), add_f32x2(c.y, d.y));
    s0 = add_f32x2(s0, s1);
    float lo, hi;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(s0));
    return lo + hi;
}

__device__ __forceinline__ float row_sum32(const float* row) {
    const ulonglong2* r = reinterpret_cast<const ulonglong2*>(row);
    unsigned long long s[8];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const ulonglong2 a = r[2 * k], b = r[2 * k + 1];
        s[2 * k] = add_f32x2(a.x, b.x);
        s[2 * k + 1] = add_f32x2(a.y, b.y);
    }
#pragma unroll
    for (int w = 4; w > 0; w >>= 1)
#pragma unroll
        for (int k = 0; k < w; ++k) s[k] = add_f32x2(s[k], s[k + w]);
    float lo, hi;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(s[0]));
    return lo + hi;
}

// Backward pass of one tile, back to front, with the splitting accumulators.
// HI: also the third and fourth moments of w d (the log-scale blocks of the
// splitting matrix over theta = (p, l, o)) into g2d_hi rows of kG2dStride:
//  0..3 sum w (dx^3, dx^2 dy, dx dy^2, dy^3), 4..8 sum w (dx^4, dx^3 dy,
//  dx^2 dy^2, dx dy^3, dy^4).
template <int TW, int TH, int BATCH, bool HI>
__device__ __forceinline__ void bwd_tile(int tile, int gx, int W, int H, uint2 rg, const uint32_t* __restrict__ gids,
                                         const float4* __restrict__ xy, const float4* __restrict__ conic_opac,
                                         const float4* __restrict__ rgb, const SetDev& st,
                                         const float* __restrict__ final_T, const uint32_t* __restrict__ n_contrib,
                                         const float* __restrict__ dL_dimage, float* __restrict__ g2d,
                                         float* __restrict__ g2d_hi, BwdSmem<BATCH, TW * TH / 32, TW / 8>& sm) {
    constexpr int BS = TW * TH;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int bx, by;
    warp_block_origin<TW>(tile, gx, TH, &bx, &by);
    const int px = bx + (lane & 7);
    const int py = by + (lane >> 3);
    const bool inside = px < W && py < H;
    const int ox = (tile % gx) * TW, oy = (tile / gx) * TH;
    const float lx = (float)(px - ox), ly = (float)(py - oy);
    const int pix = py * W + px;

    float T = inside ? final_T[pix] : 1.0f;
    const uint32_t last = inside ? n_contrib[pix] : 0u;
    const float g0 = inside ? dL_dimage[3 * pix] : 0.0f;
    const float g1 = inside ? dL_dimage[3 * pix + 1] : 0.0f;
    const float g2 = inside ? dL_dimage[3 * pix + 2] : 0.0f;
    float acc0 = st.bg[0], acc1 = st.bg[1], acc2 = st.bg[2];

    // transposed reduction: a reduced entry's per-pixel values go to rows of
    // this warp's buffer; every EPF entries (two, or one with the higher
    // moments) the first 18 lanes each sum one row and add it to the entry's
    // accumulator with one atomic
    constexpr int EPF = HI ? 1 : 2;
    float* red = sm.red[warp];
    int pend = 0;                       // entries waiting in the buffer (warp-uniform)
    uint32_t gid_a = 0u;                // the first waiting entry's Gaussian
    auto flush = [&](uint32_t gid_b, int rows) {
        __syncwarp();
        if (lane < rows) {
            const float t = row_sum32(red + lane * kRedStride);
            if constexpr (HI)
                atomicAdd((lane < 9 ? g2d : g2d_hi) + (size_t)gid_b * kG2dStride + (lane < 9 ? lane : lane - 9), t);
            else
                atomicAdd(g2d + (size_t)(lane < 9 ? gid_a : gid_b) * kG2dStride + (lane < 9 ? lane : lane - 9), t);
        }
        __syncwarp();
    };

    if (threadIdx.x == 0) sm.maxl = 0u;
    __syncthreads();
    // entries at or past a pixel's last contributor composite nothing there:
    // the tile walks up to the largest last of its pixels, each warp's list
    // stops at the largest last of its own pixels
    const int warp_last = (int)__reduce_max_sync(0xffffffffu, last);
    if (lane == 0) atomicMax(&sm.maxl, (uint32_t)warp_last);
    __syncthreads();
    const int maxl = min((int)sm.maxl, (int)(rg.y - rg.x));

    for (int end = maxl; end > 0; end -= BATCH) {
        const int start = max(0, end - BATCH);
        const int cnt = end - start;
        __syncthreads();
        for (int k = threadIdx.x; k < cnt; k += BS) {
            const uint32_t g = gids[rg.x + start + k];
            const float4 m = xy[g];
            const float4 co = conic_opac[g];
            sm.gid[k] = g;
            sm.xy[k] = make_float2((m.x - (float)ox) + m.z, (m.y - (float)oy) + m.w);
            sm.co[k] = conic_exp2(co);
            sm.rgb[k] = rgb[g];
            alpha_support_strips<TW / 8>(m, co, st.alpha_min, (float)ox, &sm.yr[0][k], BATCH);
        }
        __syncthreads();
        const int wcnt = min(cnt, warp_last - start);    // this warp's entries end at its last contributor
        const int nl = wcnt > 0 ? build_warp_list(sm.yr[warp % (TW / 8)], wcnt, (float)by, sm.list[warp]) : 0;
        for (int k = nl - 1; k >= 0; --k) {
            const int e = sm.list[warp][k];
            const float2 m = sm.xy[e];
            const float4 cp = sm.co[e];
            const float4 c = sm.rgb[e];
            const float dx = lx - m.x;
            const float dy = ly - m.y;
            const float araw = __fmul_rn(cp.w, gauss2(cp, dx, dy));
            const bool valid = inside && (uint32_t)(start + e) < last && araw >= st.alpha_min;
            if (!__any_sync(0xffffffffu, valid)) continue;     // nothing composited here by this warp
            const bool clamped = araw >= st.alpha_max;
            // branch-free: an invalid pair has alpha 0, leaving T, the colour
            // behind and every accumulated term unchanged
            const float ae = valid ? (clamped ? st.alpha_max : araw) : 0.0f;
            const float one_m = 1.0f - ae;
            T = __fdividef(T, one_m);                 // transmittance in front of this Gaussian
            const float dLda = T * (g0 * (c.x - acc0) + g1 * (c.y - acc1) + g2 * (c.z - acc2));
            acc0 += ae * (c.x - acc0);
            acc1 += ae * (c.y - acc1);
            acc2 += ae * (c.z - acc2);
            const float aT = ae * T;
            const float w = (clamped ? 0.0f : ae) * dLda;   // dL/dsigma * sigma
            const float wdx = w * dx, wdy = w * dy;
            float* rb = red + pend * 9 * kRedStride + lane;
            rb[0 * kRedStride] = wdx;
            rb[1 * kRedStride] = wdy;
            rb[2 * kRedStride] = wdx * dx;
            rb[3 * kRedStride] = wdx * dy;
            rb[4 * kRedStride] = wdy * dy;
            rb[5 * kRedStride] = w;
            rb[6 * kRedStride] = g0 * aT;
            rb[7 * kRedStride] = g1 * aT;
            rb[8 * kRedStride] = g2 * aT;
            if constexpr (HI) {
                const float wxx = wdx * dx, wyy = wdy * dy;
                rb[9 * kRedStride] = wxx * dx;
                rb[10 * kRedStride] = wxx * dy;
                rb[11 * kRedStride] = wyy * dx;
                rb[12 * kRedStride] = wyy * dy;
                rb[13 * kRedStride] = wxx * dx * dx;
                rb[14 * kRedStride] = wxx * dx * dy;
                rb[15 * kRedStride] = wxx * dy * dy;
                rb[16 * kRedStride] = wyy * dx * dy;
                rb[17 * kRedStride] = wyy * dy * dy;
            }
            const uint32_t gid = sm.gid[e];
            if (pend + 1 == EPF) {
                flush(gid, kRedRows);
                pend = 0;
            } else {
                gid_a = gid;
                ++pend;
            }
        }
    }
    if (pend > 0) flush(gid_a, 9);      // an odd entry left waiting (two-entry flushes only)
    __syncthreads();        // shared memory is reused by the next tile
}

// Backward pass of one tile over the forward pass's walk lists: each warp
// steps back to front through the entries it composited in some pixel (never
// the others), staging 32 of them at a time in its own shared-memory slots, so
// that the warps of a tile never wait for one another.  Per pixel, the
// transmittance is recovered by division and the compositing decision
// recomputed exactly as in bwd_tile.
template <int NW>
struct BwdWalkSmem {
    float4 ent[NW][3][32];  // per warp: (tile-local mean, gid bits, position bits), conic (exp2 form), colour
    alignas(16) float red[NW][kRedRows * kRedStride];
};

template <int TW, int TH, bool HI>
__device__ __forceinline__ void bwd_tile_walk(int tile, int wb, int gx, int W, int H, uint2 rg,
                                              const uint32_t* __restrict__ gids, const float4* __restrict__ xy,
                                              const float4* __restrict__ conic_opac, const float4* __restrict__ rgb,
                                              const SetDev& st, const float* __restrict__ final_T,
                                              const uint32_t* __restrict__ n_contrib,
                                              const float* __restrict__ dL_dimage, const uint32_t* __restrict__ walk,
                                              const uint32_t* __restrict__ walk_count, long long walk_cap,
                                              float* __restrict__ g2d, float* __restrict__ g2d_hi,
                                              BwdWalkSmem<TW * TH / 32>& sm) {
    constexpr int NW = TW * TH / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;   // `warp`: this warp's shared-memory slot
    const long long L = (long long)rg.y - (long long)rg.x;
    const long long wbase = (long long)NW * rg.x + (long long)wb * L;
    long long cnt = walk_count[(long long)tile * NW + wb];
    cnt = min(cnt, L);
    cnt = min(cnt, walk_cap - wbase);               // in bounds whatever the counts say
    if (cnt <= 0) return;
    const int bx = (tile % gx) * TW + (wb % (TW / 8)) * 8;   // the tile's 8x4 block wb
    const int by = (tile / gx) * TH + (wb / (TW / 8)) * 4;
    const int px = bx + (lane & 7);
    const int py = by + (lane >> 3);
    const bool inside = px < W && py < H;
    const int ox = (tile % gx) * TW, oy = (tile / gx) * TH;
    const float lx = (float)(px - ox), ly = (float)(py - oy);
    const int pix = py * W + px;
    float T = inside ? final_T[pix] : 1.0f;
    const uint32_t last = inside ? n_contrib[pix] : 0u;
    const float g0 = inside ? dL_dimage[3 * pix] : 0.0f;
    const float g1 = inside ? dL_dimage[3 * pix + 1] : 0.0f;
    const float g2 = inside ? dL_dimage[3 * pix + 2] : 0.0f;
    float acc0 = st.bg[0], acc1 = st.bg[1], acc2 = st.bg[2];

    float* red = sm.red[warp];
    uint32_t gid_a = 0u;
    auto flush = [&](uint32_t gid_b, int rows) {
        __syncwarp();
        if (lane < rows) {
            if constexpr (HI) {
                const float t = row_sum32(red + lane * kRedStride);
                atomicAdd((lane < 9 ? g2d : g2d_hi) + (size_t)gid_b * kG2dStride + (lane < 9 ? lane : lane - 9), t);
            } else {
                const float t = row_sum16(red + lane * kHalfStride);
                atomicAdd(g2d + (size_t)(lane < 9 ? gid_a : gid_b) * kG2dStride + (lane < 9 ? lane : lane - 9), t);
            }
        }
        __syncwarp();
    };

    float4* e_mu = sm.ent[warp][0];
    float4* e_co = sm.ent[warp][1];
    float4* e_c = sm.ent[warp][2];
    // an entry's per-pixel quantities that do not depend on the entries behind it
    struct Staged {
        float dx, dy, araw, c0, c1, c2;
        uint32_t gid, pos;
    };
    auto stage = [&](int k) {
        const float4 m = e_mu[k];
        const float4 cp = e_co[k];
        const float4 col = e_c[k];
        Staged a;
        a.dx = lx - m.x;
        a.dy = ly - m.y;
        a.araw = __fmul_rn(cp.w, gauss2(cp, a.dx, a.dy));
        a.c0 = col.x;
        a.c1 = col.y;
        a.c2 = col.z;
        a.gid = __float_as_uint(m.z);
        a.pos = __float_as_uint(m.w);
        return a;
    };
    // back to front through one entry: transmittance in front of it, its
    // dL/dalpha, the colour behind, and its per-pixel values into buffer slot
    // `slot` (rows 9 slot .. 9 slot + 8, and the higher moments in rows 9..17)
    auto composite = [&](const Staged& a, int slot) {
        const bool valid = a.pos < last && a.araw >= st.alpha_min;
        const bool clamped = a.araw >= st.alpha_max;
        const float ae = valid ? (clamped ? st.alpha_max : a.araw) : 0.0f;
        const float one_m = 1.0f - ae;
        T = __fdividef(T, one_m);                     // transmittance in front of this Gaussian
        const float dLda = T * (g0 * (a.c0 - acc0) + g1 * (a.c1 - acc1) + g2 * (a.c2 - acc2));
        acc0 += ae * (a.c0 - acc0);
        acc1 += ae * (a.c1 - acc1);
        acc2 += ae * (a.c2 - acc2);
        const float aT = ae * T;
        const float w = (clamped ? 0.0f : ae) * dLda;   // dL/dsigma * sigma
        const float dx = a.dx, dy = a.dy;
        const float wdx = w * dx, wdy = w * dy;
        if constexpr (!HI) {
            // lanes 16 apart exchange halves: lanes 0-15 keep values 0-3, lanes
            // 16-31 values 4-7, each summed over the pair; value 8 is summed by
            // both and written by the lower half
            const float v[8] = {wdx, wdy, wdx * dx, wdx * dy, wdy * dy, w, g0 * aT, g1 * aT};
            const bool up = lane & 16;
            float* rb = red + (slot * 9 + (up ? 4 : 0)) * kHalfStride + (lane & 15);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const float send = up ? v[j] : v[j + 4];
                const float keep = up ? v[j + 4] : v[j];
                rb[j * kHalfStride] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
            }
            const float v8 = g2 * aT;
            const float s8 = v8 + __shfl_xor_sync(0xffffffffu, v8, 16);
            if (!up) red[(slot * 9 + 8) * kHalfStride + lane] = s8;
            return a.gid;
        }
        float* rb = red + slot * 9 * kRedStride + lane;
        rb[0 * kRedStride] = wdx;
        rb[1 * kRedStride] = wdy;
        rb[2 * kRedStride] = wdx * dx;
        rb[3 * kRedStride] = wdx * dy;
        rb[4 * kRedStride] = wdy * dy;
        rb[5 * kRedStride] = w;
        rb[6 * kRedStride] = g0 * aT;
        rb[7 * kRedStride] = g1 * aT;
        rb[8 * kRedStride] = g2 * aT;
        if constexpr (HI) {
            const float wxx = wdx * dx, wyy = wdy * dy;
            rb[9 * kRedStride] = wxx * dx;
            rb[10 * kRedStride] = wxx * dy;
            rb[11 * kRedStride] = wyy * dx;
            rb[12 * kRedStride] = wyy * dy;
            rb[13 * kRedStride] = wxx * dx * dx;
            rb[14 * kRedStride] = wxx * dx * dy;
            rb[15 * kRedStride] = wxx * dy * dy;
            rb[16 * kRedStride] = wyy * dx * dy;
            rb[17 * kRedStride] = wyy * dy * dy;
        }
        return a.gid;
    };
    for (int end = (int)cnt; end > 0; end -= 32) {
        const int start = max(0, end - 32);
        const int c = end - start;
        __syncwarp();                               // the previous chunk's slots are free
        if (lane < c) {
            uint32_t pos = walk[wbase + start + lane];
            // a position past the list composites nowhere (pos >= L >= every last)
            const uint32_t g = gids[rg.x + ((long long)pos < L ? pos : 0u)];
            if ((long long)pos > L) pos = (uint32_t)L;
            const float4 m = xy[g];
            e_mu[lane] = make_float4((m.x - (float)ox) + m.z, (m.y - (float)oy) + m.w, __uint_as_float(g),
                                     __uint_as_float(pos));
            e_co[lane] = conic_exp2(conic_opac[g]);
            e_c[lane] = rgb[g];
        }
        __syncwarp();
        if constexpr (HI) {
            for (int k = c - 1; k >= 0; --k) {
                const Staged a = stage(k);
                flush(composite(a, 0), kRedRows);
            }
        } else {
            // two entries at a time: their alpha evaluations are independent
            // (only the transmittance and the colour behind are carried from
            // one entry to the next), and the pair fills one 18-row flush
            int k = c - 1;
            for (; k >= 1; k -= 2) {
                const Staged a = stage(k);
                const Staged b = stage(k - 1);
                gid_a = composite(a, 0);
                flush(composite(b, 1), kRedRows);
            }
            if (k == 0) {
                gid_a = composite(stage(0), 0);
                flush(gid_a, 9);
            }
        }
    }
}

// Clears the accumulator rows (and the higher-moment rows when given) of the
// Gaussians whose projection reached a tile: the only rows the backward adds
// to and the projection adjoint reads.
__global__ void __launch_bounds__(256) zero_reached_rows_kernel(const uint32_t* __restrict__ tiles, int n,
                                                                float4* __restrict__ g2d,
                                                                float4* __restrict__ g2d_hi) {
    pdl_wait_and_trigger();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || tiles[i] == 0u) return;
    const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int k = 0; k < kG2dStride / 4; ++k) g2d[(size_t)i * (kG2dStride / 4) + k] = z;
    if (g2d_hi) {
#pragma unroll
        for (int k = 0; k < kG2dStride / 4; ++k) g2d_hi[(size_t)i * (kG2dStride / 4) + k] = z;
    }
}

cudaError_t launch_zero_reached_rows(const uint32_t* tiles, int n, float* g2d, float* g2d_hi, cudaStream_t stream) {
    if (n == 0) return cudaSuccess;
    (void)launch_pdl(zero_reached_rows_kernel, dim3((n + 255) / 256), dim3(256), 0, stream, tiles, n,
                     reinterpret_cast<float4*>(g2d), reinterpret_cast<float4*>(g2d_hi));
    note_launch();
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Single view: one CTA per tile.  The forward is bounded to 48 resident warps
// per SM (40 registers): its per-pixel chain is latency-bound and gains from
// the extra warps more than it loses to the two spilled words.
// ---------------------------------------------------------------------------
template <int TW, int TH, bool L1, bool REC>
__global__ void __launch_bounds__(TW * TH, 1536 / (TW * TH)) render_fwd_kernel(
    const uint2* __restrict__ ranges, const uint32_t* __restrict__ gids, const float4* __restrict__ xy,
    const float4* __restrict__ conic_opac, const float4* __restrict__ rgb, int W, int H, int gx, SetDev st,
    float* __restrict__ image, float* __restrict__ final_T, uint32_t* __restrict__ n_contrib,
    const uint32_t* __restrict__ order, L1Out l1, WalkOut wo) {
    pdl_wait_and_trigger();
    __shared__ FwdSmem<TW * TH, TW * TH / 32, TW / 8> sm;
    const int t = order ? (int)order[blockIdx.x] : (int)blockIdx.x;
    if ((unsigned)t >= gridDim.x) return;      // a schedule that is not a permutation of the tiles
    fwd_tile<TW, TH, TW * TH, REC>(t, gx, W, H, ranges[t], gids, xy, conic_opac, rgb, st, image, final_T, n_contrib,
                                   sm, L1 ? &l1 : nullptr, wo);
}

// The backward kernels are bounded to 40 resident warps per SM (48 registers):
// their pair loop is issue-bound and hides its latencies with warps.
template <int TW, int TH, bool HI>
__global__ void __launch_bounds__(TW * TH, 1280 / (TW * TH)) render_bwd_kernel(
    const uint2* __restrict__ ranges, const uint32_t* __restrict__ gids, const float4* __restrict__ xy,
    const float4* __restrict__ conic_opac, const float4* __restrict__ rgb, int W, int H, int gx, SetDev st,
    const float* __restrict__ final_T, const uint32_t* __restrict__ n_contrib,
    const float* __restrict__ dL_dimage, float* __restrict__ g2d, float* __restrict__ g2d_hi,
    const uint32_t* __restrict__ order) {
    pdl_wait_and_trigger();
    __shared__ BwdSmem<TW * TH, TW * TH / 32, TW / 8> sm;
    const int t = order ? (int)order[blockIdx.x] : (int)blockIdx.x;
    if ((unsigned)t >= gridDim.x) return;      // a schedule that is not a permutation of the tiles
    bwd_tile<TW, TH, TW * TH, HI>(t, gx, W, H, ranges[t], gids, xy, conic_opac, rgb, st, final_T, n_contrib,
                                  dL_dimage, g2d, g2d_hi, sm);
}

// The backward pass over the forward's walk lists, bounded to 32 resident
// warps per SM (64 registers): the two-entry steps need the registers.
template <int TW, int TH, bool HI>
__global__ void __launch_bounds__(TW * TH, 1024 / (TW * TH)) render_bwd_walk_kernel(
    const uint2* __restrict__ ranges, const uint32_t* __restrict__ gids, const float4* __restrict__ xy,
    const float4* __restrict__ conic_opac, const float4* __restrict__ rgb, int W, int H, int gx, SetDev st,
    const float* __restrict__ final_T, const uint32_t* __restrict__ n_contrib,
    const float* __restrict__ dL_dimage, const uint32_t* __restrict__ walk,
    const uint32_t* __restrict__ walk_count, long long walk_cap, float* __restrict__ g2d,
    float* __restrict__ g2d_hi, const uint32_t* __restrict__ order) {
    pdl_wait_and_trigger();
    __shared__ BwdWalkSmem<TW * TH / 32> sm;
    const int t = order ? (int)order[blockIdx.x] : (int)blockIdx.x;
    if ((unsigned)t >= gridDim.x) return;      // a schedule that is not a permutation of the tiles
    bwd_tile_walk<TW, TH, HI>(t, threadIdx.x >> 5, gx, W, H, ranges[t], gids, xy, conic_opac, rgb, st, final_T,
                              n_contrib, dL_dimage, walk, walk_count, walk_cap, g2d, g2d_hi, sm);
}

// ---------------------------------------------------------------------------
// Several views: persistent CTAs pull global tiles from an atomic counter
// (the counter must be zero at launch).  Per-view maps are concatenated at
// pixel offsets pix_off[v].  The forward is bounded, as the single-view one,
// to 48 resident warps per SM (40 registers): unbounded it took 55 registers
// and 4 CTAs per SM, and its warps waited at the batch barriers with the
// issue slots two-thirds busy.
// ---------------------------------------------------------------------------
template <int TW, int TH, int BATCH, bool REC>
__global__ void __launch_bounds__(TW * TH, 1536 / (TW * TH)) render_fwd_views_kernel(
    ViewsDev vd, const uint2* __restrict__ ranges, const uint32_t* __restrict__ gids, const float4* __restrict__ xy,
    const float4* __restrict__ conic_opac, const float4* __restrict__ rgb, SetDev st, float* __restrict__ images,
    float* __restrict__ final_T, uint32_t* __restrict__ n_contrib, uint32_t* __restrict__ counter,
    const uint32_t* __restrict__ order, WalkOut wo) {
    pdl_wait_and_trigger();
    constexpr int NW = TW * TH / 32;
    __shared__ FwdSmem<BATCH, NW, TW / 8> sm;
    __shared__ int s_tile;
    for (;;) {
        if (threadIdx.x == 0) s_tile = (int)atomicAdd(counter, 1u);
        __syncthreads();
        const int k = s_tile;
        __syncthreads();
        if (k >= vd.T_total) break;
        const int t = order ? (int)order[k] : k;
        if ((unsigned)t >= (unsigned)vd.T_total) continue;
        const int v = view_of_tile(vd, t);
        const CamDev& c = vd.cam[v];
        const long long po = vd.pix_off[v];
        // walk lists index the global list (rows NW*start + ...) and count per
        // global tile: the view's counts start at its first global tile
        const WalkOut wv{wo.walk, wo.count ? wo.count + (long long)vd.tile_off[v] * NW : nullptr, wo.cap};
        fwd_tile<TW, TH, BATCH, REC>(t - vd.tile_off[v], c.gx, c.width, c.height, ranges[t], gids, xy, conic_opac,
                                     rgb, st, images + 3 * po, final_T + po, n_contrib + po, sm, nullptr, wv);
    }
}

// The backward pass of several views over the forward's walk lists: a block
// per global tile in the schedule's order, each warp stepping through its own
// list (as render_bwd_walk_kernel).
template <int TW, int TH>
__global__ void __launch_bounds__(TW * TH, 1024 / (TW * TH)) render_bwd_views_walk_kernel(
    ViewsDev vd, const uint2* __restrict__ ranges, const uint32_t* __restrict__ gids, const float4* __restrict__ xy,
    const float4* __restrict__ conic_opac, const float4* __restrict__ rgb, SetDev st,
    const float* __restrict__ final_T, const uint32_t* __restrict__ n_contrib, const float* __restrict__ dL,
    const uint32_t* __restrict__ walk, const uint32_t* __restrict__ walk_count, long long walk_cap,
    float* __restrict__ g2d, const uint32_t* __restrict__ order) {
    pdl_wait_and_trigger();
    constexpr int NW = TW * TH / 32;
    __shared__ BwdWalkSmem<NW> sm;
    const int t = order ? (int)order[blockIdx.x] : (int)blockIdx.x;
    if ((unsigned)t >= (unsigned)vd.T_total) return;
    const int v = view_of_tile(vd, t);
    const CamDev& c = vd.cam[v];
    const long long po = vd.pix_off[v];
    bwd_tile_walk<TW, TH, false>(t - vd.tile_off[v], threadIdx.x >> 5, c.gx, c.width, c.height, ranges[t], gids, xy,
                                 conic_opac, rgb, st, final_T + po, n_contrib + po, dL + 3 * po, walk,
                                 walk_count + (long long)vd.tile_off[v] * NW, walk_cap, g2d, nullptr, sm);
}

template <int TW, int TH, int BATCH>
__global__ void __launch_bounds__(TW * TH, 1280 / (TW * TH)) render_bwd_views_kernel(
    ViewsDev vd, const uint2* __restrict__ ranges, const uint32_t* __restrict__ gids, const float4* __restrict__ xy,
    const float4* __restrict__ conic_opac, const float4* __restrict__ rgb, SetDev st,
    const float* __restrict__ final_T, const uint32_t* __restrict__ n_contrib, const float* __restrict__ dL,
    float* __restrict__ g2d, uint32_t* __restrict__ counter, const uint32_t* __restrict__ order) {
    pdl_wait_and_trigger();
    __shared__ BwdSmem<BATCH, TW * TH / 32, TW / 8> sm;
    __shared__ int s_tile;
    for (;;) {
        if (threadIdx.x == 0) s_tile = (int)atomicAdd(counter, 1u);
        __syncthreads();
        const int k = s_tile;
        __syncthreads();
        if (k >= vd.T_total) break;
        const int t = order ? (int)order[k] : k;
        if ((unsigned)t >= (unsigned)vd.T_total) continue;
        const int v = view_of_tile(vd, t);
        const CamDev& c = vd.cam[v];
        const long long po = vd.pix_off[v];
        bwd_tile<TW, TH, BATCH, false>(t - vd.tile_off[v], c.gx, c.width, c.height, ranges[t], gids, xy,
                                       conic_opac, rgb, st, final_T + po, n_contrib + po, dL + 3 * po, g2d, nullptr,
                                       sm);
    }
}

// Pair counts of the forward walk, per pixel: (pairs evaluated, pairs
// composited), and, when warp_union is given, per 8x4 pixel block of each tile
// (the warps of the compositing kernels) the number of list entries that at
// least one of its pixels composites.  A measurement aid: it replays the walk
// over every list entry, without colour and without culling.
template <int TW, int TH>
__global__ void __launch_bounds__(TW * TH) render_stats_kernel(
    const uint2* __restrict__ ranges, const uint32_t* __restrict__ gids, const float4* __restrict__ xy,
    const float4* __restrict__ conic_opac, int W, int H, int gx, SetDev st, uint2* __restrict__ counts,
    uint32_t* __restrict__ warp_union) {
    pdl_wait_and_trigger();
    constexpr int NW = TW * TH / 32;
    const int tile = blockIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int bx, by;
    warp_block_origin<TW>(tile, gx, TH, &bx, &by);
    const int px = bx + (lane & 7);
    const int py = by + (lane >> 3);
    const bool inside = px < W && py < H;
    const int ox = (tile % gx) * TW, oy = (tile / gx) * TH;
    const float lx = (float)(px - ox), ly = (float)(py - oy);
    const uint2 rg = ranges[tile];
    float T = 1.0f;
    bool stop = !inside;
    uint32_t ev = 0, comp = 0, uni = 0;
    for (uint32_t k = rg.x; k < rg.y; ++k) {
        if (__all_sync(0xffffffffu, stop)) break;
        bool c = false;
        if (!stop) {
            const uint32_t g = gids[k];
            const float4 m = xy[g];
            const float4 cp = conic_exp2(conic_opac[g]);
            const float dx = lx - ((m.x - (float)ox) + m.z);
            const float dy = ly - ((m.y - (float)oy) + m.w);
            const float alpha = fminf(st.alpha_max, __fmul_rn(cp.w, gauss2(cp, dx, dy)));
            ++ev;
            if (alpha >= st.alpha_min) {
                const float Tn = T * (1.0f - alpha);
                if (Tn < st.T_min) {
                    stop = true;
                } else {
                    ++comp;
                    T = Tn;
                    c = true;
                }
            }
        }
        uni += __ballot_sync(0xffffffffu, c) != 0u;
    }
    if (inside) counts[py * W + px] = make_uint2(ev, comp);
    if (warp_union && lane == 0) warp_union[(long long)tile * NW + warp] = uni;
}

// FP32 FMA throughput probe (a measurement aid): eight independent FMA chains
// per thread, `iters` rounds; the result is stored so nothing is folded.
__global__ void __launch_bounds__(256) fma_probe_kernel(float* __restrict__ out, int iters, float b, float c) {
    pdl_wait_and_trigger();
    float a[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = (float)(threadIdx.x + k) * 1e-3f;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 8; ++k) a[k] = __fmaf_rn(a[k], b, c);
    }
    float s = 0.0f;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += a[k];
    out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

cudaError_t launch_fma_probe(float* out, int blocks, int iters, cudaStream_t stream) {
    (void)launch_pdl(fma_probe_kernel, dim3(blocks), dim3(256), 0, stream, out, iters, 0.999f, 1e-3f);
    note_launch();
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------
template <int TW, int TH>
static cudaError_t stats_tmpl(const sgs_proj& proj, const sgs_bins& bins, const CamDev& cam, const SetDev& st,
                              uint32_t* counts, uint32_t* warp_union, cudaStream_t stream) {
    const int T = cam.gx * cam.gy;
    (void)launch_pdl(render_stats_kernel<TW, TH>, dim3(T), dim3(TW * TH), 0, stream,
                     reinterpret_cast<const uint2*>(bins.ranges), bins.gids, reinterpret_cast<const float4*>(proj.xy),
                     reinterpret_cast<const float4*>(proj.conic_opac), cam.width, cam.height, cam.gx, st,
                     reinterpret_cast<uint2*>(counts), warp_union);
    note_launch();
    return cudaGetLastError();
}

template <int TW, int TH>
static cudaError_t fwd_tmpl(const sgs_proj& proj, const sgs_bins& bins, const CamDev& cam, const SetDev& st,
                            float* image, float* final_T, uint32_t* n_contrib, const L1Out& l1,
                            cudaStream_t stream) {
    const int T = cam.gx * cam.gy;
    const bool rec = bins.walk != nullptr;
    const WalkOut wo{bins.walk, bins.walk_count,
                     (long long)(TW * TH / 32) * (long long)bins.capacity};
    auto kern = l1.target ? (rec ? render_fwd_kernel<TW, TH, true, true> : render_fwd_kernel<TW, TH, true, false>)
                          : (rec ? render_fwd_kernel<TW, TH, false, true> : render_fwd_kernel<TW, TH, false, false>);
    (void)launch_pdl(kern, dim3(T), dim3(TW * TH), 0, stream,
                     reinterpret_cast<const uint2*>(bins.ranges), bins.gids, reinterpret_cast<const float4*>(proj.xy),
                     reinterpret_cast<const float4*>(proj.conic_opac), reinterpret_cast<const float4*>(proj.rgb),
                     cam.width, cam.height, cam.gx, st, image, final_T, n_contrib, bins.order, l1, wo);
    note_launch();
    return cudaGetLastError();
}

template <int TW, int TH>
static cudaError_t bwd_tmpl(const sgs_proj& proj, const sgs_bins& bins, const CamDev& cam, const SetDev& st,
                            const float* final_T, const uint32_t* n_contrib, const float* dL, float* g2d,
                            float* g2d_hi, cudaStream_t stream) {
    const int T = cam.gx * cam.gy;
    if (bins.walk) {                            // the forward's walk lists: composited entries only
        auto kern = g2d_hi ? render_bwd_walk_kernel<TW, TH, true> : render_bwd_walk_kernel<TW, TH, false>;
        (void)launch_pdl(kern, dim3(T), dim3(TW * TH), 0, stream, reinterpret_cast<const uint2*>(bins.ranges),
                         bins.gids, reinterpret_cast<const float4*>(proj.xy),
                         reinterpret_cast<const float4*>(proj.conic_opac), reinterpret_cast<const float4*>(proj.rgb),
                         cam.width, cam.height, cam.gx, st, final_T, n_contrib, dL, bins.walk, bins.walk_count,
                         (long long)(TW * TH / 32) * (long long)bins.capacity, g2d, g2d_hi, bins.order);
        note_launch();
        return cudaGetLastError();
    }
    auto kern = g2d_hi ? render_bwd_kernel<TW, TH, true> : render_bwd_kernel<TW, TH, false>;
    (void)launch_pdl(kern, dim3(T), dim3(TW * TH), 0, stream, reinterpret_cast<const uint2*>(bins.ranges), bins.gids,
                     reinterpret_cast<const float4*>(proj.xy), reinterpret_cast<const float4*>(proj.conic_opac),
                     reinterpret_cast<const float4*>(proj.rgb), cam.width, cam.height, cam.gx, st, final_T, n_contrib,
                     dL, g2d, g2d_hi, bins.order);
    note_launch();
    return cudaGetLastError();
}

#define SGS_TILE_DISPATCH(FN, ...)                                                                  \
    if (st.tile_w == 16 && st.tile_h == 16) return FN<16, 16>(__VA_ARGS__);                         \
    if (st.tile_w == 16 && st.tile_h == 8) return FN<16, 8>(__VA_ARGS__);                           \
    if (st.tile_w == 8 && st.tile_h == 8) return FN<8, 8>(__VA_ARGS__);                             \
    if (st.tile_w == 32 && st.tile_h == 8) return FN<32, 8>(__VA_ARGS__);                           \
    return cudaErrorInvalidValue;

cudaError_t launch_render_stats(const sgs_proj& proj, const sgs_bins& bins, const CamDev& cam, const SetDev& st,
                                uint32_t* counts, uint32_t* warp_union, cudaStream_t stream) {
    SGS_TILE_DISPATCH(stats_tmpl, proj, bins, cam, st, counts, warp_union, stream)
}

cudaError_t launch_render_fwd(const sgs_proj& proj, const sgs_bins& bins, const CamDev& cam, const SetDev& st,
                              float* image, float* final_T, uint32_t* n_contrib, const float* target, int n_views,
                              float* dL, float* loss, cudaStream_t stream) {
    L1Out l1{target, dL, loss, 0.0f};
    if (target)
        l1.norm = (float)(1.0 / (3.0 * (double)cam.height * (double)cam.width * (double)n_views));
    SGS_TILE_DISPATCH(fwd_tmpl, proj, bins, cam, st, image, final_T, n_contrib, l1, stream)
}

cudaError_t launch_render_bwd(const sgs_proj& proj, const sgs_bins& bins, const CamDev& cam, const SetDev& st,
                              const float* final_T, const uint32_t* n_contrib, const float* dL, float* g2d,
                              float* g2d_hi, cudaStream_t stream) {
    SGS_TILE_DISPATCH(bwd_tmpl, proj, bins, cam, st, final_T, n_contrib, dL, g2d, g2d_hi, stream)
}

// Persistent multi-view launches: CTAs per SM from the occupancy calculator.
template <class K>
static int persistent_grid(K kernel, int threads, int T_total) {
    int dev = 0, sms = 152, per_sm = 1;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, 0) != cudaSuccess || per_sm < 1)
        per_sm = 1;
    const int g = sms * per_sm;
    return g < T_total ? g : (T_total > 0 ? T_total : 1);
}

template <int TW, int TH, int BATCH>
static cudaError_t fwd_views_tmpl(const ViewsDev& vd, const sgs_proj& proj, const uint32_t* ranges,
                                  const uint32_t* gids, const SetDev& st, float* images, float* final_T,
                                  uint32_t* n_contrib, uint32_t* counter, const uint32_t* order,
                                  const WalkLists& wl, cudaStream_t stream) {
    auto k = wl.walk ? render_fwd_views_kernel<TW, TH, BATCH, true> : render_fwd_views_kernel<TW, TH, BATCH, false>;
    const int grid = persistent_grid(k, TW * TH, vd.T_total);
    const WalkOut wo{wl.walk, wl.count, wl.cap};
    (void)launch_pdl(k, dim3(grid), dim3(TW * TH), 0, stream, vd, reinterpret_cast<const uint2*>(ranges), gids,
                     reinterpret_cast<const float4*>(proj.xy), reinterpret_cast<const float4*>(proj.conic_opac),
                     reinterpret_cast<const float4*>(proj.rgb), st, images, final_T, n_contrib, counter, order, wo);
    note_launch();
    return cudaGetLastError();
}

template <int TW, int TH, int BATCH>
static cudaError_t bwd_views_tmpl(const ViewsDev& vd, const sgs_proj& proj, const uint32_t* ranges,
                                  const uint32_t* gids, const SetDev& st, const float* final_T,
                                  const uint32_t* n_contrib, const float* dL, float* g2d, uint32_t* counter,
                                  const uint32_t* order, const WalkLists& wl, cudaStream_t stream) {
    if (wl.walk) {
        auto k = render_bwd_views_walk_kernel<TW, TH>;
        (void)launch_pdl(k, dim3(vd.T_total > 0 ? vd.T_total : 1), dim3(TW * TH), 0, stream, vd,
                         reinterpret_cast<const uint2*>(ranges), gids, reinterpret_cast<const float4*>(proj.xy),
                         reinterpret_cast<const float4*>(proj.conic_opac), reinterpret_cast<const float4*>(proj.rgb),
                         st, final_T, n_contrib, dL, wl.walk, wl.count, wl.cap, g2d, order);
        note_launch();
        return cudaGetLastError();
    }
    auto k = render_bwd_views_kernel<TW, TH, BATCH>;
    const int grid = persistent_grid(k, TW * TH, vd.T_total);
    (void)launch_pdl(k, dim3(grid), dim3(TW * TH), 0, stream, vd, reinterpret_cast<const uint2*>(ranges), gids,
                     reinterpret_cast<const float4*>(proj.xy), reinterpret_cast<const float4*>(proj.conic_opac),
                     reinterpret_cast<const float4*>(proj.rgb), st, final_T, n_contrib, dL, g2d, counter, order);
    note_launch();
    return cudaGetLastError();
}

#define SGS_VIEWS_DISPATCH(FN, ...)                                                                        \
    switch (batch) {                                                                                       \
        case 64:                                                                                           \
            if (st.tile_w == 16 && st.tile_h == 16) return FN<16, 16, 64>(__VA_ARGS__);                   \
            if (st.tile_w == 16 && st.tile_h == 8) return FN<16, 8, 64>(__VA_ARGS__);                     \
            if (st.tile_w == 8 && st.tile_h == 8) return FN<8, 8, 64>(__VA_ARGS__);                       \
            if (st.tile_w == 32 && st.tile_h == 8) return FN<32, 8, 64>(__VA_ARGS__);                     \
            break;                                                                                         \
        case 128:                                                                                          \
            if (st.tile_w == 16 && st.tile_h == 16) return FN<16, 16, 128>(__VA_ARGS__);                  \
            if (st.tile_w == 16 && st.tile_h == 8) return FN<16, 8, 128>(__VA_ARGS__);                    \
            if (st.tile_w == 8 && st.tile_h == 8) return FN<8, 8, 128>(__VA_ARGS__);                      \
            if (st.tile_w == 32 && st.tile_h == 8) return FN<32, 8, 128>(__VA_ARGS__);                    \
            break;                                                                                         \
        case 256:                                                                                          \
            if (st.tile_w == 16 && st.tile_h == 16) return FN<16, 16, 256>(__VA_ARGS__);                  \
            if (st.tile_w == 16 && st.tile_h == 8) return FN<16, 8, 256>(__VA_ARGS__);                    \
            if (st.tile_w == 8 && st.tile_h == 8) return FN<8, 8, 256>(__VA_ARGS__);                      \
            if (st.tile_w == 32 && st.tile_h == 8) return FN<32, 8, 256>(__VA_ARGS__);                    \
            break;                                                                                         \
        default:                                                                                           \
            break;                                                                                         \
    }                                                                                                      \
    return cudaErrorInvalidValue;

cudaError_t launch_render_fwd_views(const ViewsDev& vd, const sgs_proj& proj, const uint32_t* ranges,
                                    const uint32_t* gids, const SetDev& st, int batch, float* images,
                                    float* final_T, uint32_t* n_contrib, uint32_t* counter, const uint32_t* order,
                                    const WalkLists& wl, cudaStream_t stream) {
    SGS_VIEWS_DISPATCH(fwd_views_tmpl, vd, proj, ranges, gids, st, images, final_T, n_contrib, counter, order, wl,
                       stream)
}

cudaError_t launch_render_bwd_views(const ViewsDev& vd, const sgs_proj& proj, const uint32_t* ranges,
                                    const uint32_t* gids, const SetDev& st, int batch, const float* final_T,
                                    const uint32_t* n_contrib, const float* dL, float* g2d, uint32_t* counter,
                                    const uint32_t* order, const WalkLists& wl, cudaStream_t stream) {
    SGS_VIEWS_DISPATCH(bwd_views_tmpl, vd, proj, ranges, gids, st, final_T, n_contrib, dL, g2d, counter, order, wl,
                       stream)
}

}  // namespace sgs
