// Projection of the Gaussians into one view and its adjoint with the lift of
// the 2-D splitting accumulators to the 3x3 splitting matrix.
//
// Paper: Section 3, Eq. sigma_3D (sigma = o N(xi; p, Sigma)), Eq. sigma_2D and
// the affine-Pi footnote (Sigma2D = P Sigma P^T); Appendix "Deriving Hessian of
// Gaussian" (Hess_p sigma = sigma (Y Y^T - P^T Sigma2D^-1 P), Y = P^T
// Sigma2D^-1 (x - Pi(p)), with P, Sigma2D and colour frozen).
#include <type_traits>

#include "common.cuh"

namespace sgs {

// ---------------------------------------------------------------------------
// float32 exponential used by the integer stage: Cody-Waite range reduction
// (x = k ln2 + r, ln2 split so that k*ln2_hi is exact) and the degree-7 Taylor
// polynomial of e^r in Horner form, each step rounded separately, then the
// exact scaling by 2^k.  Within 2 ulp of exp for |x| <= 87.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float exp_stage(float x) {
    x = fminf(fmaxf(x, -87.0f), 88.0f);
    float k = rintf(mul_rn(x, 0x1.715476p+0f));
    float r = sub_rn(sub_rn(x, mul_rn(k, 0x1.62e4p-1f)), mul_rn(k, 0x1.7f7d1cp-20f));
    float p = 0x1.a01a02p-13f;
    p = mad_rn(p, r, 0x1.6c16c2p-10f);
    p = mad_rn(p, r, 0x1.111112p-7f);
    p = mad_rn(p, r, 0x1.555556p-5f);
    p = mad_rn(p, r, 0x1.555556p-3f);
    p = mad_rn(p, r, 0.5f);
    p = mad_rn(p, r, 1.0f);
    p = mad_rn(p, r, 1.0f);
    int ki = (int)k;
    return mul_rn(p, __int_as_float((ki + 127) << 23));
}

// Integer stage: camera-space mean, clamped Jacobian, rotation, scales and the
// dilated 2-D covariance in float32 with a fixed operation order; radius
// ceil(radius_sigma sqrt(lambda_max)); inclusive tile rect of the bounding
// square.  Sums are left to right.
__device__ Stage integer_stage(const float* __restrict__ means, const float* __restrict__ log_scales,
                               const float* __restrict__ quats, int i, const CamDev& cam,
                               const SetDev& st) {
    Stage o;
    o.culled = true;
    o.x_lo = 0; o.x_hi = -1; o.y_lo = 0; o.y_hi = -1;
    const float p0 = means[3 * i], p1 = means[3 * i + 1], p2 = means[3 * i + 2];
    const float* R = cam.R;
    o.tx = add_rn(add_rn(add_rn(mul_rn(R[0], p0), mul_rn(R[1], p1)), mul_rn(R[2], p2)), cam.t[0]);
    o.ty = add_rn(add_rn(add_rn(mul_rn(R[3], p0), mul_rn(R[4], p1)), mul_rn(R[5], p2)), cam.t[1]);
    o.tz = add_rn(add_rn(add_rn(mul_rn(R[6], p0), mul_rn(R[7], p1)), mul_rn(R[8], p2)), cam.t[2]);
    if (!(o.tz > cam.near_z)) return o;
    const float tz = o.tz;
    float mx = add_rn(div_rn(mul_rn(cam.fx, o.tx), tz), cam.cx);
    float my = add_rn(div_rn(mul_rn(cam.fy, o.ty), tz), cam.cy);
    float limx = div_rn(mul_rn(st.fov_clamp, mul_rn(0.5f, (float)cam.width)), cam.fx);
    float limy = div_rn(mul_rn(st.fov_clamp, mul_rn(0.5f, (float)cam.height)), cam.fy);
    float rx = div_rn(o.tx, tz), ry = div_rn(o.ty, tz);
    o.clx = (rx < -limx) || (rx > limx);
    o.cly = (ry < -limy) || (ry > limy);
    o.ux = fminf(fmaxf(rx, -limx), limx);
    o.uy = fminf(fmaxf(ry, -limy), limy);
    float J00 = div_rn(cam.fx, tz), J02 = div_rn(-mul_rn(cam.fx, o.ux), tz);
    float J11 = div_rn(cam.fy, tz), J12 = div_rn(-mul_rn(cam.fy, o.uy), tz);
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        o.T[j] = add_rn(mul_rn(J00, R[j]), mul_rn(J02, R[6 + j]));
        o.T[3 + j] = add_rn(mul_rn(J11, R[3 + j]), mul_rn(J12, R[6 + j]));
    }
    const float q0 = quats[4 * i], q1 = quats[4 * i + 1], q2 = quats[4 * i + 2], q3 = quats[4 * i + 3];
    float qn = sqrt_rn(add_rn(add_rn(add_rn(mul_rn(q0, q0), mul_rn(q1, q1)), mul_rn(q2, q2)), mul_rn(q3, q3)));
    o.qn = qn;
    if (!(qn > 0.0f)) return o;
    float w = div_rn(q0, qn), x = div_rn(q1, qn), y = div_rn(q2, qn), z = div_rn(q3, qn);
    float* Rq = o.Rq;
    Rq[0] = sub_rn(1.0f, mul_rn(2.0f, add_rn(mul_rn(y, y), mul_rn(z, z))));
    Rq[1] = mul_rn(2.0f, sub_rn(mul_rn(x, y), mul_rn(w, z)));
    Rq[2] = mul_rn(2.0f, add_rn(mul_rn(x, z), mul_rn(w, y)));
    Rq[3] = mul_rn(2.0f, add_rn(mul_rn(x, y), mul_rn(w, z)));
    Rq[4] = sub_rn(1.0f, mul_rn(2.0f, add_rn(mul_rn(x, x), mul_rn(z, z))));
    Rq[5] = mul_rn(2.0f, sub_rn(mul_rn(y, z), mul_rn(w, x)));
    Rq[6] = mul_rn(2.0f, sub_rn(mul_rn(x, z), mul_rn(w, y)));
    Rq[7] = mul_rn(2.0f, add_rn(mul_rn(y, z), mul_rn(w, x)));
    Rq[8] = sub_rn(1.0f, mul_rn(2.0f, add_rn(mul_rn(x, x), mul_rn(y, y))));
#pragma unroll
    for (int k = 0; k < 3; ++k) o.s[k] = exp_stage(log_scales[3 * i + k]);
    float M[9];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) M[3 * r + c] = mul_rn(Rq[3 * r + c], o.s[c]);
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int j = 0; j < 3; ++j)
            o.V[3 * a + j] = add_rn(add_rn(mul_rn(o.T[3 * a], M[j]), mul_rn(o.T[3 * a + 1], M[3 + j])),
                                    mul_rn(o.T[3 * a + 2], M[6 + j]));
    const float* V = o.V;
    o.a = add_rn(add_rn(add_rn(mul_rn(V[0], V[0]), mul_rn(V[1], V[1])), mul_rn(V[2], V[2])), st.dilation);
    o.b = add_rn(add_rn(mul_rn(V[0], V[3]), mul_rn(V[1], V[4])), mul_rn(V[2], V[5]));
    o.c = add_rn(add_rn(add_rn(mul_rn(V[3], V[3]), mul_rn(V[4], V[4])), mul_rn(V[5], V[5])), st.dilation);
    float det = sub_rn(mul_rn(o.a, o.c), mul_rn(o.b, o.b));
    if (!(det > 0.0f)) return o;
    float mid = mul_rn(0.5f, add_rn(o.a, o.c));
    float lam = add_rn(mid, sqrt_rn(fmaxf(0.1f, sub_rn(mul_rn(mid, mid), det))));
    float rad = ceilf(mul_rn(st.radius_sigma, sqrt_rn(lam)));
    float fxlo = floorf(div_rn(sub_rn(mx, rad), (float)st.tile_w));
    float fxhi = floorf(div_rn(add_rn(mx, rad), (float)st.tile_w));
    float fylo = floorf(div_rn(sub_rn(my, rad), (float)st.tile_h));
    float fyhi = floorf(div_rn(add_rn(my, rad), (float)st.tile_h));
    if (!(fxhi >= 0.0f && fxlo <= (float)(cam.gx - 1) && fyhi >= 0.0f && fylo <= (float)(cam.gy - 1)))
        return o;
    o.x_lo = (int)fmaxf(fxlo, 0.0f);
    o.x_hi = (int)fminf(fxhi, (float)(cam.gx - 1));
    o.y_lo = (int)fmaxf(fylo, 0.0f);
    o.y_hi = (int)fminf(fyhi, (float)(cam.gy - 1));
    o.culled = false;
    return o;
}

// ---------------------------------------------------------------------------
// Unevaluated float pairs (hi + lo) for the 2-D mean: error-free transforms
// (Knuth two-sum, FMA two-product).
// ---------------------------------------------------------------------------
struct F2 {
    float hi, lo;
};
__device__ __forceinline__ F2 two_sum(float a, float b) {
    float s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}
__device__ __forceinline__ F2 fast_two_sum(float a, float b) {
    float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ F2 two_prod(float a, float b) {
    float p = __fmul_rn(a, b);
    return {p, __fmaf_rn(a, b, -p)};
}
__device__ __forceinline__ F2 f2_add(F2 x, F2 y) {
    F2 s = two_sum(x.hi, y.hi);
    return fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo)));
}
__device__ __forceinline__ F2 f2_mul(F2 x, float b) {
    F2 p = two_prod(x.hi, b);
    return fast_two_sum(p.hi, __fmaf_rn(x.lo, b, p.lo));
}
__device__ __forceinline__ F2 f2_div(F2 x, F2 y) {
    float q1 = __fdiv_rn(x.hi, y.hi);
    F2 p = f2_mul(y, q1);
    F2 r = f2_add(x, F2{-p.hi, -p.lo});
    float q2 = __fdiv_rn(r.hi, y.hi);
    return fast_two_sum(q1, q2);
}
__device__ __forceinline__ F2 dot3_plus(const float* R, float p0, float p1, float p2, float t) {
    F2 acc = two_prod(R[0], p0);
    acc = f2_add(acc, two_prod(R[1], p1));
    acc = f2_add(acc, two_prod(R[2], p2));
    return f2_add(acc, F2{t, 0.0f});
}

// ---------------------------------------------------------------------------
// Real spherical harmonics, degree <= 3, orthonormal on the sphere, with the
// sign pattern of the common graphics convention.  Coefficients are
// 1/(2 sqrt(pi)), sqrt(3/(4 pi)), (1/2) sqrt(15/pi), (1/4) sqrt(5/pi),
// (1/4) sqrt(15/pi), (1/4) sqrt(35/(2 pi)), (1/2) sqrt(105/pi),
// (1/4) sqrt(21/(2 pi)), (1/4) sqrt(7/pi), (1/4) sqrt(105/pi).
// ---------------------------------------------------------------------------
constexpr float kC0 = 2.8209479177e-01f;
constexpr float kC1 = 4.8860251190e-01f;
constexpr float kC2a = 1.0925484306e+00f;
constexpr float kC2b = 3.1539156525e-01f;
constexpr float kC2c = 5.4627421530e-01f;
constexpr float kC3a = 5.9004358993e-01f;
constexpr float kC3b = 2.8906114426e+00f;
constexpr float kC3c = 4.5704579946e-01f;
constexpr float kC3d = 3.7317633259e-01f;
constexpr float kC3e = 1.4453057213e+00f;

__device__ __forceinline__ void sh_basis(int deg, float x, float y, float z, float* Y) {
    Y[0] = kC0;
    if (deg < 1) return;
    Y[1] = -kC1 * y; Y[2] = kC1 * z; Y[3] = -kC1 * x;
    if (deg < 2) return;
    float xx = x * x, yy = y * y, zz = z * z;
    Y[4] = kC2a * x * y;
    Y[5] = -kC2a * y * z;
    Y[6] = kC2b * (2.0f * zz - xx - yy);
    Y[7] = -kC2a * x * z;
    Y[8] = kC2c * (xx - yy);
    if (deg < 3) return;
    Y[9] = -kC3a * y * (3.0f * xx - yy);
    Y[10] = kC3b * x * y * z;
    Y[11] = -kC3c * y * (4.0f * zz - xx - yy);
    Y[12] = kC3d * z * (2.0f * zz - 3.0f * xx - 3.0f * yy);
    Y[13] = -kC3c * x * (4.0f * zz - xx - yy);
    Y[14] = kC3e * z * (xx - yy);
    Y[15] = -kC3a * x * (xx - 3.0f * yy);
}

// Gradient of the basis polynomials, dY[k][axis].
__device__ __forceinline__ void sh_basis_grad(int deg, float x, float y, float z, float (*dY)[3]) {
    dY[0][0] = dY[0][1] = dY[0][2] = 0.0f;
    if (deg < 1) return;
    dY[1][0] = 0.0f; dY[1][1] = -kC1; dY[1][2] = 0.0f;
    dY[2][0] = 0.0f; dY[2][1] = 0.0f; dY[2][2] = kC1;
    dY[3][0] = -kC1; dY[3][1] = 0.0f; dY[3][2] = 0.0f;
    if (deg < 2) return;
    float xx = x * x, yy = y * y, zz = z * z;
    dY[4][0] = kC2a * y; dY[4][1] = kC2a * x; dY[4][2] = 0.0f;
    dY[5][0] = 0.0f; dY[5][1] = -kC2a * z; dY[5][2] = -kC2a * y;
    dY[6][0] = -2.0f * kC2b * x; dY[6][1] = -2.0f * kC2b * y; dY[6][2] = 4.0f * kC2b * z;
    dY[7][0] = -kC2a * z; dY[7][1] = 0.0f; dY[7][2] = -kC2a * x;
    dY[8][0] = 2.0f * kC2c * x; dY[8][1] = -2.0f * kC2c * y; dY[8][2] = 0.0f;
    if (deg < 3) return;
    dY[9][0] = -6.0f * kC3a * x * y; dY[9][1] = -kC3a * (3.0f * xx - 3.0f * yy); dY[9][2] = 0.0f;
    dY[10][0] = kC3b * y * z; dY[10][1] = kC3b * x * z; dY[10][2] = kC3b * x * y;
    dY[11][0] = 2.0f * kC3c * x * y; dY[11][1] = -kC3c * (4.0f * zz - xx - 3.0f * yy); dY[11][2] = -8.0f * kC3c * y * z;
    dY[12][0] = -6.0f * kC3d * x * z; dY[12][1] = -6.0f * kC3d * y * z; dY[12][2] = kC3d * (6.0f * zz - 3.0f * xx - 3.0f * yy);
    dY[13][0] = -kC3c * (4.0f * zz - 3.0f * xx - yy); dY[13][1] = 2.0f * kC3c * x * y; dY[13][2] = -8.0f * kC3c * x * z;
    dY[14][0] = 2.0f * kC3e * x * z; dY[14][1] = -2.0f * kC3e * y * z; dY[14][2] = kC3e * (xx - yy);
    dY[15][0] = -kC3a * (3.0f * xx - 3.0f * yy); dY[15][1] = 6.0f * kC3a * x * y; dY[15][2] = 0.0f;
}

// Loads the 3K SH coefficients of Gaussian i (16-byte loads when 3K is a
// multiple of 4; rows of 3K floats start 16-byte aligned then).
template <int DEG>
__device__ __forceinline__ void load_sh(const float* __restrict__ sh, int i, float (&c)[3 * (DEG + 1) * (DEG + 1)]) {
    constexpr int K3 = 3 * (DEG + 1) * (DEG + 1);
    const float* src = sh + (size_t)i * K3;
    if constexpr (K3 % 4 == 0) {
        const float4* s4 = reinterpret_cast<const float4*>(src);
#pragma unroll
        for (int q = 0; q < K3 / 4; ++q) {
            const float4 t = __ldg(s4 + q);
            c[4 * q] = t.x; c[4 * q + 1] = t.y; c[4 * q + 2] = t.z; c[4 * q + 3] = t.w;
        }
    } else {
#pragma unroll
        for (int q = 0; q < K3; ++q) c[q] = __ldg(src + q);
    }
}

// e = sum_k w_k grad Y_k (the gradient of the polynomials, k >= 1), without
// materialising the 16 x 3 table of basis gradients.
template <int DEG>
__device__ __forceinline__ void sh_weighted_grad(float x, float y, float z, const float* w, float& e0, float& e1,
                                                 float& e2) {
    e0 = 0.0f; e1 = 0.0f; e2 = 0.0f;
    if constexpr (DEG >= 1) {
        e0 += -kC1 * w[3];
        e1 += -kC1 * w[1];
        e2 += kC1 * w[2];
    }
    if constexpr (DEG >= 2) {
        const float xx = x * x, yy = y * y;
        e0 += kC2a * (y * w[4] - z * w[7]) - 2.0f * kC2b * x * w[6] + 2.0f * kC2c * x * w[8];
        e1 += kC2a * (x * w[4] - z * w[5]) - 2.0f * kC2b * y * w[6] - 2.0f * kC2c * y * w[8];
        e2 += -kC2a * (y * w[5] + x * w[7]) + 4.0f * kC2b * z * w[6];
        (void)xx; (void)yy;
    }
    if constexpr (DEG >= 3) {
        const float xx = x * x, yy = y * y, zz = z * z;
        e0 += -6.0f * kC3a * x * y * w[9] + kC3b * y * z * w[10] + 2.0f * kC3c * x * y * w[11] -
              6.0f * kC3d * x * z * w[12] - kC3c * (4.0f * zz - 3.0f * xx - yy) * w[13] +
              2.0f * kC3e * x * z * w[14] - kC3a * (3.0f * xx - 3.0f * yy) * w[15];
        e1 += -kC3a * (3.0f * xx - 3.0f * yy) * w[9] + kC3b * x * z * w[10] -
              kC3c * (4.0f * zz - xx - 3.0f * yy) * w[11] - 6.0f * kC3d * y * z * w[12] +
              2.0f * kC3c * x * y * w[13] - 2.0f * kC3e * y * z * w[14] + 6.0f * kC3a * x * y * w[15];
        e2 += kC3b * x * y * w[10] - 8.0f * kC3c * y * z * w[11] + kC3d * (6.0f * zz - 3.0f * xx - 3.0f * yy) * w[12] -
              8.0f * kC3c * x * z * w[13] + kC3e * (xx - yy) * w[14];
    }
}

// ---------------------------------------------------------------------------
// Forward projection: one thread per Gaussian.
// ---------------------------------------------------------------------------
// Projected state of Gaussian i in one view, written to projection row `row`.
template <int DEG>
__device__ __forceinline__ void project_one(const float* __restrict__ means, const float* __restrict__ log_scales,
                                            const float* __restrict__ quats,
                                            const float* __restrict__ opacity_logit, const float* __restrict__ sh,
                                            int i, long long row, const CamDev& cam, const SetDev& st,
                                            float4* __restrict__ xy, float4* __restrict__ conic_opac,
                                            float4* __restrict__ rgb_out, float* __restrict__ depth,
                                            short4* __restrict__ rect, uint32_t* __restrict__ tiles) {
    Stage s = integer_stage(means, log_scales, quats, i, cam, st);
    depth[row] = s.tz;
    if (s.culled) {              // no instance reads this row's mean, conic or colour
        tiles[row] = 0;
        rect[row] = make_short4(0, 0, -1, -1);
        return;
    }
    tiles[row] = (uint32_t)((s.x_hi - s.x_lo + 1) * (s.y_hi - s.y_lo + 1));
    rect[row] = make_short4((short)s.x_lo, (short)s.y_lo, (short)s.x_hi, (short)s.y_hi);
    // 2-D mean as a float pair: mu = f (t_xy / t_z) + c
    const float p0 = means[3 * i], p1 = means[3 * i + 1], p2 = means[3 * i + 2];
    F2 tx = dot3_plus(cam.R, p0, p1, p2, cam.t[0]);
    F2 ty = dot3_plus(cam.R + 3, p0, p1, p2, cam.t[1]);
    F2 tz = dot3_plus(cam.R + 6, p0, p1, p2, cam.t[2]);
    F2 mx = f2_add(f2_mul(f2_div(tx, tz), cam.fx), F2{cam.cx, 0.0f});
    F2 my = f2_add(f2_mul(f2_div(ty, tz), cam.fy), F2{cam.cy, 0.0f});
    xy[row] = make_float4(mx.hi, my.hi, mx.lo, my.lo);
    float det = s.a * s.c - s.b * s.b;
    float inv = 1.0f / det;
    float o = 1.0f / (1.0f + expf(-opacity_logit[i]));
    conic_opac[row] = make_float4(s.c * inv, -s.b * inv, s.a * inv, o);
    // view-dependent colour
    float d0 = p0 - cam.cc[0], d1 = p1 - cam.cc[1], d2 = p2 - cam.cc[2];
    float dn = sqrtf(d0 * d0 + d1 * d1 + d2 * d2);
    float inv_dn = 1.0f / dn;
    constexpr int K = (DEG + 1) * (DEG + 1);
    float Y[16];
    sh_basis(DEG, d0 * inv_dn, d1 * inv_dn, d2 * inv_dn, Y);
    float c[3 * K];
    load_sh<DEG>(sh, i, c);
    float r = 0.5f, g = 0.5f, b = 0.5f;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        r += Y[k] * c[3 * k];
        g += Y[k] * c[3 * k + 1];
        b += Y[k] * c[3 * k + 2];
    }
    rgb_out[row] = make_float4(fmaxf(r, 0.0f), fmaxf(g, 0.0f), fmaxf(b, 0.0f), 0.0f);
}

// One thread per projection row (view v, Gaussian i of view v's scene).
template <int DEG>
__global__ void __launch_bounds__(256, 6) project_kernel(ScenesDev sc, ViewsDev vd, SetDev st,
    float4* __restrict__ xy, float4* __restrict__ conic_opac, float4* __restrict__ rgb_out,
    float* __restrict__ depth, short4* __restrict__ rect, uint32_t* __restrict__ tiles) {
    pdl_wait_and_trigger();
    const long long row = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (row >= vd.row_off[vd.nv]) return;
    const int v = view_of_row(vd, row);
    const int i = (int)(row - vd.row_off[v]);
    project_one<DEG>(sc.means[v], sc.log_scales[v], sc.quats[v], sc.opacity_logit[v], sc.sh[v], i, row, vd.cam[v],
                     st, xy, conic_opac, rgb_out, depth, rect, tiles);
}

// Views that share one scene of n Gaussians (rows v n + i): one thread per
// Gaussian walks all the views, so that its parameters and SH row come from
// DRAM once and from the caches for the other views (the per-row kernel
// streams every view's rows, and the scene with them, one view after another).
template <int DEG>
__global__ void __launch_bounds__(256, 4) project_views_kernel(ScenesDev sc, ViewsDev vd, SetDev st, int n,
    float4* __restrict__ xy, float4* __restrict__ conic_opac, float4* __restrict__ rgb_out,
    float* __restrict__ depth, short4* __restrict__ rect, uint32_t* __restrict__ tiles) {
    pdl_wait_and_trigger();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int v = 0; v < vd.nv; ++v)
        project_one<DEG>(sc.means[0], sc.log_scales[0], sc.quats[0], sc.opacity_logit[0], sc.sh[0], i,
                         (long long)v * n + i, vd.cam[v], st, xy, conic_opac, rgb_out, depth, rect, tiles);
}

cudaError_t launch_project(const ScenesDev& sc, int sh_degree, const ViewsDev& vd, const SetDev& st,
                           const sgs_proj& out, cudaStream_t stream) {
    const long long rows = vd.row_off[vd.nv];
    if (rows == 0) return cudaSuccess;
    // several views of one scene with the same rows each: the per-Gaussian form
    bool shared = vd.nv > 1;
    const int n = vd.row_off[1] - vd.row_off[0];
    for (int v = 1; v < vd.nv && shared; ++v)
        shared = vd.row_off[v + 1] - vd.row_off[v] == n && sc.means[v] == sc.means[0] &&
                 sc.log_scales[v] == sc.log_scales[0] && sc.quats[v] == sc.quats[0] &&
                 sc.opacity_logit[v] == sc.opacity_logit[0] && sc.sh[v] == sc.sh[0];
    if (shared) {
        auto kern = sh_degree == 0 ? project_views_kernel<0>
                  : sh_degree == 1 ? project_views_kernel<1>
                  : sh_degree == 2 ? project_views_kernel<2> : project_views_kernel<3>;
        (void)launch_pdl(kern, dim3((n + 255) / 256), dim3(256), 0, stream, sc, vd, st, n,
                         reinterpret_cast<float4*>(out.xy), reinterpret_cast<float4*>(out.conic_opac),
                         reinterpret_cast<float4*>(out.rgb), out.depth, reinterpret_cast<short4*>(out.rect),
                         out.tiles_touched);
    } else {
        const int blocks = (int)((rows + 255) / 256);
        auto kern = sh_degree == 0 ? project_kernel<0>
                  : sh_degree == 1 ? project_kernel<1>
                  : sh_degree == 2 ? project_kernel<2> : project_kernel<3>;
        (void)launch_pdl(kern, dim3(blocks), dim3(256), 0, stream, sc, vd, st, reinterpret_cast<float4*>(out.xy),
                         reinterpret_cast<float4*>(out.conic_opac), reinterpret_cast<float4*>(out.rgb), out.depth,
                         reinterpret_cast<short4*>(out.rect), out.tiles_touched);
    }
    note_launch();
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Adjoint of the projection plus the lift of the splitting accumulators.
// g2d row (16 floats; 9 used), from the rasteriser's backward pass, with
// w = dL/dalpha * alpha and d = x - mu per composited, unclamped pair:
//   0..1 sum w d,  2..4 D = sum w d d^T (xx, xy, yy),  5 a0 = sum w,
//   6..8 dL/drgb.
// Then dL/dmu = Q sum w d, dL/dQ = -D/2 (the off-diagonal value counted once:
// -D_xy), dL/dopacity = a0 / o, and the splitting accumulator
// A2 = sum w u u^T = Q D Q (u = Q d), so this view adds
// S += P^T (A2 - a0 Q) P.
//
// One thread per Gaussian; each warp stages its 32 Gaussians' SH rows through
// shared memory so that the 3K-float rows are read and updated with coalesced
// accesses.
// ---------------------------------------------------------------------------

// Geometry adjoint of one Gaussian in one view: adds the view's splitting
// matrix to S6 and its parameter gradients to the accumulators.
template <bool PO, bool LS>
__device__ __forceinline__ void geometry_adjoint(const CamDev& cam, float p0, float p1, float p2, float4 q4,
                                                 const float* sc, float4 co, const float* gg, const float* gh,
                                                 float* S6, float* Spo, float* Sls,
                                                 float& gm0, float& gm1, float& gm2, float& gl0, float& gl1,
                                                 float& gl2, float4& gq, float& glog) {
    const float* R = cam.R;
    const float fx = cam.fx, fy = cam.fy;
    const float tx = R[0] * p0 + R[1] * p1 + R[2] * p2 + cam.t[0];
    const float ty = R[3] * p0 + R[4] * p1 + R[5] * p2 + cam.t[1];
    const float tz = R[6] * p0 + R[7] * p1 + R[8] * p2 + cam.t[2];
    const float itz = 1.0f / tz, itz2 = itz * itz;
    const float rx = tx * itz, ry = ty * itz;
    const bool clx = (rx < -cam.limx) || (rx > cam.limx);
    const bool cly = (ry < -cam.limy) || (ry > cam.limy);
    const float ux = fminf(fmaxf(rx, -cam.limx), cam.limx);
    const float uy = fminf(fmaxf(ry, -cam.limy), cam.limy);
    const float J00 = fx * itz, J02 = -fx * ux * itz, J11 = fy * itz, J12 = -fy * uy * itz;
    float P[6];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        P[j] = J00 * R[j] + J02 * R[6 + j];
        P[3 + j] = J11 * R[3 + j] + J12 * R[6 + j];
    }
    const float inv_qn = rsqrtf(q4.x * q4.x + q4.y * q4.y + q4.z * q4.z + q4.w * q4.w);
    const float w = q4.x * inv_qn, x = q4.y * inv_qn, y = q4.z * inv_qn, z = q4.w * inv_qn;
    float Rq[9];
    Rq[0] = 1.0f - 2.0f * (y * y + z * z); Rq[1] = 2.0f * (x * y - w * z); Rq[2] = 2.0f * (x * z + w * y);
    Rq[3] = 2.0f * (x * y + w * z); Rq[4] = 1.0f - 2.0f * (x * x + z * z); Rq[5] = 2.0f * (y * z - w * x);
    Rq[6] = 2.0f * (x * z - w * y); Rq[7] = 2.0f * (y * z + w * x); Rq[8] = 1.0f - 2.0f * (x * x + y * y);
    float M[9];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) M[3 * r + c] = Rq[3 * r + c] * sc[c];
    float V[6];
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int j = 0; j < 3; ++j) V[3 * a + j] = P[3 * a] * M[j] + P[3 * a + 1] * M[3 + j] + P[3 * a + 2] * M[6 + j];
    const float Qa = co.x, Qb = co.y, Qc = co.z, o = co.w;
    const float sx = gg[0], sy = gg[1], D00 = gg[2], D01 = gg[3], D11 = gg[4], a0 = gg[5];
    const float dmx = Qa * sx + Qb * sy, dmy = Qb * sx + Qc * sy;

    // splitting matrix of this view: S += P^T (Q D Q - a0 Q) P
    {
        const float m00 = Qa * D00 + Qb * D01, m01 = Qa * D01 + Qb * D11;
        const float m10 = Qb * D00 + Qc * D01, m11 = Qb * D01 + Qc * D11;
        const float K00 = (m00 * Qa + m01 * Qb) - a0 * Qa;
        const float K01 = (m00 * Qb + m01 * Qc) - a0 * Qb;
        const float K11 = (m10 * Qb + m11 * Qc) - a0 * Qc;
        int k = 0;
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = a; b < 3; ++b)
                S6[k++] += K00 * P[a] * P[b] + K01 * (P[a] * P[3 + b] + P[3 + a] * P[b]) + K11 * P[3 + a] * P[3 + b];
    }
    // position-opacity block of the splitting matrix over theta = (p, o):
    // sum dL/dsigma G P^T Q d = P^T Q (sum w d) / o  (d^2 sigma / dp do = G Y)
    if constexpr (PO) {
        const float io = o > 0.0f ? 1.0f / o : 0.0f;
#pragma unroll
        for (int j = 0; j < 3; ++j) Spo[j] += (P[j] * dmx + P[3 + j] * dmy) * io;
    }
    // log-scale blocks of the splitting matrix over theta = (p, l, o), P
    // frozen: with a_k = P Rq e_k, b_k = Q a_k, t_k = b_k . d, s2_k = exp(2 l_k)
    // (dQ/dl_k = -2 s2_k b_k b_k^T), summed over the view's pixels with
    // w = dL/dsigma sigma through the moments of w d up to fourth order:
    //   p-l[j][k] = s2_k sum w t_k^2 (Q P e_j).d - 2 s2_k (P^T b_k)_j sum w t_k
    //   l-l[k][l] = s2_k s2_l sum w t_k^2 t_l^2 + 2 delta_kl s2_k sum w t_k^2
    //               - 4 s2_k s2_l (a_k . b_l) sum w t_k t_l
    //   l-o[k]    = s2_k sum w t_k^2 / o
    if constexpr (LS) {
        const float T0 = gh[0], T1 = gh[1], T2 = gh[2], T3 = gh[3];             // x3 x2y xy2 y3
        const float F0 = gh[4], F1 = gh[5], F2 = gh[6], F3 = gh[7], F4 = gh[8];  // x4 x3y x2y2 xy3 y4
        float ak0[3], ak1[3], bk0[3], bk1[3], s2[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            ak0[k] = P[0] * Rq[k] + P[1] * Rq[3 + k] + P[2] * Rq[6 + k];
            ak1[k] = P[3] * Rq[k] + P[4] * Rq[3 + k] + P[5] * Rq[6 + k];
            bk0[k] = Qa * ak0[k] + Qb * ak1[k];
            bk1[k] = Qb * ak0[k] + Qc * ak1[k];
            s2[k] = sc[k] * sc[k];
        }
        auto quad = [&](float u0, float u1, float v0, float v1) {
            return u0 * v0 * D00 + (u0 * v1 + u1 * v0) * D01 + u1 * v1 * D11;
        };
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const float q0 = Qa * P[j] + Qb * P[3 + j], q1 = Qb * P[j] + Qc * P[3 + j];
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const float u0 = bk0[k], u1 = bk1[k];
                const float cubic = u0 * u0 * q0 * T0 + (u0 * u0 * q1 + 2.0f * u0 * u1 * q0) * T1 +
                                    (2.0f * u0 * u1 * q1 + u1 * u1 * q0) * T2 + u1 * u1 * q1 * T3;
                const float tk = u0 * sx + u1 * sy;
                const float ptb = P[j] * u0 + P[3 + j] * u1;
                Sls[3 * j + k] += s2[k] * cubic - 2.0f * s2[k] * ptb * tk;
            }
        }
        int q = 9;
#pragma unroll
        for (int k = 0; k < 3; ++k)
#pragma unroll
            for (int l = k; l < 3; ++l) {
                const float u0 = bk0[k], u1 = bk1[k], v0 = bk0[l], v1 = bk1[l];
                const float quart = u0 * u0 * v0 * v0 * F0 +
                                    (2.0f * u0 * u0 * v0 * v1 + 2.0f * u0 * u1 * v0 * v0) * F1 +
                                    (u0 * u0 * v1 * v1 + 4.0f * u0 * u1 * v0 * v1 + u1 * u1 * v0 * v0) * F2 +
                                    (2.0f * u0 * u1 * v1 * v1 + 2.0f * u1 * u1 * v0 * v1) * F3 + u1 * u1 * v1 * v1 * F4;
                const float quv = quad(u0, u1, v0, v1);
                const float ckl = ak0[k] * v0 + ak1[k] * v1;
                Sls[q++] += s2[k] * s2[l] * quart + (k == l ? 2.0f * s2[k] * quv : 0.0f) -
                            4.0f * s2[k] * s2[l] * ckl * quv;
            }
        const float io = o > 0.0f ? 1.0f / o : 0.0f;
#pragma unroll
        for (int k = 0; k < 3; ++k) Sls[15 + k] += s2[k] * quad(bk0[k], bk1[k], bk0[k], bk1[k]) * io;
    }
    // opacity: dL/do = a0 / o (unclamped pairs carry alpha = o G)
    glog += (o > 0.0f ? a0 / o : 0.0f) * o * (1.0f - o);

    // 2-D mean
    float dt0 = dmx * fx * itz;
    float dt1 = dmy * fy * itz;
    float dt2 = -(dmx * fx * tx + dmy * fy * ty) * itz2;
    // conic -> Sigma2D: G2 = -Q GQ Q with GQ = -D/2
    const float dQa = -0.5f * D00, dQb = -D01, dQc = -0.5f * D11;
    const float h = 0.5f * dQb;
    const float t00 = Qa * dQa + Qb * h, t01 = Qa * h + Qb * dQc;
    const float t10 = Qb * dQa + Qc * h, t11 = Qb * h + Qc * dQc;
    const float G00 = -(t00 * Qa + t01 * Qb);
    const float Gs01 = -0.5f * ((t00 * Qb + t01 * Qc) + (t10 * Qa + t11 * Qb));
    const float G11 = -(t10 * Qb + t11 * Qc);
    // Sigma2D = V V^T, V = P M: dV = 2 G2 V; dP = dV M^T; dM = P^T dV
    float dV[6];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        dV[j] = 2.0f * (G00 * V[j] + Gs01 * V[3 + j]);
        dV[3 + j] = 2.0f * (Gs01 * V[j] + G11 * V[3 + j]);
    }
    float dJ[6];
#pragma unroll
    for (int a = 0; a < 2; ++a) {
        const float dP0 = dV[3 * a] * M[0] + dV[3 * a + 1] * M[1] + dV[3 * a + 2] * M[2];
        const float dP1 = dV[3 * a] * M[3] + dV[3 * a + 1] * M[4] + dV[3 * a + 2] * M[5];
        const float dP2 = dV[3 * a] * M[6] + dV[3 * a + 1] * M[7] + dV[3 * a + 2] * M[8];
#pragma unroll
        for (int k = 0; k < 3; ++k) dJ[3 * a + k] = dP0 * R[3 * k] + dP1 * R[3 * k + 1] + dP2 * R[3 * k + 2];
    }
    // J = [[fx/tz, 0, -fx ux/tz], [0, fy/tz, -fy uy/tz]], ux = clamp(tx/tz)
    dt2 += dJ[0] * (-fx * itz2) + dJ[4] * (-fy * itz2);
    {
        const float dux_dtx = clx ? 0.0f : itz;
        const float dux_dtz = clx ? 0.0f : -tx * itz2;
        dt0 += dJ[2] * (-fx * itz) * dux_dtx;
        dt2 += dJ[2] * ((-fx * itz) * dux_dtz + fx * ux * itz2);
        const float duy_dty = cly ? 0.0f : itz;
        const float duy_dtz = cly ? 0.0f : -ty * itz2;
        dt1 += dJ[5] * (-fy * itz) * duy_dty;
        dt2 += dJ[5] * ((-fy * itz) * duy_dtz + fy * uy * itz2);
    }
    // t = W p + t_w
    gm0 += R[0] * dt0 + R[3] * dt1 + R[6] * dt2;
    gm1 += R[1] * dt0 + R[4] * dt1 + R[7] * dt2;
    gm2 += R[2] * dt0 + R[5] * dt1 + R[8] * dt2;
    // scales and rotation: dM = P^T dV, dRq = dM diag(s); dL/dlog s_c = sum_r dRq[r][c] Rq[r][c]
    float dRq[9];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) dRq[3 * r + c] = (P[r] * dV[c] + P[3 + r] * dV[3 + c]) * sc[c];
    gl0 += dRq[0] * Rq[0] + dRq[3] * Rq[3] + dRq[6] * Rq[6];
    gl1 += dRq[1] * Rq[1] + dRq[4] * Rq[4] + dRq[7] * Rq[7];
    gl2 += dRq[2] * Rq[2] + dRq[5] * Rq[5] + dRq[8] * Rq[8];
    const float* d = dRq;
    const float dw = 2.0f * (-z * d[1] + y * d[2] + z * d[3] - x * d[5] - y * d[6] + x * d[7]);
    const float dx = 2.0f * (y * d[1] + z * d[2] + y * d[3] - 2.0f * x * d[4] - w * d[5] + z * d[6] + w * d[7] - 2.0f * x * d[8]);
    const float dy = 2.0f * (-2.0f * y * d[0] + x * d[1] + w * d[2] + x * d[3] + z * d[5] - w * d[6] + z * d[7] - 2.0f * y * d[8]);
    const float dz = 2.0f * (-2.0f * z * d[0] - w * d[1] + x * d[2] + w * d[3] - 2.0f * z * d[4] + y * d[5] + x * d[6] + y * d[7]);
    const float dot = dw * w + dx * x + dy * y + dz * z;
    gq.x += (dw - dot * w) * inv_qn;
    gq.y += (dx - dot * x) * inv_qn;
    gq.z += (dy - dot * y) * inv_qn;
    gq.w += (dz - dot * z) * inv_qn;
}

// One thread per Gaussian, looping over the views; each warp stages its 32
// Gaussians' SH rows (coefficients and gradient increments) through shared
// memory so that the 3K-float rows are read and updated with coalesced
// accesses.
// MULTI = false is the single-view case: no view loop, and the SH gradient
// increments overwrite the staged coefficients once they have been used.
template <int DEG, bool MULTI, bool PO, bool LS>
__global__ void __launch_bounds__(MULTI ? 64 : 128, MULTI ? 8 : (LS ? 3 : 7)) project_bwd_kernel(
    const float* __restrict__ means, const float* __restrict__ log_scales, const float* __restrict__ quats,
    const float* __restrict__ sh, int n, ViewsDev vd, const float4* __restrict__ conic_opac,
    const uint32_t* __restrict__ tiles, const float* __restrict__ g2d, const float* __restrict__ g2d_hi,
    int flags,
    float* __restrict__ g_means, float* __restrict__ g_ls, float* __restrict__ g_quats,
    float* __restrict__ g_logit, float* __restrict__ g_sh, float* __restrict__ S_accum,
    float* __restrict__ S_po_accum, float* __restrict__ S_ls_accum) {
    pdl_wait_and_trigger();
    constexpr int THREADS = MULTI ? 64 : 128;
    constexpr int K = (DEG + 1) * (DEG + 1);
    constexpr int K3 = 3 * K;
    constexpr int ROW = K3 + 1;                      // padded row: conflict-free per-thread access
    __shared__ float s_coef[THREADS / 32][32 * ROW];
    __shared__ float s_inc[MULTI ? THREADS / 32 : 1][MULTI ? 32 * ROW : 1];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int base = blockIdx.x * THREADS + warp * 32;
    if (base >= n) return;
    const int i = base + lane;
    float* wc = s_coef[warp];
    float* wi = MULTI ? s_inc[warp] : s_coef[warp];

    // views whose projection reached a tile (tiles_touched > 0)
    uint32_t tmask = 0u;
    const int nv = MULTI ? vd.nv : 1;
    if (i < n)
        for (int v = 0; v < nv; ++v)
            if (tiles[(long long)v * n + i] != 0u) tmask |= 1u << v;
    const uint32_t vis = __ballot_sync(0xffffffffu, tmask != 0u);
    const bool accumulate = (flags & kBwdAccumulateGrads) != 0;
    const bool reset_S = (flags & kBwdResetS) != 0;
    if (vis == 0u && accumulate && !reset_S) return;  // nothing in this warp reached a tile
    const int rows = min(32, n - base);
    if (vis == 0u && reset_S) {                      // unreached rows of a reset: zero splitting matrices
        for (int f = lane; f < 6 * rows; f += 32) S_accum[6 * (size_t)base + f] = 0.0f;
        if constexpr (PO)
            for (int f = lane; f < 3 * rows; f += 32) S_po_accum[3 * (size_t)base + f] = 0.0f;
        if constexpr (LS)
            for (int f = lane; f < 18 * rows; f += 32) S_ls_accum[18 * (size_t)base + f] = 0.0f;
        if (accumulate) return;
    }
    if (vis == 0u) {                                 // unreached rows: zero gradients, nothing staged
        for (int f = lane; f < 3 * rows; f += 32) {
            g_means[3 * (size_t)base + f] = 0.0f;
            g_ls[3 * (size_t)base + f] = 0.0f;
        }
        if (lane < rows) {
            reinterpret_cast<float4*>(g_quats)[base + lane] = make_float4(0.f, 0.f, 0.f, 0.f);
            g_logit[base + lane] = 0.0f;
        }
        if ((K3 & 3) == 0 && (reinterpret_cast<uintptr_t>(g_sh) & 15u) == 0) {
            float4* o4 = reinterpret_cast<float4*>(g_sh + (size_t)base * K3);
            for (int f = lane; f < rows * K3 / 4; f += 32) o4[f] = make_float4(0.f, 0.f, 0.f, 0.f);
        } else {
            for (int f = lane; f < rows * K3; f += 32) g_sh[(size_t)base * K3 + f] = 0.0f;
        }
        return;
    }
    // stage the SH coefficient rows of the reached Gaussians with asynchronous
    // 4-byte copies (all in flight at once, no registers), while the
    // accumulator rows and the parameters load; clear increments
    {
        const int nf = rows * K3;
        for (int f = lane; f < nf; f += 32) {
            const int r = f / K3;
            const int o = r * ROW + (f - r * K3);
            if ((vis >> r) & 1u) {
                const unsigned dst = (unsigned)__cvta_generic_to_shared(wc + o);
                asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(dst), "l"(sh + (size_t)base * K3 + f)
                             : "memory");
            }
            if constexpr (MULTI) wi[o] = 0.0f;
        }
        asm volatile("cp.async.commit_group;\n" ::: "memory");
    }
    // which views composited this Gaussian somewhere
    uint32_t vmask = 0u;
    for (int v = 0; v < nv; ++v) {
        if (!((tmask >> v) & 1u)) continue;
        const long long row = (long long)v * n + i;
        const float4* r4 = reinterpret_cast<const float4*>(g2d + (size_t)row * 16);
        const float4 a = r4[0], b = r4[1], c = r4[2];
        if (a.x != 0.f || a.y != 0.f || a.z != 0.f || a.w != 0.f || b.x != 0.f || b.y != 0.f || b.z != 0.f ||
            b.w != 0.f || c.x != 0.f)
            vmask |= 1u << v;
    }
    const bool work = vmask != 0u;
    const uint32_t need = __ballot_sync(0xffffffffu, work);

    // parameters of this lane's Gaussian (their loads overlap the SH copies)
    float p0 = 0.f, p1 = 0.f, p2 = 0.f, ls0 = 0.f, ls1 = 0.f, ls2 = 0.f;
    float4 q4 = make_float4(1.f, 0.f, 0.f, 0.f);
    if (work) {
        p0 = means[3 * i]; p1 = means[3 * i + 1]; p2 = means[3 * i + 2];
        q4 = reinterpret_cast<const float4*>(quats)[i];
        ls0 = log_scales[3 * i]; ls1 = log_scales[3 * i + 1]; ls2 = log_scales[3 * i + 2];
    }

    asm volatile("cp.async.wait_all;\n" ::: "memory");
    __syncwarp();

    float gm0 = 0.f, gm1 = 0.f, gm2 = 0.f, gl0 = 0.f, gl1 = 0.f, gl2 = 0.f, glog = 0.f;
    float4 gq = make_float4(0.f, 0.f, 0.f, 0.f);
    float S6[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    float Spo[3] = {0.f, 0.f, 0.f};
    float Sls[LS ? 18 : 1];
#pragma unroll
    for (int k = 0; k < (LS ? 18 : 1); ++k) Sls[k] = 0.0f;
    if (work) {
        const float sc[3] = {__expf(ls0), __expf(ls1), __expf(ls2)};
        const float* crow = wc + lane * ROW;
        float* irow = wi + lane * ROW;
        for (int v = 0; v < nv; ++v) {
            if (!((vmask >> v) & 1u)) continue;
            const CamDev& cam = vd.cam[v];
            const long long row = (long long)v * n + i;
            float gg[9];
            {
                const float4* r4 = reinterpret_cast<const float4*>(g2d + (size_t)row * 16);
                const float4 a = r4[0], b = r4[1], c = r4[2];
                gg[0] = a.x; gg[1] = a.y; gg[2] = a.z; gg[3] = a.w;
                gg[4] = b.x; gg[5] = b.y; gg[6] = b.z; gg[7] = b.w; gg[8] = c.x;
            }
            float gh[LS ? 9 : 1];
            if constexpr (LS) {
#pragma unroll
                for (int k = 0; k < 9; ++k) gh[k] = g2d_hi[(size_t)row * 16 + k];
            }
            geometry_adjoint<PO, LS>(cam, p0, p1, p2, q4, sc, conic_opac[row], gg, gh, S6, Spo, Sls, gm0, gm1, gm2,
                                     gl0, gl1, gl2, gq, glog);
            // colour (SH) of this view
            const float d0 = p0 - cam.cc[0], d1 = p1 - cam.cc[1], d2 = p2 - cam.cc[2];
            const float inv_dn = rsqrtf(d0 * d0 + d1 * d1 + d2 * d2);
            const float h0 = d0 * inv_dn, h1 = d1 * inv_dn, h2 = d2 * inv_dn;
            float Y[16];
            sh_basis(DEG, h0, h1, h2, Y);
            float raw0 = 0.5f, raw1 = 0.5f, raw2 = 0.5f;
#pragma unroll
            for (int k = 0; k < K; ++k) {
                raw0 += Y[k] * crow[3 * k];
                raw1 += Y[k] * crow[3 * k + 1];
                raw2 += Y[k] * crow[3 * k + 2];
            }
            const float gc0 = raw0 > 0.0f ? gg[6] : 0.0f;
            const float gc1 = raw1 > 0.0f ? gg[7] : 0.0f;
            const float gc2 = raw2 > 0.0f ? gg[8] : 0.0f;
            if constexpr (DEG > 0) {
                float wk[16];
#pragma unroll
                for (int k = 0; k < K; ++k) wk[k] = gc0 * crow[3 * k] + gc1 * crow[3 * k + 1] + gc2 * crow[3 * k + 2];
                float e0, e1, e2;
                sh_weighted_grad<DEG>(h0, h1, h2, wk, e0, e1, e2);
                const float pr = e0 * h0 + e1 * h1 + e2 * h2;
                gm0 += (e0 - pr * h0) * inv_dn;
                gm1 += (e1 - pr * h1) * inv_dn;
                gm2 += (e2 - pr * h2) * inv_dn;
            }
            if constexpr (MULTI) {
#pragma unroll
                for (int k = 0; k < K; ++k) {
                    irow[3 * k] += Y[k] * gc0;
                    irow[3 * k + 1] += Y[k] * gc1;
                    irow[3 * k + 2] += Y[k] * gc2;
                }
            } else {                                 // the coefficients are no longer needed
#pragma unroll
                for (int k = 0; k < K; ++k) {
                    irow[3 * k] = Y[k] * gc0;
                    irow[3 * k + 1] = Y[k] * gc1;
                    irow[3 * k + 2] = Y[k] * gc2;
                }
            }
        }
    }
    // splitting matrices: added (Algorithm 1 sums them over views and steps),
    // or, on a reset, written for every row (zeros where nothing composited)
    if (i < n && (work || reset_S)) {
        float* So = S_accum + (size_t)i * 6;
#pragma unroll
        for (int k = 0; k < 6; ++k) So[k] = reset_S ? S6[k] : So[k] + S6[k];
        if constexpr (PO) {
            float* Sp = S_po_accum + (size_t)i * 3;
#pragma unroll
            for (int k = 0; k < 3; ++k) Sp[k] = reset_S ? Spo[k] : Sp[k] + Spo[k];
        }
        if constexpr (LS) {
            float* Sl = S_ls_accum + (size_t)i * 18;
#pragma unroll
            for (int k = 0; k < 18; ++k) Sl[k] = reset_S ? Sls[k] : Sl[k] + Sls[k];
        }
    }
    if (i < n) {
        if (accumulate) {
            if (work) {
                g_means[3 * i] += gm0; g_means[3 * i + 1] += gm1; g_means[3 * i + 2] += gm2;
                g_ls[3 * i] += gl0; g_ls[3 * i + 1] += gl1; g_ls[3 * i + 2] += gl2;
                float4* gp = reinterpret_cast<float4*>(g_quats) + i;
                float4 t = *gp;
                t.x += gq.x; t.y += gq.y; t.z += gq.z; t.w += gq.w;
                *gp = t;
                g_logit[i] += glog;
            }
        } else {
            g_means[3 * i] = gm0; g_means[3 * i + 1] = gm1; g_means[3 * i + 2] = gm2;
            g_ls[3 * i] = gl0; g_ls[3 * i + 1] = gl1; g_ls[3 * i + 2] = gl2;
            reinterpret_cast<float4*>(g_quats)[i] = gq;
            g_logit[i] = glog;
        }
    }
    __syncwarp();

    // SH gradient rows (coalesced): added, or written (zeros for untouched rows)
    for (int f = lane; f < rows * K3; f += 32) {
        const int r = f / K3;
        const float val = ((need >> r) & 1u) ? wi[r * ROW + (f - r * K3)] : 0.0f;
        if (!accumulate)
            g_sh[(size_t)base * K3 + f] = val;
        else if ((need >> r) & 1u)
            g_sh[(size_t)base * K3 + f] += val;
    }
}

cudaError_t launch_project_bwd(const sgs_gaussians& g, const sgs_proj& proj, const ViewsDev& vd, const float* g2d,
                               const float* g2d_hi, int flags, const sgs_grads& grads, float* S_accum,
                               float* S_po_accum, float* S_ls_accum, cudaStream_t stream) {
    if (g.n == 0) return cudaSuccess;
    const bool multi = vd.nv > 1;
    const int threads = multi ? 64 : 128;
    const int blocks = (g.n + threads - 1) / threads;
    auto pick = [&](auto po) {
        constexpr bool PO = decltype(po)::value;
        return multi ? (g.sh_degree == 0 ? project_bwd_kernel<0, true, PO, false>
                      : g.sh_degree == 1 ? project_bwd_kernel<1, true, PO, false>
                      : g.sh_degree == 2 ? project_bwd_kernel<2, true, PO, false>
                                         : project_bwd_kernel<3, true, PO, false>)
                     : (g.sh_degree == 0 ? project_bwd_kernel<0, false, PO, false>
                      : g.sh_degree == 1 ? project_bwd_kernel<1, false, PO, false>
                      : g.sh_degree == 2 ? project_bwd_kernel<2, false, PO, false>
                                         : project_bwd_kernel<3, false, PO, false>);
    };
    // the (p, o) and (p, l, o) blocks are separate instantiations, so the
    // common position-only kernel carries none of their code; (p, l, o) is
    // single-view only
    auto kern = S_po_accum ? pick(std::true_type{}) : pick(std::false_type{});
    if (S_ls_accum && !multi)
        kern = g.sh_degree == 0 ? project_bwd_kernel<0, false, true, true>
             : g.sh_degree == 1 ? project_bwd_kernel<1, false, true, true>
             : g.sh_degree == 2 ? project_bwd_kernel<2, false, true, true> : project_bwd_kernel<3, false, true, true>;
    (void)launch_pdl(kern, dim3(blocks), dim3(threads), 0, stream, g.means, g.log_scales, g.quats, g.sh, g.n, vd,
                     reinterpret_cast<const float4*>(proj.conic_opac), proj.tiles_touched, g2d, g2d_hi,
                     flags, grads.means, grads.log_scales, grads.quats, grads.opacity_logit, grads.sh,
                     S_accum, S_po_accum, S_ls_accum);
    note_launch();
    return cudaGetLastError();
}

}  // namespace sgs
