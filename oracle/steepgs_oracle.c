/*
 * steepgs_oracle.c -- plain, slow CPU oracle for the SteepGS splitting path.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call this code:
 * only the tests, the smoke check and the CPU-baseline leg of the benchmark
 * load it.  It shares no code, header, table or constant generator with the
 * CUDA library.
 *
 * What it computes (paper: "Steepest Descent Density Control for Compact 3D
 * Gaussian Splatting", arXiv 2505.05587):
 *   - Section 3, Eq. sigma_3D / sigma_2D / alpha_blend: projection of each
 *     Gaussian and front-to-back alpha compositing of the depth-sorted list.
 *   - Section 3, Eq. loss: L1 photometric loss (SSIM dropped, as the paper does).
 *   - Section 4.4 and Algorithm 1: back-propagation of dL/dtheta and the
 *     per-Gaussian splitting matrix S = sum dl/dsigma * Hess_p(sigma), with the
 *     closed-form Hessian of Appendix "Deriving Hessian of Gaussian"
 *     (sigma (Y Y^T - P^T Sigma2D^-1 P), Y = P^T Sigma2D^-1 (x - Pi(p))).
 *   - Appendix "Eigendecomposition": trigonometric root formula for the
 *     minimum eigenpair of the 3x3 symmetric S; a cyclic Jacobi solver is kept
 *     beside it as an independent cross-check.
 *   - Theorem 2 / Algorithm 1: split into two offspring p +- eps v_min with
 *     opacity o/2, compacted by an exclusive prefix sum.
 *
 * Precision: float64 for every continuous quantity.  The *integer stage*
 * (depth key, 2-D mean, radius and tile rectangle, which decide tile
 * membership and sort order) is evaluated in float32 with one fixed sequence
 * of IEEE operations (compile with -ffp-contract=off), because those decisions
 * must be bit-identical to the CUDA path.  The scale activation inside that
 * stage uses a float32 exponential written out below (Cody-Waite reduction +
 * degree-7 Taylor polynomial), so that it is a fixed sequence of IEEE
 * operations too.
 *
 * Where the paper leaves a point open, the reading taken is stated at the
 * code that implements it.
 * Parity status: every exported function here is pinned by a CPU test
 * (tests/test_oracle_*.py) against finite differences, closed forms, library
 * routines or brute force.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define PI_D 3.14159265358979323846

typedef struct {
    const float *means;         /* [N,3] */
    const float *log_scales;    /* [N,3] */
    const float *quats;         /* [N,4] (w,x,y,z) */
    const float *opacity_logit; /* [N] */
    const float *sh;            /* [N,K,3] */
    int32_t n;
    int32_t sh_degree;
} orc_scene;

typedef struct {
    float R[9];
    float t[3];
    float fx, fy, cx, cy;
    int32_t width, height;
    float near_z;
} orc_camera;

typedef struct {
    int32_t tile_w, tile_h;
    float alpha_min, alpha_max, T_min, radius_sigma, dilation, fov_clamp;
    float bg[3];
} orc_settings;

/* ------------------------------------------------------------------------ */
/* Integer stage (float32, fixed IEEE operation sequence)                    */
/* ------------------------------------------------------------------------ */

/* exp(x) in float32: k = rint(x log2 e); r = (x - k ln2_hi) - k ln2_lo;
 * p = Taylor series of e^r to degree 7 (Horner); result p * 2^k.
 * ln2_hi has 15 significant bits so k*ln2_hi is exact for |k| <= 127. */
static float orc_exp_f32(float x)
{
    x = fminf(fmaxf(x, -87.0f), 88.0f);
    float k = rintf(x * 0x1.715476p+0f);
    float r = (x - k * 0x1.62e4p-1f) - k * 0x1.7f7d1cp-20f;
    float p = 0x1.a01a02p-13f;          /* 1/5040 */
    p = p * r + 0x1.6c16c2p-10f;        /* 1/720  */
    p = p * r + 0x1.111112p-7f;         /* 1/120  */
    p = p * r + 0x1.555556p-5f;         /* 1/24   */
    p = p * r + 0x1.555556p-3f;         /* 1/6    */
    p = p * r + 0.5f;
    p = p * r + 1.0f;
    p = p * r + 1.0f;
    int ki = (int)k;
    uint32_t bits = (uint32_t)(ki + 127) << 23;
    float two_k;
    memcpy(&two_k, &bits, 4);
    return p * two_k;
}

float orc_exp_f32_export(float x) { return orc_exp_f32(x); }

typedef struct {
    int culled;
    float tx, ty, tz, mx, my;
    float a, b, c;          /* Sigma2D (with dilation) */
    int x_lo, x_hi, y_lo, y_hi;
    int tiles;
} orc_istage;

/* Float32 integer stage of one Gaussian.  Sums are evaluated left to right,
 * every product and sum rounded to float32, no fused multiply-add. */
static orc_istage orc_integer_stage_one(const orc_scene *sc, const orc_camera *cam,
                                        const orc_settings *st, int i)
{
    orc_istage o;
    memset(&o, 0, sizeof(o));
    o.culled = 1;
    const float *p = sc->means + 3 * i;
    const float *R = cam->R;
    float tx = ((R[0] * p[0] + R[1] * p[1]) + R[2] * p[2]) + cam->t[0];
    float ty = ((R[3] * p[0] + R[4] * p[1]) + R[5] * p[2]) + cam->t[1];
    float tz = ((R[6] * p[0] + R[7] * p[1]) + R[8] * p[2]) + cam->t[2];
    o.tx = tx; o.ty = ty; o.tz = tz;
    if (!(tz > cam->near_z)) return o;
    float mx = (cam->fx * tx) / tz + cam->cx;
    float my = (cam->fy * ty) / tz + cam->cy;
    o.mx = mx; o.my = my;
    /* Jacobian of the pinhole projection with the off-screen clamp. */
    float limx = (st->fov_clamp * (0.5f * (float)cam->width)) / cam->fx;
    float limy = (st->fov_clamp * (0.5f * (float)cam->height)) / cam->fy;
    float ux = fminf(fmaxf(tx / tz, -limx), limx);
    float uy = fminf(fmaxf(ty / tz, -limy), limy);
    float J00 = cam->fx / tz, J02 = -(cam->fx * ux) / tz;
    float J11 = cam->fy / tz, J12 = -(cam->fy * uy) / tz;
    float T[6];
    for (int j = 0; j < 3; ++j) {
        T[j] = J00 * R[j] + J02 * R[6 + j];
        T[3 + j] = J11 * R[3 + j] + J12 * R[6 + j];
    }
    const float *q = sc->quats + 4 * i;
    float qn = sqrtf(((q[0] * q[0] + q[1] * q[1]) + q[2] * q[2]) + q[3] * q[3]);
    if (!(qn > 0.0f)) return o;
    float w = q[0] / qn, x = q[1] / qn, y = q[2] / qn, z = q[3] / qn;
    float Rq[9];
    Rq[0] = 1.0f - 2.0f * (y * y + z * z);
    Rq[1] = 2.0f * (x * y - w * z);
    Rq[2] = 2.0f * (x * z + w * y);
    Rq[3] = 2.0f * (x * y + w * z);
    Rq[4] = 1.0f - 2.0f * (x * x + z * z);
    Rq[5] = 2.0f * (y * z - w * x);
    Rq[6] = 2.0f * (x * z - w * y);
    Rq[7] = 2.0f * (y * z + w * x);
    Rq[8] = 1.0f - 2.0f * (x * x + y * y);
    const float *ls = sc->log_scales + 3 * i;
    float s[3] = {orc_exp_f32(ls[0]), orc_exp_f32(ls[1]), orc_exp_f32(ls[2])};
    float M[9];
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) M[3 * r + c] = Rq[3 * r + c] * s[c];
    float V[6];
    for (int a = 0; a < 2; ++a)
        for (int j = 0; j < 3; ++j)
            V[3 * a + j] = (T[3 * a + 0] * M[j] + T[3 * a + 1] * M[3 + j]) + T[3 * a + 2] * M[6 + j];
    float sa = ((V[0] * V[0] + V[1] * V[1]) + V[2] * V[2]) + st->dilation;
    float sb = (V[0] * V[3] + V[1] * V[4]) + V[2] * V[5];
    float sc2 = ((V[3] * V[3] + V[4] * V[4]) + V[5] * V[5]) + st->dilation;
    o.a = sa; o.b = sb; o.c = sc2;
    float det = sa * sc2 - sb * sb;
    if (!(det > 0.0f)) return o;
    float mid = 0.5f * (sa + sc2);
    float lam = mid + sqrtf(fmaxf(0.1f, mid * mid - det));
    float rad = ceilf(st->radius_sigma * sqrtf(lam));
    int gx = (cam->width + st->tile_w - 1) / st->tile_w;
    int gy = (cam->height + st->tile_h - 1) / st->tile_h;
    float fxlo = floorf((mx - rad) / (float)st->tile_w);
    float fxhi = floorf((mx + rad) / (float)st->tile_w);
    float fylo = floorf((my - rad) / (float)st->tile_h);
    float fyhi = floorf((my + rad) / (float)st->tile_h);
    if (!(fxhi >= 0.0f && fxlo <= (float)(gx - 1) && fyhi >= 0.0f && fylo <= (float)(gy - 1)))
        return o;
    o.x_lo = (int)fmaxf(fxlo, 0.0f);
    o.x_hi = (int)fminf(fxhi, (float)(gx - 1));
    o.y_lo = (int)fmaxf(fylo, 0.0f);
    o.y_hi = (int)fminf(fyhi, (float)(gy - 1));
    o.tiles = (o.x_hi - o.x_lo + 1) * (o.y_hi - o.y_lo + 1);
    o.culled = 0;
    return o;
}

int orc_integer_stage(const orc_scene *sc, const orc_camera *cam, const orc_settings *st,
                      float *mean2d, float *depth, int32_t *rect, int32_t *tiles)
{
    for (int i = 0; i < sc->n; ++i) {
        orc_istage o = orc_integer_stage_one(sc, cam, st, i);
        if (mean2d) { mean2d[2 * i] = o.mx; mean2d[2 * i + 1] = o.my; }
        if (depth) depth[i] = o.tz;
        if (rect) {
            rect[4 * i + 0] = o.x_lo; rect[4 * i + 1] = o.x_hi;
            rect[4 * i + 2] = o.y_lo; rect[4 * i + 3] = o.y_hi;
        }
        if (tiles) tiles[i] = o.culled ? 0 : o.tiles;
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Small float64 linear algebra                                              */
/* ------------------------------------------------------------------------ */

static void mat3_mul(const double *A, const double *B, double *C)
{
    double t[9];
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) {
            double s = 0.0;
            for (int k = 0; k < 3; ++k) s += A[3 * r + k] * B[3 * k + c];
            t[3 * r + c] = s;
        }
    memcpy(C, t, sizeof(t));
}

static void mat3_transpose(const double *A, double *B)
{
    double t[9];
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) t[3 * c + r] = A[3 * r + c];
    memcpy(B, t, sizeof(t));
}

/* ------------------------------------------------------------------------ */
/* Real spherical harmonics up to degree 3 (Section 3: colours are stored as  */
/* SH coefficients and converted to RGB at render time).                     */
/* Y_k are orthonormal on the unit sphere; sign pattern (-1)^m on m != 0      */
/* terms of odd order as in the common graphics convention.                  */
/* ------------------------------------------------------------------------ */

static void sh_basis(int degree, const double d[3], double *Y, double *dY /* [K][3] or NULL */)
{
    double x = d[0], y = d[1], z = d[2];
    const double c0 = 0.5 / sqrt(PI_D);
    const double c1 = sqrt(3.0 / (4.0 * PI_D));
    const double c2a = 0.5 * sqrt(15.0 / PI_D);
    const double c2b = 0.25 * sqrt(5.0 / PI_D);
    const double c2c = 0.25 * sqrt(15.0 / PI_D);
    const double c3a = 0.25 * sqrt(35.0 / (2.0 * PI_D));
    const double c3b = 0.5 * sqrt(105.0 / PI_D);
    const double c3c = 0.25 * sqrt(21.0 / (2.0 * PI_D));
    const double c3d = 0.25 * sqrt(7.0 / PI_D);
    const double c3e = 0.25 * sqrt(105.0 / PI_D);
    int K = (degree + 1) * (degree + 1);
    if (dY) memset(dY, 0, sizeof(double) * 3 * K);
    Y[0] = c0;
    if (degree < 1) return;
    Y[1] = -c1 * y; Y[2] = c1 * z; Y[3] = -c1 * x;
    if (dY) { dY[3 * 1 + 1] = -c1; dY[3 * 2 + 2] = c1; dY[3 * 3 + 0] = -c1; }
    if (degree < 2) return;
    Y[4] = c2a * x * y;
    Y[5] = -c2a * y * z;
    Y[6] = c2b * (2.0 * z * z - x * x - y * y);
    Y[7] = -c2a * x * z;
    Y[8] = c2c * (x * x - y * y);
    if (dY) {
        dY[12] = c2a * y; dY[13] = c2a * x; dY[14] = 0;
        dY[15] = 0; dY[16] = -c2a * z; dY[17] = -c2a * y;
        dY[18] = -2.0 * c2b * x; dY[19] = -2.0 * c2b * y; dY[20] = 4.0 * c2b * z;
        dY[21] = -c2a * z; dY[22] = 0; dY[23] = -c2a * x;
        dY[24] = 2.0 * c2c * x; dY[25] = -2.0 * c2c * y; dY[26] = 0;
    }
    if (degree < 3) return;
    Y[9] = -c3a * y * (3.0 * x * x - y * y);
    Y[10] = c3b * x * y * z;
    Y[11] = -c3c * y * (4.0 * z * z - x * x - y * y);
    Y[12] = c3d * z * (2.0 * z * z - 3.0 * x * x - 3.0 * y * y);
    Y[13] = -c3c * x * (4.0 * z * z - x * x - y * y);
    Y[14] = c3e * z * (x * x - y * y);
    Y[15] = -c3a * x * (x * x - 3.0 * y * y);
    if (dY) {
        dY[27] = -c3a * 6.0 * x * y;           dY[28] = -c3a * (3.0 * x * x - 3.0 * y * y); dY[29] = 0;
        dY[30] = c3b * y * z;                  dY[31] = c3b * x * z;                         dY[32] = c3b * x * y;
        dY[33] = c3c * 2.0 * x * y;            dY[34] = -c3c * (4.0 * z * z - x * x - 3.0 * y * y); dY[35] = -c3c * 8.0 * y * z;
        dY[36] = -c3d * 6.0 * x * z;           dY[37] = -c3d * 6.0 * y * z;                  dY[38] = c3d * (6.0 * z * z - 3.0 * x * x - 3.0 * y * y);
        dY[39] = -c3c * (4.0 * z * z - 3.0 * x * x - y * y); dY[40] = c3c * 2.0 * x * y;     dY[41] = -c3c * 8.0 * x * z;
        dY[42] = c3e * 2.0 * x * z;            dY[43] = -c3e * 2.0 * y * z;                  dY[44] = c3e * (x * x - y * y);
        dY[45] = -c3a * (3.0 * x * x - 3.0 * y * y); dY[46] = c3a * 6.0 * x * y;             dY[47] = 0;
    }
}

void orc_sh_basis(int degree, const double *dirs, int n, double *Y, double *dY)
{
    int K = (degree + 1) * (degree + 1);
    for (int i = 0; i < n; ++i) sh_basis(degree, dirs + 3 * i, Y + K * i, dY ? dY + 3 * K * i : NULL);
}

/* ------------------------------------------------------------------------ */
/* Float64 projection of one Gaussian into one view (Section 3, Eq. sigma_2D, */
/* footnote on the affine Pi: Sigma2D = P Sigma P^T with P the local 2x3      */
/* linearisation of the pinhole projection at p).                           */
/* ------------------------------------------------------------------------ */

typedef struct {
    orc_istage is;        /* float32 integer stage (membership and order) */
    double t[3];          /* camera-space mean */
    double mu[2];         /* 2-D mean */
    double ux, uy;        /* clamped tx/tz, ty/tz */
    int clx, cly;         /* 1 if the clamp is active */
    double J[6];          /* 2x3 Jacobian of the pinhole map (camera space) */
    double P[6];          /* 2x3 = J W : linearisation of Pi at p */
    double qhat[4], qnorm;
    double Rq[9], s[3], M[9], Sig3[9];
    double Sig2[3];       /* a, b, c (with dilation) */
    double Q[3];          /* inverse: a, b, c */
    double o;             /* opacity */
    double dir[3], dnorm; /* view direction p - camera centre */
    double rgb_raw[3], rgb[3];
} orc_proj;

static void project_one(const orc_scene *sc, const orc_camera *cam, const orc_settings *st,
                        int i, orc_proj *pr)
{
    memset(pr, 0, sizeof(*pr));
    pr->is = orc_integer_stage_one(sc, cam, st, i);
    double R[9], tw[3];
    for (int k = 0; k < 9; ++k) R[k] = cam->R[k];
    for (int k = 0; k < 3; ++k) tw[k] = cam->t[k];
    double p[3] = {sc->means[3 * i], sc->means[3 * i + 1], sc->means[3 * i + 2]};
    for (int r = 0; r < 3; ++r) pr->t[r] = R[3 * r] * p[0] + R[3 * r + 1] * p[1] + R[3 * r + 2] * p[2] + tw[r];
    double fx = cam->fx, fy = cam->fy, cx = cam->cx, cy = cam->cy;
    double tx = pr->t[0], ty = pr->t[1], tz = pr->t[2];
    if (pr->is.culled) return;
    pr->mu[0] = fx * tx / tz + cx;
    pr->mu[1] = fy * ty / tz + cy;
    double limx = (double)st->fov_clamp * 0.5 * cam->width / fx;
    double limy = (double)st->fov_clamp * 0.5 * cam->height / fy;
    double ux = tx / tz, uy = ty / tz;
    pr->clx = (ux < -limx || ux > limx);
    pr->cly = (uy < -limy || uy > limy);
    pr->ux = ux < -limx ? -limx : (ux > limx ? limx : ux);
    pr->uy = uy < -limy ? -limy : (uy > limy ? limy : uy);
    pr->J[0] = fx / tz; pr->J[1] = 0.0; pr->J[2] = -fx * pr->ux / tz;
    pr->J[3] = 0.0; pr->J[4] = fy / tz; pr->J[5] = -fy * pr->uy / tz;
    for (int a = 0; a < 2; ++a)
        for (int j = 0; j < 3; ++j) {
            double s = 0.0;
            for (int k = 0; k < 3; ++k) s += pr->J[3 * a + k] * R[3 * k + j];
            pr->P[3 * a + j] = s;
        }
    const float *q = sc->quats + 4 * i;
    double qn = sqrt((double)q[0] * q[0] + (double)q[1] * q[1] + (double)q[2] * q[2] + (double)q[3] * q[3]);
    pr->qnorm = qn;
    for (int k = 0; k < 4; ++k) pr->qhat[k] = q[k] / qn;
    double w = pr->qhat[0], x = pr->qhat[1], y = pr->qhat[2], z = pr->qhat[3];
    double *Rq = pr->Rq;
    Rq[0] = 1 - 2 * (y * y + z * z); Rq[1] = 2 * (x * y - w * z); Rq[2] = 2 * (x * z + w * y);
    Rq[3] = 2 * (x * y + w * z); Rq[4] = 1 - 2 * (x * x + z * z); Rq[5] = 2 * (y * z - w * x);
    Rq[6] = 2 * (x * z - w * y); Rq[7] = 2 * (y * z + w * x); Rq[8] = 1 - 2 * (x * x + y * y);
    for (int k = 0; k < 3; ++k) pr->s[k] = exp((double)sc->log_scales[3 * i + k]);
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) pr->M[3 * r + c] = Rq[3 * r + c] * pr->s[c];
    double Mt[9];
    mat3_transpose(pr->M, Mt);
    mat3_mul(pr->M, Mt, pr->Sig3);
    /* Sigma2D = P Sigma3D P^T + dilation I */
    double PS[6];
    for (int a = 0; a < 2; ++a)
        for (int j = 0; j < 3; ++j) {
            double s = 0.0;
            for (int k = 0; k < 3; ++k) s += pr->P[3 * a + k] * pr->Sig3[3 * k + j];
            PS[3 * a + j] = s;
        }
    double S2[4];
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) {
            double s = 0.0;
            for (int k = 0; k < 3; ++k) s += PS[3 * a + k] * pr->P[3 * b + k];
            S2[2 * a + b] = s;
        }
    pr->Sig2[0] = S2[0] + st->dilation;
    pr->Sig2[1] = 0.5 * (S2[1] + S2[2]);
    pr->Sig2[2] = S2[3] + st->dilation;
    double det = pr->Sig2[0] * pr->Sig2[2] - pr->Sig2[1] * pr->Sig2[1];
    pr->Q[0] = pr->Sig2[2] / det;
    pr->Q[1] = -pr->Sig2[1] / det;
    pr->Q[2] = pr->Sig2[0] / det;
    pr->o = 1.0 / (1.0 + exp(-(double)sc->opacity_logit[i]));
    /* colour from SH at the direction from the camera centre c = -R^T t */
    double cc[3];
    for (int k = 0; k < 3; ++k) cc[k] = -(R[k] * tw[0] + R[3 + k] * tw[1] + R[6 + k] * tw[2]);
    for (int k = 0; k < 3; ++k) pr->dir[k] = p[k] - cc[k];
    pr->dnorm = sqrt(pr->dir[0] * pr->dir[0] + pr->dir[1] * pr->dir[1] + pr->dir[2] * pr->dir[2]);
    double dh[3] = {pr->dir[0] / pr->dnorm, pr->dir[1] / pr->dnorm, pr->dir[2] / pr->dnorm};
    int K = (sc->sh_degree + 1) * (sc->sh_degree + 1);
    double Y[16];
    sh_basis(sc->sh_degree, dh, Y, NULL);
    for (int ch = 0; ch < 3; ++ch) {
        double v = 0.5;
        for (int k = 0; k < K; ++k) v += Y[k] * sc->sh[(size_t)(i * K + k) * 3 + ch];
        pr->rgb_raw[ch] = v;
        pr->rgb[ch] = v > 0.0 ? v : 0.0;
    }
}

int orc_project(const orc_scene *sc, const orc_camera *cam, const orc_settings *st,
                double *mean2d, double *conic, double *opacity, double *rgb, double *P,
                double *depth, int32_t *tiles)
{
    orc_proj pr;
    for (int i = 0; i < sc->n; ++i) {
        project_one(sc, cam, st, i, &pr);
        if (mean2d) { mean2d[2 * i] = pr.mu[0]; mean2d[2 * i + 1] = pr.mu[1]; }
        if (conic) for (int k = 0; k < 3; ++k) conic[3 * i + k] = pr.Q[k];
        if (opacity) opacity[i] = pr.o;
        if (rgb) for (int k = 0; k < 3; ++k) rgb[3 * i + k] = pr.rgb[k];
        if (P) for (int k = 0; k < 6; ++k) P[6 * i + k] = pr.P[k];
        if (depth) depth[i] = pr.t[2];
        if (tiles) tiles[i] = pr.is.culled ? 0 : pr.is.tiles;
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Binning and depth sort: one instance per (Gaussian, covered tile), ordered */
/* by (tile id, float32 depth bits, Gaussian id).  (Section 3: 3DGS sorts the */
/* primitives by view-dependent depth before compositing.)                   */
/* ------------------------------------------------------------------------ */

typedef struct { uint64_t key; uint32_t gid; } orc_inst;

static int inst_cmp(const void *pa, const void *pb)
{
    const orc_inst *a = (const orc_inst *)pa, *b = (const orc_inst *)pb;
    if (a->key != b->key) return a->key < b->key ? -1 : 1;
    if (a->gid != b->gid) return a->gid < b->gid ? -1 : 1;
    return 0;
}

static uint32_t f32_bits(float f) { uint32_t u; memcpy(&u, &f, 4); return u; }

/* Returns the number of instances M; fills arrays when capacity allows. */
int64_t orc_bin_sort(const orc_scene *sc, const orc_camera *cam, const orc_settings *st,
                     uint64_t *keys, uint32_t *gids, uint32_t *ranges, int64_t capacity)
{
    int gx = (cam->width + st->tile_w - 1) / st->tile_w;
    int gy = (cam->height + st->tile_h - 1) / st->tile_h;
    int64_t M = 0;
    orc_istage *is = (orc_istage *)malloc(sizeof(orc_istage) * (size_t)(sc->n > 0 ? sc->n : 1));
    for (int i = 0; i < sc->n; ++i) {
        is[i] = orc_integer_stage_one(sc, cam, st, i);
        if (!is[i].culled) M += is[i].tiles;
    }
    if (M > capacity || keys == NULL) { free(is); return M; }
    orc_inst *inst = (orc_inst *)malloc(sizeof(orc_inst) * (size_t)(M > 0 ? M : 1));
    int64_t m = 0;
    for (int i = 0; i < sc->n; ++i) {
        if (is[i].culled) continue;
        uint32_t db = f32_bits(is[i].tz);
        for (int ty = is[i].y_lo; ty <= is[i].y_hi; ++ty)
            for (int tx = is[i].x_lo; tx <= is[i].x_hi; ++tx) {
                uint64_t tile = (uint64_t)(ty * gx + tx);
                inst[m].key = (tile << 32) | db;
                inst[m].gid = (uint32_t)i;
                ++m;
            }
    }
    qsort(inst, (size_t)M, sizeof(orc_inst), inst_cmp);
    for (int t = 0; t < gx * gy; ++t) { ranges[2 * t] = 0; ranges[2 * t + 1] = 0; }
    for (int64_t k = 0; k < M; ++k) {
        keys[k] = inst[k].key;
        gids[k] = inst[k].gid;
        uint32_t tile = (uint32_t)(inst[k].key >> 32);
        if (k == 0 || (uint32_t)(inst[k - 1].key >> 32) != tile) ranges[2 * tile] = (uint32_t)k;
        if (k == M - 1 || (uint32_t)(inst[k + 1].key >> 32) != tile) ranges[2 * tile + 1] = (uint32_t)(k + 1);
    }
    (void)gy;
    free(inst);
    free(is);
    return M;
}

/* ------------------------------------------------------------------------ */
/* Shared per-view state for render / backward                              */
/* ------------------------------------------------------------------------ */

typedef struct {
    int n, gx, gy, ntiles;
    orc_proj *pr;
    uint32_t *gids;
    uint32_t *ranges;
    int64_t M;
} orc_view;

static int view_build(const orc_scene *sc, const orc_camera *cam, const orc_settings *st, orc_view *v)
{
    v->n = sc->n;
    v->gx = (cam->width + st->tile_w - 1) / st->tile_w;
    v->gy = (cam->height + st->tile_h - 1) / st->tile_h;
    v->ntiles = v->gx * v->gy;
    v->pr = (orc_proj *)malloc(sizeof(orc_proj) * (size_t)(sc->n > 0 ? sc->n : 1));
    for (int i = 0; i < sc->n; ++i) project_one(sc, cam, st, i, &v->pr[i]);
    v->M = orc_bin_sort(sc, cam, st, NULL, NULL, NULL, 0);
    uint64_t *keys = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(v->M > 0 ? v->M : 1));
    v->gids = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(v->M > 0 ? v->M : 1));
    v->ranges = (uint32_t *)malloc(sizeof(uint32_t) * 2 * (size_t)v->ntiles);
    orc_bin_sort(sc, cam, st, keys, v->gids, v->ranges, v->M);
    free(keys);
    return 0;
}

static void view_free(orc_view *v)
{
    free(v->pr); free(v->gids); free(v->ranges);
}

/* Evaluate the 2-D Gaussian of projected state (mu, Q) at pixel offset. */
static double gauss2d(const double *mu, const double *Q, double px, double py, double *dx, double *dy)
{
    *dx = px - mu[0];
    *dy = py - mu[1];
    double power = -0.5 * (Q[0] * (*dx) * (*dx) + 2.0 * Q[1] * (*dx) * (*dy) + Q[2] * (*dy) * (*dy));
    return exp(power);
}

/* Conic of Gaussian pr in the frozen model (P fixed) with its log-scales   */
/* moved by dls: Sigma2D = P Rq diag(exp(2 (l + dls))) Rq^T P^T + dilation I. */
static void frozen_conic(const orc_proj *pr, const orc_settings *st, const double *dls, double *Q)
{
    double a[2][3];
    for (int u = 0; u < 2; ++u)
        for (int k = 0; k < 3; ++k) {
            double v = 0.0;
            for (int j = 0; j < 3; ++j) v += pr->P[3 * u + j] * pr->Rq[3 * j + k];
            a[u][k] = v;                        /* a_k = P Rq e_k, component u */
        }
    double S2[3] = {st->dilation, 0.0, st->dilation};
    for (int k = 0; k < 3; ++k) {
        double s2 = pr->s[k] * pr->s[k] * exp(2.0 * (dls ? dls[k] : 0.0));
        S2[0] += s2 * a[0][k] * a[0][k];
        S2[1] += s2 * a[0][k] * a[1][k];
        S2[2] += s2 * a[1][k] * a[1][k];
    }
    double det = S2[0] * S2[2] - S2[1] * S2[1];
    Q[0] = S2[2] / det;
    Q[1] = -S2[1] / det;
    Q[2] = S2[0] / det;
}

/* ------------------------------------------------------------------------ */
/* Forward compositing (Section 3, Eq. alpha_blend):                         */
/*   alpha = min(alpha_max, o G); skipped if alpha < alpha_min; the walk stops */
/*   before a Gaussian whose compositing would take T below T_min;           */
/*   C = sum c alpha T + T_final bg.                                         */
/* band[pixel] flags a pixel where one of those decisions lies within a      */
/* relative 1e-5 of its threshold (float32 and float64 may disagree there).  */
/* ------------------------------------------------------------------------ */

#define BAND_REL 1e-5

static int near_thr(double v, double thr)
{
    return fabs(v - thr) <= BAND_REL * fabs(thr);
}

/* Rows [y0, y1) of the view; outputs are [(y1 - y0), W] (row py at py - y0). */
static void render_view(const orc_view *v, const orc_camera *cam, const orc_settings *st, int y0, int y1,
                        double *image, double *final_T, int32_t *n_contrib, uint8_t *band)
{
    int W = cam->width;
    for (int py = y0; py < y1; ++py)
        for (int px = 0; px < W; ++px) {
            int tile = (py / st->tile_h) * v->gx + (px / st->tile_w);
            uint32_t s = v->ranges[2 * tile], e = v->ranges[2 * tile + 1];
            double T = 1.0, C[3] = {0, 0, 0};
            int last = 0, b = 0;
            for (uint32_t k = s; k < e; ++k) {
                const orc_proj *pr = &v->pr[v->gids[k]];
                double dx, dy;
                double G = gauss2d(pr->mu, pr->Q, px, py, &dx, &dy);
                double araw = pr->o * G;
                double alpha = araw < st->alpha_max ? araw : st->alpha_max;
                b |= near_thr(araw, st->alpha_max) | near_thr(alpha, st->alpha_min);
                if (alpha < st->alpha_min) continue;
                double Tn = T * (1.0 - alpha);
                b |= near_thr(Tn, st->T_min);
                if (Tn < st->T_min) break;
                for (int ch = 0; ch < 3; ++ch) C[ch] += pr->rgb[ch] * alpha * T;
                T = Tn;
                last = (int)(k - s) + 1;
            }
            size_t pix = (size_t)(py - y0) * W + px;
            for (int ch = 0; ch < 3; ++ch) image[3 * pix + ch] = C[ch] + T * st->bg[ch];
            if (final_T) final_T[pix] = T;
            if (n_contrib) n_contrib[pix] = last;
            if (band) band[pix] = (uint8_t)(b != 0);
        }
}

int orc_render(const orc_scene *sc, const orc_camera *cam, const orc_settings *st,
               double *image, double *final_T, int32_t *n_contrib, uint8_t *band)
{
    orc_view v;
    view_build(sc, cam, st, &v);
    render_view(&v, cam, st, 0, cam->height, image, final_T, n_contrib, band);
    view_free(&v);
    return 0;
}

/* Rows [y0, y0 + h) of the full view (the same projection, tiles and lists as
 * the whole image); outputs are [h, W]. */
int orc_render_rows(const orc_scene *sc, const orc_camera *cam, const orc_settings *st, int y0, int h,
                    double *image, double *final_T, int32_t *n_contrib, uint8_t *band)
{
    if (y0 < 0 || h < 0 || y0 + h > cam->height) return -1;
    orc_view v;
    view_build(sc, cam, st, &v);
    render_view(&v, cam, st, y0, y0 + h, image, final_T, n_contrib, band);
    view_free(&v);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* L1 loss (Section 3, Eq. loss with l = |.|): mean over pixels and channels  */
/* of one view, then mean over the views; dL/dC = sign(C - Chat) / (3 H W V) */
/* ------------------------------------------------------------------------ */

double orc_l1_loss_grad(const double *image, const float *target, int H, int W, int n_views,
                        double *dL_dC)
{
    double norm = 1.0 / (3.0 * (double)H * (double)W * (double)n_views);
    double L = 0.0;
    for (size_t k = 0; k < (size_t)H * W * 3; ++k) {
        double r = image[k] - (double)target[k];
        L += fabs(r);
        if (dL_dC) dL_dC[k] = (r > 0 ? 1.0 : (r < 0 ? -1.0 : 0.0)) * norm;
    }
    return L * norm;
}

/* ------------------------------------------------------------------------ */
/* Backward pass with splitting matrices (Section 4.4, Algorithm 1).          */
/* Per pixel the composited list is replayed front to back, then walked back */
/* to front:                                                                 */
/*   dL/dalpha_i = T_i * sum_ch g_ch (c_i,ch - B_i,ch), where B_i is the      */
/*   colour seen behind Gaussian i (later Gaussians and the background,       */
/*   normalised by T_{i+1}).                                                  */
/*   S_i += dL/dalpha_i * alpha_i * (Y Y^T - P^T Q P), Y = P^T Q (x - mu)     */
/*   (the Appendix's Hessian of sigma w.r.t. p with P, Sigma2D, colour frozen)*/
/* A clamped alpha (o G > alpha_max) is a constant of the parameters: it      */
/* contributes neither gradient nor splitting matrix.                        */
/* The 2-D gradients are then chained to the parameters exactly.             */
/* ------------------------------------------------------------------------ */

typedef struct {
    double mu[2], Q[3], o, rgb[3];
} grad2d_t;

typedef struct {
    int gid;
    double alpha, T, G, dx, dy;
    int clamped;
} pair_t;

/* Rows [y0, y1) of the view; dL_dC is [(y1 - y0), W, 3] (row py at py - y0). */
static void backward_view(const orc_scene *sc, const orc_view *v, const orc_camera *cam,
                          const orc_settings *st, int y0, int y1, const double *dL_dC, grad2d_t *g2, double *S,
                          double *S_po, double *S_ls)
{
    int W = cam->width;
    pair_t *list = NULL;
    size_t cap = 0;
    for (int py = y0; py < y1; ++py)
        for (int px = 0; px < W; ++px) {
            int tile = (py / st->tile_h) * v->gx + (px / st->tile_w);
            uint32_t s = v->ranges[2 * tile], e = v->ranges[2 * tile + 1];
            if (cap < (size_t)(e - s)) {
                cap = (size_t)(e - s);
                list = (pair_t *)realloc(list, sizeof(pair_t) * cap);
            }
            int nl = 0;
            double T = 1.0;
            for (uint32_t k = s; k < e; ++k) {
                const orc_proj *pr = &v->pr[v->gids[k]];
                double dx, dy;
                double G = gauss2d(pr->mu, pr->Q, px, py, &dx, &dy);
                double araw = pr->o * G;
                int clamped = !(araw < st->alpha_max);
                double alpha = clamped ? st->alpha_max : araw;
                if (alpha < st->alpha_min) continue;
                double Tn = T * (1.0 - alpha);
                if (Tn < st->T_min) break;
                list[nl].gid = (int)v->gids[k];
                list[nl].alpha = alpha; list[nl].T = T; list[nl].G = G;
                list[nl].dx = dx; list[nl].dy = dy; list[nl].clamped = clamped;
                ++nl;
                T = Tn;
            }
            size_t pix = (size_t)(py - y0) * W + px;
            const double *g = dL_dC + 3 * pix;
            double B[3] = {st->bg[0], st->bg[1], st->bg[2]};
            for (int k = nl - 1; k >= 0; --k) {
                const pair_t *pp = &list[k];
                const orc_proj *pr = &v->pr[pp->gid];
                grad2d_t *gg = &g2[pp->gid];
                double dLda = 0.0;
                for (int ch = 0; ch < 3; ++ch) {
                    dLda += g[ch] * pp->T * (pr->rgb[ch] - B[ch]);
                    gg->rgb[ch] += g[ch] * pp->alpha * pp->T;
                }
                for (int ch = 0; ch < 3; ++ch) B[ch] = pp->alpha * pr->rgb[ch] + (1.0 - pp->alpha) * B[ch];
                if (pp->clamped) continue;
                /* alpha = o G, G = exp(-0.5 d^T Q d), d = x - mu */
                double dLdG = dLda * pr->o;
                gg->o += dLda * pp->G;
                double Qd0 = pr->Q[0] * pp->dx + pr->Q[1] * pp->dy;
                double Qd1 = pr->Q[1] * pp->dx + pr->Q[2] * pp->dy;
                gg->mu[0] += dLdG * pp->G * Qd0;
                gg->mu[1] += dLdG * pp->G * Qd1;
                gg->Q[0] += dLdG * pp->G * (-0.5 * pp->dx * pp->dx);
                gg->Q[1] += dLdG * pp->G * (-pp->dx * pp->dy);
                gg->Q[2] += dLdG * pp->G * (-0.5 * pp->dy * pp->dy);
                double Y[3];
                for (int j = 0; j < 3; ++j) Y[j] = pr->P[j] * Qd0 + pr->P[3 + j] * Qd1;
                if (S_ls) {
                    /* blocks of the Hessian of sigma = o exp(-d^T Q d / 2) over theta =  */
                    /* (p, l, o), l the log-scales, P frozen: with a_k = P Rq e_k,        */
                    /* b_k = Q a_k, t_k = b_k . d, c_kl = a_k . b_l, s2_k = exp(2 l_k):   */
                    /*  dQ/dl_k = -2 s2_k b_k b_k^T,  dsigma/dl_k = sigma s2_k t_k^2,      */
                    /*  d2/dp dl_k = sigma s2_k t_k^2 Y - 2 sigma s2_k t_k P^T b_k,        */
                    /*  d2/dl_k dl_l = sigma (s2_k s2_l t_k^2 t_l^2 + 2 delta_kl s2_k t_k^2 */
                    /*                  - 4 s2_k s2_l c_kl t_k t_l),                      */
                    /*  d2/dl_k do = G s2_k t_k^2.                                        */
                    /* Layout [N,18]: p-l (3x3, row p, column l), l-l (xx xy xz yy yz zz), */
                    /* l-o (3).                                                           */
                    double a[2][3], b[2][3], t[3], s2[3], c[3][3], Ptb[3][3];
                    for (int k = 0; k < 3; ++k) {
                        for (int u = 0; u < 2; ++u) {
                            double vv = 0.0;
                            for (int j = 0; j < 3; ++j) vv += pr->P[3 * u + j] * pr->Rq[3 * j + k];
                            a[u][k] = vv;
                        }
                        b[0][k] = pr->Q[0] * a[0][k] + pr->Q[1] * a[1][k];
                        b[1][k] = pr->Q[1] * a[0][k] + pr->Q[2] * a[1][k];
                        t[k] = b[0][k] * pp->dx + b[1][k] * pp->dy;
                        s2[k] = pr->s[k] * pr->s[k];
                        for (int j = 0; j < 3; ++j) Ptb[k][j] = pr->P[j] * b[0][k] + pr->P[3 + j] * b[1][k];
                    }
                    for (int k = 0; k < 3; ++k)
                        for (int l = 0; l < 3; ++l) c[k][l] = a[0][k] * b[0][l] + a[1][k] * b[1][l];
                    double sig = pp->alpha;
                    double *Sl = S_ls + 18 * (size_t)pp->gid;
                    for (int j = 0; j < 3; ++j)
                        for (int k = 0; k < 3; ++k)
                            Sl[3 * j + k] += dLda * (sig * s2[k] * t[k] * t[k] * Y[j] -
                                                     2.0 * sig * s2[k] * t[k] * Ptb[k][j]);
                    int q = 9;
                    for (int k = 0; k < 3; ++k)
                        for (int l = k; l < 3; ++l)
                            Sl[q++] += dLda * sig * (s2[k] * s2[l] * t[k] * t[k] * t[l] * t[l] +
                                                     (k == l ? 2.0 * s2[k] * t[k] * t[k] : 0.0) -
                                                     4.0 * s2[k] * s2[l] * c[k][l] * t[k] * t[l]);
                    for (int k = 0; k < 3; ++k) Sl[15 + k] += dLda * pp->G * s2[k] * t[k] * t[k];
                }
                if (S_po) {
                    /* mixed block of the Hessian of sigma = o G(p) w.r.t. theta = (p, o): */
                    /* d^2 sigma / dp do = dG/dp = G Y  (d^2 sigma / do^2 = 0)               */
                    double *So = S_po + 3 * (size_t)pp->gid;
                    for (int a = 0; a < 3; ++a) So[a] += dLda * pp->G * Y[a];
                }
                if (S) {
                    /* Hessian of sigma = alpha w.r.t. p (frozen P, Sigma2D, colour) */
                    double PQP[9];
                    /* (P^T Q P)_ab = Q00 P0a P0b + Q01 (P0a P1b + P1a P0b) + Q11 P1a P1b */
                    for (int a = 0; a < 3; ++a)
                        for (int b = 0; b < 3; ++b)
                            PQP[3 * a + b] = pr->Q[0] * (pr->P[a] * pr->P[b]) +
                                             pr->Q[1] * (pr->P[a] * pr->P[3 + b] + pr->P[3 + a] * pr->P[b]) +
                                             pr->Q[2] * (pr->P[3 + a] * pr->P[3 + b]);
                    double sigma = pp->alpha;
                    double *Si = S + 9 * (size_t)pp->gid;
                    for (int a = 0; a < 3; ++a)
                        for (int b = 0; b < 3; ++b)
                            Si[3 * a + b] += dLda * sigma * (Y[a] * Y[b] - PQP[3 * a + b]);
                }
            }
        }
    free(list);
}

/* Chain rule from the 2-D quantities to the parameters of one Gaussian. */
static void chain_to_params(const orc_scene *sc, const orc_camera *cam, const orc_proj *pr,
                            const grad2d_t *gg, int i, double *g_means, double *g_log_scales,
                            double *g_quats, double *g_logit, double *g_sh)
{
    double R[9];
    for (int k = 0; k < 9; ++k) R[k] = cam->R[k];
    double fx = cam->fx, fy = cam->fy;
    double tx = pr->t[0], ty = pr->t[1], tz = pr->t[2];
    double dt[3] = {0, 0, 0};
    double dp[3] = {0, 0, 0};
    /* opacity: o = sigmoid(logit) */
    g_logit[i] += gg->o * pr->o * (1.0 - pr->o);
    /* colour: rgb = max(0, 0.5 + sum_k Y_k(dir) sh_k) */
    int K = (sc->sh_degree + 1) * (sc->sh_degree + 1);
    double dh[3] = {pr->dir[0] / pr->dnorm, pr->dir[1] / pr->dnorm, pr->dir[2] / pr->dnorm};
    double Y[16], dY[48];
    sh_basis(sc->sh_degree, dh, Y, dY);
    double ddh[3] = {0, 0, 0};
    for (int ch = 0; ch < 3; ++ch) {
        if (!(pr->rgb_raw[ch] > 0.0)) continue;
        double gc = gg->rgb[ch];
        for (int k = 0; k < K; ++k) {
            g_sh[(size_t)(i * K + k) * 3 + ch] += Y[k] * gc;
            double c = sc->sh[(size_t)(i * K + k) * 3 + ch];
            for (int a = 0; a < 3; ++a) ddh[a] += gc * c * dY[3 * k + a];
        }
    }
    /* dir_hat = dir/|dir|: d dir_hat/d dir = (I - dh dh^T)/|dir| */
    double proj = ddh[0] * dh[0] + ddh[1] * dh[1] + ddh[2] * dh[2];
    for (int a = 0; a < 3; ++a) dp[a] += (ddh[a] - proj * dh[a]) / pr->dnorm;
    /* 2-D mean: mu = (fx tx/tz + cx, fy ty/tz + cy) */
    dt[0] += gg->mu[0] * fx / tz;
    dt[1] += gg->mu[1] * fy / tz;
    dt[2] += -gg->mu[0] * fx * tx / (tz * tz) - gg->mu[1] * fy * ty / (tz * tz);
    /* conic Q = Sigma2D^{-1}: with Q as a symmetric matrix whose off-diagonal  */
    /* value b appears twice, dL/dQ_01 = dL/dQ_10 = dL/db / 2.                  */
    double GQ[4] = {gg->Q[0], 0.5 * gg->Q[1], 0.5 * gg->Q[1], gg->Q[2]};
    double Qm[4] = {pr->Q[0], pr->Q[1], pr->Q[1], pr->Q[2]};
    double tmp[4], G2[4];
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) tmp[2 * a + b] = Qm[2 * a] * GQ[b] + Qm[2 * a + 1] * GQ[2 + b];
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) G2[2 * a + b] = -(tmp[2 * a] * Qm[b] + tmp[2 * a + 1] * Qm[2 + b]);
    /* Sigma2D = P Sigma3D P^T (+ dilation): dL/dSigma3D = P^T G2 P, dL/dP = 2 G2 P Sigma3D */
    double G3[9];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            double s = 0.0;
            for (int u = 0; u < 2; ++u)
                for (int w = 0; w < 2; ++w) s += pr->P[3 * u + a] * G2[2 * u + w] * pr->P[3 * w + b];
            G3[3 * a + b] = s;
        }
    double dP[6];
    for (int a = 0; a < 2; ++a)
        for (int j = 0; j < 3; ++j) {
            double s = 0.0;
            for (int w = 0; w < 2; ++w)
                for (int k = 0; k < 3; ++k) s += G2[2 * a + w] * pr->P[3 * w + k] * pr->Sig3[3 * k + j];
            dP[3 * a + j] = 2.0 * s;
        }
    /* P = J W: dL/dJ = dL/dP W^T */
    double dJ[6];
    for (int a = 0; a < 2; ++a)
        for (int k = 0; k < 3; ++k) {
            double s = 0.0;
            for (int j = 0; j < 3; ++j) s += dP[3 * a + j] * R[3 * k + j];
            dJ[3 * a + k] = s;
        }
    /* J = [[fx/tz, 0, -fx ux/tz], [0, fy/tz, -fy uy/tz]], ux = clamp(tx/tz) */
    dt[2] += dJ[0] * (-fx / (tz * tz)) + dJ[4] * (-fy / (tz * tz));
    {
        double dux_dtx = pr->clx ? 0.0 : 1.0 / tz;
        double dux_dtz = pr->clx ? 0.0 : -tx / (tz * tz);
        dt[0] += dJ[2] * (-fx / tz) * dux_dtx;
        dt[2] += dJ[2] * ((-fx / tz) * dux_dtz + fx * pr->ux / (tz * tz));
        double duy_dty = pr->cly ? 0.0 : 1.0 / tz;
        double duy_dtz = pr->cly ? 0.0 : -ty / (tz * tz);
        dt[1] += dJ[5] * (-fy / tz) * duy_dty;
        dt[2] += dJ[5] * ((-fy / tz) * duy_dtz + fy * pr->uy / (tz * tz));
    }
    /* t = W p + t_w */
    for (int a = 0; a < 3; ++a) dp[a] += R[a] * dt[0] + R[3 + a] * dt[1] + R[6 + a] * dt[2];
    for (int a = 0; a < 3; ++a) g_means[3 * i + a] += dp[a];
    /* Sigma3D = M M^T, M = Rq diag(s): dL/dM = 2 G3 M */
    double dM[9];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            double s = 0.0;
            for (int k = 0; k < 3; ++k) s += G3[3 * a + k] * pr->M[3 * k + b];
            dM[3 * a + b] = 2.0 * s;
        }
    double dRq[9];
    for (int b = 0; b < 3; ++b) {
        double ds = 0.0;
        for (int a = 0; a < 3; ++a) {
            ds += dM[3 * a + b] * pr->Rq[3 * a + b];
            dRq[3 * a + b] = dM[3 * a + b] * pr->s[b];
        }
        g_log_scales[3 * i + b] += ds * pr->s[b];
    }
    /* rotation from the unit quaternion (w,x,y,z) */
    double w = pr->qhat[0], x = pr->qhat[1], y = pr->qhat[2], z = pr->qhat[3];
    const double *d = dRq;
    double dw = 2.0 * (-z * d[1] + y * d[2] + z * d[3] - x * d[5] - y * d[6] + x * d[7]);
    double dx = 2.0 * (y * d[1] + z * d[2] + y * d[3] - 2.0 * x * d[4] - w * d[5] + z * d[6] + w * d[7] - 2.0 * x * d[8]);
    double dy = 2.0 * (-2.0 * y * d[0] + x * d[1] + w * d[2] + x * d[3] + z * d[5] - w * d[6] + z * d[7] - 2.0 * y * d[8]);
    double dz = 2.0 * (-2.0 * z * d[0] - w * d[1] + x * d[2] + w * d[3] - 2.0 * z * d[4] + y * d[5] + x * d[6] + y * d[7]);
    double dq[4] = {dw, dx, dy, dz};
    double dotq = dq[0] * w + dq[1] * x + dq[2] * y + dq[3] * z;
    for (int k = 0; k < 4; ++k) g_quats[4 * i + k] += (dq[k] - dotq * pr->qhat[k]) / pr->qnorm;
}

/* Accumulates (+=) parameter gradients and the full 3x3 splitting matrices of
 * rows [y0, y0 + h) of one view (dL_dC is [h, W, 3]; orc_backward: all rows),
 * pixels outside carrying no gradient; S_po (optional, [N,3]) accumulates the position-opacity block of
 * the splitting matrix over theta = (p, o).  grad2d (optional, [N,9] = mu 2,
 * conic a b c 3, opacity 1, rgb 3) receives this view's 2-D gradients
 * (overwritten). */
int orc_backward_rows(const orc_scene *sc, const orc_camera *cam, const orc_settings *st, int y0, int h,
                      const double *dL_dC, double *g_means, double *g_log_scales, double *g_quats,
                      double *g_logit, double *g_sh, double *S, double *S_po, double *S_ls, double *grad2d)
{
    if (y0 < 0 || h < 0 || y0 + h > cam->height) return -1;
    orc_view v;
    view_build(sc, cam, st, &v);
    grad2d_t *g2 = (grad2d_t *)calloc((size_t)(sc->n > 0 ? sc->n : 1), sizeof(grad2d_t));
    backward_view(sc, &v, cam, st, y0, y0 + h, dL_dC, g2, S, S_po, S_ls);
    for (int i = 0; i < sc->n; ++i) {
        if (grad2d) {
            double *o = grad2d + 9 * (size_t)i;
            o[0] = g2[i].mu[0]; o[1] = g2[i].mu[1];
            o[2] = g2[i].Q[0]; o[3] = g2[i].Q[1]; o[4] = g2[i].Q[2];
            o[5] = g2[i].o; o[6] = g2[i].rgb[0]; o[7] = g2[i].rgb[1]; o[8] = g2[i].rgb[2];
        }
        if (v.pr[i].is.culled) continue;
        chain_to_params(sc, cam, &v.pr[i], &g2[i], i, g_means, g_log_scales, g_quats, g_logit, g_sh);
    }
    free(g2);
    view_free(&v);
    return 0;
}

int orc_backward(const orc_scene *sc, const orc_camera *cam, const orc_settings *st,
                 const double *dL_dC, double *g_means, double *g_log_scales, double *g_quats,
                 double *g_logit, double *g_sh, double *S, double *S_po, double *S_ls, double *grad2d)
{
    return orc_backward_rows(sc, cam, st, 0, cam->height, dL_dC, g_means, g_log_scales, g_quats, g_logit, g_sh,
                             S, S_po, S_ls, grad2d);
}

/* ------------------------------------------------------------------------ */
/* The same render and backward on all host cores (a timing baseline; the    */
/* single-thread functions above are the pinned reference).  Rows are dealt  */
/* to threads one at a time, each thread runs render_view / backward_view on */
/* its rows exactly as above, into its own copy of the per-Gaussian sums,    */
/* and the copies are added at the end: the same terms, summed in another    */
/* order.  Without OpenMP these run on one thread.                           */
/* ------------------------------------------------------------------------ */

int orc_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

static void view_build_mt(const orc_scene *sc, const orc_camera *cam, const orc_settings *st, orc_view *v)
{
    v->n = sc->n;
    v->gx = (cam->width + st->tile_w - 1) / st->tile_w;
    v->gy = (cam->height + st->tile_h - 1) / st->tile_h;
    v->ntiles = v->gx * v->gy;
    v->pr = (orc_proj *)malloc(sizeof(orc_proj) * (size_t)(sc->n > 0 ? sc->n : 1));
#pragma omp parallel for schedule(static)
    for (int i = 0; i < sc->n; ++i) project_one(sc, cam, st, i, &v->pr[i]);
    v->M = orc_bin_sort(sc, cam, st, NULL, NULL, NULL, 0);
    uint64_t *keys = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(v->M > 0 ? v->M : 1));
    v->gids = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(v->M > 0 ? v->M : 1));
    v->ranges = (uint32_t *)malloc(sizeof(uint32_t) * 2 * (size_t)v->ntiles);
    orc_bin_sort(sc, cam, st, keys, v->gids, v->ranges, v->M);
    free(keys);
}

int orc_render_rows_mt(const orc_scene *sc, const orc_camera *cam, const orc_settings *st, int y0, int h,
                       double *image, double *final_T, int32_t *n_contrib, uint8_t *band)
{
    if (y0 < 0 || h < 0 || y0 + h > cam->height) return -1;
    orc_view v;
    view_build_mt(sc, cam, st, &v);
    const size_t W = (size_t)cam->width;
#pragma omp parallel for schedule(dynamic, 1)
    for (int r = 0; r < h; ++r)
        render_view(&v, cam, st, y0 + r, y0 + r + 1, image + 3 * W * r, final_T ? final_T + W * r : NULL,
                    n_contrib ? n_contrib + W * r : NULL, band ? band + W * r : NULL);
    view_free(&v);
    return 0;
}

int orc_backward_rows_mt(const orc_scene *sc, const orc_camera *cam, const orc_settings *st, int y0, int h,
                         const double *dL_dC, double *g_means, double *g_log_scales, double *g_quats,
                         double *g_logit, double *g_sh, double *S, double *S_po, double *S_ls, double *grad2d)
{
    if (y0 < 0 || h < 0 || y0 + h > cam->height) return -1;
    orc_view v;
    view_build_mt(sc, cam, st, &v);
    const size_t n = (size_t)(sc->n > 0 ? sc->n : 1), W = (size_t)cam->width;
    const int T = orc_threads();
    grad2d_t *g2 = (grad2d_t *)calloc(n * (size_t)T, sizeof(grad2d_t));
    double *St = S ? (double *)calloc(9 * n * (size_t)T, sizeof(double)) : NULL;
    double *Pt = S_po ? (double *)calloc(3 * n * (size_t)T, sizeof(double)) : NULL;
    double *Lt = S_ls ? (double *)calloc(18 * n * (size_t)T, sizeof(double)) : NULL;
#pragma omp parallel
    {
#ifdef _OPENMP
        const size_t t = (size_t)omp_get_thread_num();
#else
        const size_t t = 0;
#endif
#pragma omp for schedule(dynamic, 1)
        for (int r = 0; r < h; ++r)
            backward_view(sc, &v, cam, st, y0 + r, y0 + r + 1, dL_dC + 3 * W * r, g2 + n * t,
                          St ? St + 9 * n * t : NULL, Pt ? Pt + 3 * n * t : NULL, Lt ? Lt + 18 * n * t : NULL);
    }
#pragma omp parallel for schedule(static)
    for (int i = 0; i < sc->n; ++i) {
        grad2d_t sum;
        memset(&sum, 0, sizeof sum);
        for (int t = 0; t < T; ++t) {
            const grad2d_t *q = g2 + n * (size_t)t + i;
            sum.mu[0] += q->mu[0]; sum.mu[1] += q->mu[1];
            for (int k = 0; k < 3; ++k) { sum.Q[k] += q->Q[k]; sum.rgb[k] += q->rgb[k]; }
            sum.o += q->o;
            if (S) for (int k = 0; k < 9; ++k) S[9 * (size_t)i + k] += St[9 * (n * t + i) + k];
            if (S_po) for (int k = 0; k < 3; ++k) S_po[3 * (size_t)i + k] += Pt[3 * (n * t + i) + k];
            if (S_ls) for (int k = 0; k < 18; ++k) S_ls[18 * (size_t)i + k] += Lt[18 * (n * t + i) + k];
        }
        if (grad2d) {
            double *o = grad2d + 9 * (size_t)i;
            o[0] = sum.mu[0]; o[1] = sum.mu[1];
            o[2] = sum.Q[0]; o[3] = sum.Q[1]; o[4] = sum.Q[2];
            o[5] = sum.o; o[6] = sum.rgb[0]; o[7] = sum.rgb[1]; o[8] = sum.rgb[2];
        }
        if (!v.pr[i].is.culled)
            chain_to_params(sc, cam, &v.pr[i], &sum, i, g_means, g_log_scales, g_quats, g_logit, g_sh);
    }
    free(g2); free(St); free(Pt); free(Lt);
    view_free(&v);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Frozen-linearisation evaluation (Appendix "Deriving Hessian of Gaussian"): */
/* Pi is replaced by its affine approximation at the current p (mu(p') =     */
/* mu + P (p' - p)); P, Sigma2D, colour, opacity, tile lists and order stay   */
/* at their values at theta.  Gaussian `idx` is displaced by dp (its opacity */
/* by d_o, its log-scales by d_ls with P frozen), or, when mix_v is given,    */
/* replaced by the mixture slot 0.5 sigma(p + mix_v, l + d_ls, o + d_o) +     */
/* 0.5 sigma(p - mix_v, l - d_ls, o - d_o) (Theorem 1's                       */
/* w = 1/2 split with both offspring sharing the parent's depth slot).       */
/* Returns sum g . C (mode 0) or the L1 loss against `target` (mode 1).      */
/* ------------------------------------------------------------------------ */

double orc_frozen_eval(const orc_scene *sc, const orc_camera *cam, const orc_settings *st,
                       int mode, const double *g, const float *target, int idx,
                       const double *dp, const double *mix_v, double d_o, const double *d_ls)
{
    orc_view v;
    view_build(sc, cam, st, &v);
    int W = cam->width, H = cam->height;
    double acc = 0.0;
    for (int py = 0; py < H; ++py)
        for (int px = 0; px < W; ++px) {
            int tile = (py / st->tile_h) * v.gx + (px / st->tile_w);
            uint32_t s = v.ranges[2 * tile], e = v.ranges[2 * tile + 1];
            double T = 1.0, C[3] = {0, 0, 0};
            for (uint32_t k = s; k < e; ++k) {
                int gid = (int)v.gids[k];
                const orc_proj *pr = &v.pr[gid];
                double alpha;
                double dx, dy;
                if (gid == idx) {
                    double sh1[2] = {0, 0}, sh2[2] = {0, 0};
                    const double *d1 = mix_v ? mix_v : dp;
                    for (int a = 0; a < 2; ++a)
                        for (int j = 0; j < 3; ++j) sh1[a] += pr->P[3 * a + j] * (d1 ? d1[j] : 0.0);
                    double mu1[2] = {pr->mu[0] + sh1[0], pr->mu[1] + sh1[1]};
                    double Q1[3] = {pr->Q[0], pr->Q[1], pr->Q[2]}, Q2[3] = {pr->Q[0], pr->Q[1], pr->Q[2]};
                    if (d_ls) {
                        double m_ls[3] = {-d_ls[0], -d_ls[1], -d_ls[2]};
                        frozen_conic(pr, st, d_ls, Q1);
                        frozen_conic(pr, st, m_ls, Q2);
                    }
                    double a1 = (pr->o + d_o) * gauss2d(mu1, Q1, px, py, &dx, &dy);
                    if (mix_v) {
                        for (int a = 0; a < 2; ++a) sh2[a] = -sh1[a];
                        double mu2[2] = {pr->mu[0] + sh2[0], pr->mu[1] + sh2[1]};
                        double a2 = (pr->o - d_o) * gauss2d(mu2, Q2, px, py, &dx, &dy);
                        alpha = 0.5 * a1 + 0.5 * a2;
                    } else {
                        alpha = a1;
                    }
                } else {
                    alpha = pr->o * gauss2d(pr->mu, pr->Q, px, py, &dx, &dy);
                }
                if (alpha > st->alpha_max) alpha = st->alpha_max;
                if (alpha < st->alpha_min) continue;
                double Tn = T * (1.0 - alpha);
                if (Tn < st->T_min) break;
                for (int ch = 0; ch < 3; ++ch) C[ch] += pr->rgb[ch] * alpha * T;
                T = Tn;
            }
            size_t pix = (size_t)py * W + px;
            for (int ch = 0; ch < 3; ++ch) {
                double c = C[ch] + T * st->bg[ch];
                if (mode == 0) acc += g[3 * pix + ch] * c;
                else acc += fabs(c - (double)target[3 * pix + ch]);
            }
        }
    view_free(&v);
    if (mode == 1) acc /= 3.0 * (double)H * (double)W;
    return acc;
}

/* ------------------------------------------------------------------------ */
/* Minimum eigenpair of a symmetric 3x3 matrix (Appendix "Eigendecomposition") */
/* A = p B + q I, q = tr(A)/3, p = sqrt(tr((A - qI)^2)/6); det(beta I - B) =  */
/* beta^3 - 3 beta - det(B); beta = 2 cos(arccos(det(B)/2)/3 + 2 k pi/3).     */
/* phi = arccos(r)/3 lies in [0, pi/3]; the smallest root is k = 1.          */
/* Eigenvector: the largest cross product of two rows of A - lambda I        */
/* (those rows span the orthogonal complement of v).  Degenerate and sign    */
/* conventions are readings (the paper gives eigenvalues only):              */
/*   p = 0            -> lambda = q, v = e_x;                                 */
/*   all crosses < 1e-12 p^2 (repeated lambda_min) -> v = n x e_k, n the      */
/*   largest row of A - lambda I, e_k the axis of n's smallest |component|;  */
/*   sign: the component of largest magnitude is positive (lowest index on   */
/*   ties).                                                                  */
/* ------------------------------------------------------------------------ */

static void cross3(const double *a, const double *b, double *c)
{
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

static double norm3(const double *a) { return sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]); }

static void canon_sign(double *v)
{
    int k = 0;
    for (int j = 1; j < 3; ++j)
        if (fabs(v[j]) > fabs(v[k])) k = j;
    if (v[k] < 0) { v[0] = -v[0]; v[1] = -v[1]; v[2] = -v[2]; }
}

static void eig3_min_one(const double *A, double *lam_out, double *v_out)
{
    double q = (A[0] + A[4] + A[8]) / 3.0;
    double B0[9];
    for (int k = 0; k < 9; ++k) B0[k] = A[k];
    B0[0] -= q; B0[4] -= q; B0[8] -= q;
    double ss = 0.0;
    for (int k = 0; k < 9; ++k) ss += B0[k] * B0[k];
    double p = sqrt(ss / 6.0);
    if (p == 0.0) {
        *lam_out = q;
        v_out[0] = 1.0; v_out[1] = 0.0; v_out[2] = 0.0;
        return;
    }
    double B[9];
    for (int k = 0; k < 9; ++k) B[k] = B0[k] / p;
    double detB = B[0] * (B[4] * B[8] - B[5] * B[7]) - B[1] * (B[3] * B[8] - B[5] * B[6]) +
                  B[2] * (B[3] * B[7] - B[4] * B[6]);
    double r = detB / 2.0;
    if (r < -1.0) r = -1.0;
    if (r > 1.0) r = 1.0;
    double phi = acos(r) / 3.0;
    double lam = q + p * 2.0 * cos(phi + 2.0 * PI_D / 3.0);
    *lam_out = lam;
    double Am[9];
    for (int k = 0; k < 9; ++k) Am[k] = A[k];
    Am[0] -= lam; Am[4] -= lam; Am[8] -= lam;
    const double *r0 = Am, *r1 = Am + 3, *r2 = Am + 6;
    double c[3][3];
    cross3(r0, r1, c[0]);
    cross3(r0, r2, c[1]);
    cross3(r1, r2, c[2]);
    double n[3] = {norm3(c[0]), norm3(c[1]), norm3(c[2])};
    int best = 0;
    for (int k = 1; k < 3; ++k)
        if (n[k] > n[best]) best = k;
    if (n[best] >= 1e-12 * p * p) {
        for (int j = 0; j < 3; ++j) v_out[j] = c[best][j] / n[best];
    } else {
        double rn[3] = {norm3(r0), norm3(r1), norm3(r2)};
        int rb = 0;
        for (int k = 1; k < 3; ++k)
            if (rn[k] > rn[rb]) rb = k;
        const double *row = Am + 3 * rb;
        int ax = 0;
        for (int j = 1; j < 3; ++j)
            if (fabs(row[j]) < fabs(row[ax])) ax = j;
        double e[3] = {0, 0, 0};
        e[ax] = 1.0;
        double vv[3];
        cross3(row, e, vv);
        double nv = norm3(vv);
        for (int j = 0; j < 3; ++j) v_out[j] = vv[j] / nv;
    }
    canon_sign(v_out);
}

void orc_eig3_min(const double *S, double scale, int n, double *lam, double *v)
{
    for (int i = 0; i < n; ++i) {
        double A[9];
        for (int k = 0; k < 9; ++k) A[k] = S[9 * (size_t)i + k] * scale;
        eig3_min_one(A, lam + i, v + 3 * (size_t)i);
    }
}

/* Cyclic Jacobi rotations (textbook), all three eigenpairs, ascending. */
void orc_jacobi3(const double *S, int n, double *evals, double *evecs)
{
    for (int i = 0; i < n; ++i) {
        double a[3][3], V[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c) a[r][c] = S[9 * (size_t)i + 3 * r + c];
        for (int sweep = 0; sweep < 100; ++sweep) {
            double off = a[0][1] * a[0][1] + a[0][2] * a[0][2] + a[1][2] * a[1][2];
            double tot = off;
            for (int k = 0; k < 3; ++k) tot += a[k][k] * a[k][k];
            if (off <= 1e-40 * tot || off == 0.0) break;
            for (int pq = 0; pq < 3; ++pq) {
                int p = pq == 2 ? 1 : 0, q = pq == 0 ? 1 : 2;
                if (a[p][q] == 0.0) continue;
                double theta = (a[q][q] - a[p][p]) / (2.0 * a[p][q]);
                double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
                for (int k = 0; k < 3; ++k) {
                    double akp = a[k][p], akq = a[k][q];
                    a[k][p] = c * akp - s * akq;
                    a[k][q] = s * akp + c * akq;
                }
                for (int k = 0; k < 3; ++k) {
                    double apk = a[p][k], aqk = a[q][k];
                    a[p][k] = c * apk - s * aqk;
                    a[q][k] = s * apk + c * aqk;
                }
                for (int k = 0; k < 3; ++k) {
                    double vkp = V[k][p], vkq = V[k][q];
                    V[k][p] = c * vkp - s * vkq;
                    V[k][q] = s * vkp + c * vkq;
                }
            }
        }
        int idx[3] = {0, 1, 2};
        for (int x = 0; x < 3; ++x)
            for (int y = x + 1; y < 3; ++y)
                if (a[idx[y]][idx[y]] < a[idx[x]][idx[x]]) { int t = idx[x]; idx[x] = idx[y]; idx[y] = t; }
        for (int k = 0; k < 3; ++k) {
            evals[3 * (size_t)i + k] = a[idx[k]][idx[k]];
            double vv[3] = {V[0][idx[k]], V[1][idx[k]], V[2][idx[k]]};
            canon_sign(vv);
            for (int r = 0; r < 3; ++r) evecs[9 * (size_t)i + 3 * k + r] = vv[r];
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Split and compaction (Theorem 2, Algorithm 1).                             */
/* flag_i = lambda_min < eps_split (and, when grad_norm is given,             */
/* grad_norm <= eps_grad: the "compactest" gate of the Variants section).     */
/* excl = exclusive prefix sum of the flags.  Output row i holds Gaussian i,  */
/* moved to p + eps_i v with opacity o/2 when flagged; row N + excl[i] holds  */
/* its second offspring p - eps_i v with opacity o/2.  Scales, rotation and  */
/* colour are copied.  eps_i = step_scale * max_k exp(log_scale_ik) (the      */
/* paper leaves the step size open).  Opacity o/2 in logit space:            */
/* logit(o/2) = -log(1 + 2 exp(-x)).                                         */
/* ------------------------------------------------------------------------ */

/* Increment budget (the "Densification with Increment Budget" variant): when
 * more than `budget` Gaussians qualify, only the `budget` ones with the least
 * lambda_min are split (ties by index).
 *
 * flags_in, when not NULL, gives the split decisions instead of the rule
 * above (no gate, no budget): the exclusive scan and the offspring rows then
 * follow from those flags alone.  A decision taken in float32 can differ from
 * the float64 one only where lambda_min lies within rounding of eps_split;
 * handing the other side's flags to this scan keeps the compaction indices
 * and offspring comparable everywhere. */
static const double *g_sel_lam;
static int sel_cmp(const void *pa, const void *pb)
{
    int a = *(const int *)pa, b = *(const int *)pb;
    if (g_sel_lam[a] != g_sel_lam[b]) return g_sel_lam[a] < g_sel_lam[b] ? -1 : 1;
    return a < b ? -1 : (a > b);
}

int orc_split(const orc_scene *sc, const double *lam, const double *v, double eps_split,
              double step_scale, const double *grad_norm, double eps_grad, int64_t budget,
              double *out_means, double *out_log_scales, double *out_quats,
              double *out_logit, double *out_sh, int32_t *parent, uint8_t *flags,
              const uint8_t *flags_in)
{
    int n = sc->n;
    int K = (sc->sh_degree + 1) * (sc->sh_degree + 1);
    int32_t *excl = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    int32_t run = 0;
    int cand = 0;
    for (int i = 0; i < n; ++i) {
        int f;
        if (flags_in) {
            f = flags_in[i] != 0;
        } else {
            f = lam[i] < eps_split;
            if (grad_norm) f = f && (grad_norm[i] <= eps_grad);
        }
        flags[i] = (uint8_t)f;
        cand += f;
    }
    if (!flags_in && budget > 0 && cand > budget) {
        int *idx = (int *)malloc(sizeof(int) * (size_t)cand);
        int m = 0;
        for (int i = 0; i < n; ++i)
            if (flags[i]) idx[m++] = i;
        g_sel_lam = lam;
        qsort(idx, (size_t)cand, sizeof(int), sel_cmp);
        for (int k = (int)budget; k < cand; ++k) flags[idx[k]] = 0;
        free(idx);
    }
    for (int i = 0; i < n; ++i) {
        excl[i] = run;
        run += flags[i];
    }
    for (int i = 0; i < n; ++i) {
        double p[3], e = 0.0;
        for (int k = 0; k < 3; ++k) {
            p[k] = sc->means[3 * i + k];
            double s = exp((double)sc->log_scales[3 * i + k]);
            if (s > e) e = s;
        }
        e *= step_scale;
        double x = sc->opacity_logit[i];
        double half = x > 0 ? -log1p(2.0 * exp(-x)) : x - log(exp(x) + 2.0);
        int rows[2] = {i, flags[i] ? n + excl[i] : -1};
        for (int r = 0; r < 2; ++r) {
            int row = rows[r];
            if (row < 0) continue;
            double sgn = r == 0 ? 1.0 : -1.0;
            for (int k = 0; k < 3; ++k) {
                out_means[3 * (size_t)row + k] = flags[i] ? p[k] + sgn * e * v[3 * (size_t)i + k] : p[k];
                out_log_scales[3 * (size_t)row + k] = sc->log_scales[3 * i + k];
            }
            for (int k = 0; k < 4; ++k) out_quats[4 * (size_t)row + k] = sc->quats[4 * i + k];
            out_logit[row] = flags[i] ? half : x;
            for (int k = 0; k < 3 * K; ++k) out_sh[(size_t)row * 3 * K + k] = sc->sh[(size_t)i * 3 * K + k];
            parent[row] = i;
        }
    }
    free(excl);
    return n + run;
}
