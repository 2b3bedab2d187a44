// Steepest density control: minimum eigenpair of the averaged splitting
// matrices, split decision, offspring generation and prefix-sum compaction;
// plus the L1 photometric loss and its gradient.
//
// Paper: Theorem 2 (m = 2, w = 1/2, delta = +-v_min when lambda_min < 0),
// Algorithm 1 (S /= T_split; replace theta by (theta +- eps delta, o/2)),
// Appendix "Eigendecomposition" (A = p B + q I, beta = 2 cos(arccos(det B / 2)
// / 3 + 2 k pi / 3)), the "Compactest Splitting Strategy" variant (gradient
// gate), Section 3 Eq. loss (L1).
#include <algorithm>
#include <type_traits>

#include "common.cuh"

namespace sgs {

struct Eig {
    float lam;
    float v[3];
};

__device__ __forceinline__ void cross3(const float* a, const float* b, float* c) {
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

// Minimum eigenpair of the symmetric matrix (xx, xy, xz, yy, yz, zz).
// Trigonometric root formula; when the two smallest roots are the close pair
// (det(B)/2 > 0) the largest, well-separated eigenpair is deflated and the
// 2x2 block on its complement is solved in closed form; otherwise the
// eigenvector is the largest cross product of two rows of A - lambda I (with a
// repeated-root fallback).  Then one Rayleigh quotient v^T A v.
__device__ Eig eig3_min(const float* s6, float scale) {
    const float a00 = s6[0] * scale, a01 = s6[1] * scale, a02 = s6[2] * scale;
    const float a11 = s6[3] * scale, a12 = s6[4] * scale, a22 = s6[5] * scale;
    Eig e;
    const float q = (a00 + a11 + a22) * (1.0f / 3.0f);
    const float b00 = a00 - q, b11 = a11 - q, b22 = a22 - q;
    const float p2 = (b00 * b00 + b11 * b11 + b22 * b22 + 2.0f * (a01 * a01 + a02 * a02 + a12 * a12)) *
                     (1.0f / 6.0f);
    if (!(p2 > 0.0f)) {
        e.lam = q;
        e.v[0] = 1.0f; e.v[1] = 0.0f; e.v[2] = 0.0f;
        return e;
    }
    const float p = sqrtf(p2);
    const float ip = 1.0f / p;
    const float B00 = b00 * ip, B11 = b11 * ip, B22 = b22 * ip;
    const float B01 = a01 * ip, B02 = a02 * ip, B12 = a12 * ip;
    const float detB = B00 * (B11 * B22 - B12 * B12) - B01 * (B01 * B22 - B12 * B02) +
                       B02 * (B01 * B12 - B11 * B02);
    const float r = fminf(fmaxf(0.5f * detB, -1.0f), 1.0f);
    const float phi = acosf(r) * (1.0f / 3.0f);
    if (r > 0.0f) {
        // The two smallest roots are the close pair (r -> 1 makes them equal),
        // where arccos loses ~sqrt(eps) p and their eigenvectors mix.  Deflate
        // the well-separated largest eigenpair and take the smaller eigenvalue
        // of the 2x2 block on its orthogonal complement in closed form.
        const float lmax = q + 2.0f * p * cosf(phi);
        const float m0[3] = {a00 - lmax, a01, a02};
        const float m1[3] = {a01, a11 - lmax, a12};
        const float m2[3] = {a02, a12, a22 - lmax};
        float cc[3][3];
        cross3(m0, m1, cc[0]);
        cross3(m0, m2, cc[1]);
        cross3(m1, m2, cc[2]);
        float nb = 0.0f, b0 = 0.0f, b1 = 0.0f, b2 = 0.0f;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const float nk = cc[k][0] * cc[k][0] + cc[k][1] * cc[k][1] + cc[k][2] * cc[k][2];
            const bool take = nk > nb;
            nb = take ? nk : nb;
            b0 = take ? cc[k][0] : b0;
            b1 = take ? cc[k][1] : b1;
            b2 = take ? cc[k][2] : b2;
        }
        if (nb > 0.0f) {
            const float in = rsqrtf(nb);
            const float u[3] = {b0 * in, b1 * in, b2 * in};   // v_max
            // orthonormal basis (e1, e2) of v_max's complement
            const float au0 = fabsf(u[0]), au1 = fabsf(u[1]), au2 = fabsf(u[2]);
            float ax[3] = {0.0f, 0.0f, 0.0f};
            if (au0 <= au1 && au0 <= au2) ax[0] = 1.0f;
            else if (au1 <= au2) ax[1] = 1.0f;
            else ax[2] = 1.0f;
            float e1[3], e2[3];
            cross3(u, ax, e1);
            const float i1 = rsqrtf(e1[0] * e1[0] + e1[1] * e1[1] + e1[2] * e1[2]);
            e1[0] *= i1; e1[1] *= i1; e1[2] *= i1;
            cross3(u, e1, e2);
            const float A1[3] = {a00 * e1[0] + a01 * e1[1] + a02 * e1[2], a01 * e1[0] + a11 * e1[1] + a12 * e1[2],
                                 a02 * e1[0] + a12 * e1[1] + a22 * e1[2]};
            const float A2[3] = {a00 * e2[0] + a01 * e2[1] + a02 * e2[2], a01 * e2[0] + a11 * e2[1] + a12 * e2[2],
                                 a02 * e2[0] + a12 * e2[1] + a22 * e2[2]};
            const float m00 = e1[0] * A1[0] + e1[1] * A1[1] + e1[2] * A1[2];
            const float m01 = e1[0] * A2[0] + e1[1] * A2[1] + e1[2] * A2[2];
            const float m11 = e2[0] * A2[0] + e2[1] * A2[1] + e2[2] * A2[2];
            const float h = 0.5f * (m00 - m11);
            const float sq = sqrtf(h * h + m01 * m01);
            // eigenvector of [[m00, m01], [m01, m11]] for m_mean - sq, from the
            // better-conditioned row
            const float w0 = h >= 0.0f ? m01 : sq - h;
            const float w1 = h >= 0.0f ? -(h + sq) : -m01;
            float v[3] = {w0 * e1[0] + w1 * e2[0], w0 * e1[1] + w1 * e2[1], w0 * e1[2] + w1 * e2[2]};
            const float nv = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
            if (nv > 0.0f) {
                const float iv = rsqrtf(nv);
                v[0] *= iv; v[1] *= iv; v[2] *= iv;
            } else {
                v[0] = e1[0]; v[1] = e1[1]; v[2] = e1[2];
            }
            float big = v[0];
            if (fabsf(v[1]) > fabsf(big)) big = v[1];
            if (fabsf(v[2]) > fabsf(big)) big = v[2];
            if (big < 0.0f) { v[0] = -v[0]; v[1] = -v[1]; v[2] = -v[2]; }
            const float Av0 = a00 * v[0] + a01 * v[1] + a02 * v[2];
            const float Av1 = a01 * v[0] + a11 * v[1] + a12 * v[2];
            const float Av2 = a02 * v[0] + a12 * v[1] + a22 * v[2];
            e.lam = v[0] * Av0 + v[1] * Av1 + v[2] * Av2;
            e.v[0] = v[0]; e.v[1] = v[1]; e.v[2] = v[2];
            return e;
        }
    }
    const float lam0 = q + 2.0f * p * cosf(phi + 2.0943951023931953f);
    const float r0[3] = {a00 - lam0, a01, a02};
    const float r1[3] = {a01, a11 - lam0, a12};
    const float r2[3] = {a02, a12, a22 - lam0};
    float c[3][3];
    cross3(r0, r1, c[0]);
    cross3(r0, r2, c[1]);
    cross3(r1, r2, c[2]);
    float n2[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) n2[k] = c[k][0] * c[k][0] + c[k][1] * c[k][1] + c[k][2] * c[k][2];
    float bn = n2[0], bc0 = c[0][0], bc1 = c[0][1], bc2 = c[0][2];
    if (n2[1] > bn) { bn = n2[1]; bc0 = c[1][0]; bc1 = c[1][1]; bc2 = c[1][2]; }
    if (n2[2] > bn) { bn = n2[2]; bc0 = c[2][0]; bc1 = c[2][1]; bc2 = c[2][2]; }
    float v[3];
    if (bn > 0.0f) {
        const float in = rsqrtf(bn);
        v[0] = bc0 * in; v[1] = bc1 * in; v[2] = bc2 * in;
    } else {
        // repeated minimum root: any unit vector orthogonal to the largest row
        const float rn0 = r0[0] * r0[0] + r0[1] * r0[1] + r0[2] * r0[2];
        const float rn1 = r1[0] * r1[0] + r1[1] * r1[1] + r1[2] * r1[2];
        const float rn2 = r2[0] * r2[0] + r2[1] * r2[1] + r2[2] * r2[2];
        float row[3] = {r0[0], r0[1], r0[2]};
        float rb = rn0;
        if (rn1 > rb) { row[0] = r1[0]; row[1] = r1[1]; row[2] = r1[2]; rb = rn1; }
        if (rn2 > rb) { row[0] = r2[0]; row[1] = r2[1]; row[2] = r2[2]; rb = rn2; }
        const float a0 = fabsf(row[0]), a1 = fabsf(row[1]), a2 = fabsf(row[2]);
        float ev[3];
        ev[0] = (a0 <= a1 && a0 <= a2) ? 1.0f : 0.0f;
        ev[1] = (ev[0] == 0.0f && a1 <= a2) ? 1.0f : 0.0f;
        ev[2] = (ev[0] == 0.0f && ev[1] == 0.0f) ? 1.0f : 0.0f;
        cross3(row, ev, v);
        const float in = rsqrtf(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
        v[0] *= in; v[1] *= in; v[2] *= in;
    }
    // canonical sign: largest-magnitude component positive (lowest index on ties)
    float big = v[0];
    if (fabsf(v[1]) > fabsf(big)) big = v[1];
    if (fabsf(v[2]) > fabsf(big)) big = v[2];
    if (big < 0.0f) { v[0] = -v[0]; v[1] = -v[1]; v[2] = -v[2]; }
    const float Av0 = a00 * v[0] + a01 * v[1] + a02 * v[2];
    const float Av1 = a01 * v[0] + a11 * v[1] + a12 * v[2];
    const float Av2 = a02 * v[0] + a12 * v[1] + a22 * v[2];
    e.lam = v[0] * Av0 + v[1] * Av1 + v[2] * Av2;
    e.v[0] = v[0]; e.v[1] = v[1]; e.v[2] = v[2];
    return e;
}

// Minimum eigenpair of a small symmetric matrix (the splitting matrix over
// theta = (p, o), N = 4, or theta = (p, l, o), N = 7) by cyclic Jacobi
// rotations (Jacobi's method; Golub & Van Loan, Matrix Computations, Sec.
// 8.5) in the parallel round-robin order (each round rotates disjoint pairs,
// whose angles are independent: instruction-level parallelism for one thread).
// Only the upper triangle is held (constant indices after unrolling, so it
// stays in registers); each rotation zeroes one off-diagonal pair exactly.
// Sweeps run until the off-diagonal mass is below float32 resolution of
// ||A||_F (at most 12), the eigenvector is the column of the accumulated
// rotations at the smallest diagonal entry, lambda the Rayleigh quotient of
// the input matrix, sign canonical (largest magnitude component positive,
// lowest index on ties).  entry(r, c) returns the scaled input entry, r <= c.
template <int N>
struct EigN {
    float lam;
    float v[N];
};

__host__ __device__ constexpr int upper_index(int r, int c, int n) {
    return r <= c ? r * n - r * (r - 1) / 2 + (c - r) : c * n - c * (c - 1) / 2 + (r - c);
}

// Round-robin (circle method) pairing of M indices, M even: in round r
// (0 <= r < M - 1) index 0 meets 1 + r and, for k = 1 .. M/2 - 1, index
// 1 + (r + k) mod (M - 1) meets 1 + (r + M - 1 - k) mod (M - 1).  The pairs of
// a round are disjoint and the M - 1 rounds cover every pair once.
__host__ __device__ constexpr int rr_a(int r, int k, int M) { return k == 0 ? 0 : 1 + (r + k) % (M - 1); }
__host__ __device__ constexpr int rr_b(int r, int k, int M) { return k == 0 ? 1 + r : 1 + (r + M - 1 - k) % (M - 1); }
__host__ __device__ constexpr int rr_low(int r, int k, int M) {
    return rr_a(r, k, M) < rr_b(r, k, M) ? rr_a(r, k, M) : rr_b(r, k, M);
}
__host__ __device__ constexpr int rr_high(int r, int k, int M) {
    return rr_a(r, k, M) < rr_b(r, k, M) ? rr_b(r, k, M) : rr_a(r, k, M);
}

template <int N, class Entry>
__device__ __forceinline__ EigN<N> jacobi_min(Entry entry) {
    constexpr int NU = N * (N + 1) / 2;
    constexpr int M = N + (N & 1);
    float u[NU];
    float total = 0.0f;
#pragma unroll
    for (int r = 0; r < N; ++r)
#pragma unroll
        for (int c = r; c < N; ++c) {
            const float x = entry(r, c);
            u[upper_index(r, c, N)] = x;
            total += (r == c ? 1.0f : 2.0f) * x * x;
        }
    float V[N][N];
#pragma unroll
    for (int r = 0; r < N; ++r)
#pragma unroll
        for (int c = 0; c < N; ++c) V[r][c] = r == c ? 1.0f : 0.0f;
#pragma unroll 1
    for (int sweep = 0; sweep < 12; ++sweep) {
        float off = 0.0f;
#pragma unroll
        for (int p = 0; p < N - 1; ++p)
#pragma unroll
            for (int q = p + 1; q < N; ++q) off += u[upper_index(p, q, N)] * u[upper_index(p, q, N)];
        if (!(2.0f * off > 1e-14f * total)) break;
        // one sweep = M - 1 rounds of M / 2 disjoint pairs (round-robin order
        // over M = N rounded up to even; pairs with the padding index skipped)
#pragma unroll
        for (int r = 0; r < M - 1; ++r) {
            float c[M / 2], s[M / 2], t[M / 2], a[M / 2];
#pragma unroll
            for (int k = 0; k < M / 2; ++k) {           // the round's angles, independent of each other
                const int p = rr_low(r, k, M), q = rr_high(r, k, M);
                if (q >= N) continue;
                const float apq = u[upper_index(p, q, N)];
                // t = tan(phi), the smaller root of t^2 + 2 theta t - 1 = 0
                const float theta = (u[upper_index(q, q, N)] - u[upper_index(p, p, N)]) / (2.0f * apq);
                const float tk = copysignf(1.0f, theta) / (fabsf(theta) + sqrtf(theta * theta + 1.0f));
                t[k] = apq == 0.0f ? 0.0f : tk;
                c[k] = rsqrtf(t[k] * t[k] + 1.0f);
                s[k] = t[k] * c[k];
                a[k] = apq;
            }
#pragma unroll
            for (int k = 0; k < M / 2; ++k) {           // disjoint rotations commute
                const int p = rr_low(r, k, M), q = rr_high(r, k, M);
                if (q >= N) continue;
#pragma unroll
                for (int m = 0; m < N; ++m) {
                    if (m == p || m == q) continue;
                    const float amp = u[upper_index(m, p, N)], amq = u[upper_index(m, q, N)];
                    u[upper_index(m, p, N)] = c[k] * amp - s[k] * amq;
                    u[upper_index(m, q, N)] = s[k] * amp + c[k] * amq;
                }
                u[upper_index(p, p, N)] -= t[k] * a[k];
                u[upper_index(q, q, N)] += t[k] * a[k];
                u[upper_index(p, q, N)] = 0.0f;
#pragma unroll
                for (int m = 0; m < N; ++m) {
                    const float vmp = V[m][p], vmq = V[m][q];
                    V[m][p] = c[k] * vmp - s[k] * vmq;
                    V[m][q] = s[k] * vmp + c[k] * vmq;
                }
            }
        }
    }
    // column of the smallest diagonal entry (first on ties), selected with
    // constant indices so that u and V stay in registers
    float dmin = u[0];
    float v[N];
#pragma unroll
    for (int r = 0; r < N; ++r) v[r] = V[r][0];
#pragma unroll
    for (int k = 1; k < N; ++k) {
        const float d = u[upper_index(k, k, N)];
        const bool take = d < dmin;
        dmin = take ? d : dmin;
#pragma unroll
        for (int r = 0; r < N; ++r) v[r] = take ? V[r][k] : v[r];
    }
    float nrm = 0.0f;
#pragma unroll
    for (int k = 0; k < N; ++k) nrm += v[k] * v[k];
    const float inv = rsqrtf(nrm);
    float big = 0.0f;
#pragma unroll
    for (int k = 0; k < N; ++k) {
        v[k] *= inv;
        big = fabsf(v[k]) > fabsf(big) ? v[k] : big;
    }
    const float sg = big < 0.0f ? -1.0f : 1.0f;
    EigN<N> e;
#pragma unroll
    for (int k = 0; k < N; ++k) e.v[k] = sg * v[k];
    float lam = 0.0f;
#pragma unroll
    for (int r = 0; r < N; ++r) {
        float Av = 0.0f;
#pragma unroll
        for (int c = 0; c < N; ++c) Av += entry(r < c ? r : c, r < c ? c : r) * e.v[c];
        lam += e.v[r] * Av;
    }
    e.lam = lam;
    return e;
}

// Entry (r <= c) of the splitting matrix over theta = (p, o) (N = 4) or
// theta = (p, l, o) (N = 7) from its stored blocks: s6 the p-p upper triangle
// (xx xy xz yy yz zz), spo the p-o column, sls the p-l block (row p, column
// l), the l-l upper triangle and the l-o column; o-o is zero.
template <int N>
__device__ __forceinline__ float theta_entry(const float* s6, const float* spo, const float* sls, int r, int c) {
    constexpr int O = N - 1;
    if (c < 3) return s6[upper_index(r, c, 3)];
    if (c == O) return r == O ? 0.0f : (r < 3 ? spo[r] : sls[15 + r - 3]);
    if (r < 3) return sls[3 * r + (c - 3)];
    return sls[9 + upper_index(r - 3, c - 3, 3)];
}

template <int N>
__device__ __forceinline__ void load_theta(const float* __restrict__ S, const float* __restrict__ S_po,
                                           const float* __restrict__ S_ls, int i, float* s6, float* spo, float* sls) {
#pragma unroll
    for (int k = 0; k < 6; ++k) s6[k] = S[(size_t)i * 6 + k];
    if constexpr (N > 3) {
#pragma unroll
        for (int k = 0; k < 3; ++k) spo[k] = S_po[(size_t)i * 3 + k];
    }
    if constexpr (N == 7) {
#pragma unroll
        for (int k = 0; k < 18; ++k) sls[k] = S_ls[(size_t)i * 18 + k];
    }
}

__device__ __forceinline__ bool write_flag(int i, float lam, float eps_split, const float* __restrict__ grad_norm,
                                           float eps_grad, uint32_t* __restrict__ flags) {
    bool f = lam < eps_split;
    if (grad_norm) f = f && (grad_norm[i] <= eps_grad);
    flags[i] = f ? 1u : 0u;
    return f;
}

// The splitting matrix of a Gaussian that no pixel reached is zero, and its
// minimum eigenpair is (0, e_0), what both solvers return for it.  This kernel
// writes those directly and appends the others to a work list (one atomic per
// block), so that the rotations run in full warps.
template <int N>
__global__ void __launch_bounds__(256) eig_triage_kernel(const float* __restrict__ S,
                                                               const float* __restrict__ S_po,
                                                               const float* __restrict__ S_ls, int n,
                                                               float eps_split, const float* __restrict__ grad_norm,
                                                               float eps_grad, float* __restrict__ lam_out,
                                                               float* __restrict__ v_out, uint32_t* __restrict__ flags,
                                                               uint32_t* __restrict__ work,
                                                               uint32_t* __restrict__ n_work) {
    pdl_wait_and_trigger();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    bool nz = false;
    if (i < n) {
        float s6[6], spo[3], sls[N == 7 ? 18 : 1];
        load_theta<N>(S, S_po, S_ls, i, s6, spo, sls);
#pragma unroll
        for (int k = 0; k < 6; ++k) nz |= s6[k] != 0.0f;
        if constexpr (N > 3) {
#pragma unroll
            for (int k = 0; k < 3; ++k) nz |= spo[k] != 0.0f;
        }
        if constexpr (N == 7) {
#pragma unroll
            for (int k = 0; k < 18; ++k) nz |= sls[k] != 0.0f;
        }
        if (!nz) {
            lam_out[i] = 0.0f;
#pragma unroll
            for (int k = 0; k < N; ++k) v_out[N * (size_t)i + k] = k == 0 ? 1.0f : 0.0f;
            write_flag(i, 0.0f, eps_split, grad_norm, eps_grad, flags);
        }
    }
    // one atomic per block: warp counts, their prefix, then the block's base
    __shared__ uint32_t s_cnt[8];
    __shared__ uint32_t s_base;
    const int warp = threadIdx.x >> 5;
    const unsigned m = __ballot_sync(0xffffffffu, nz);
    if (lane == 0) s_cnt[warp] = (uint32_t)__popc(m);
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t t = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            const uint32_t c = s_cnt[w];
            s_cnt[w] = t;
            t += c;
        }
        s_base = t ? atomicAdd(n_work, t) : 0u;
    }
    __syncthreads();
    if (nz) work[s_base + s_cnt[warp] + __popc(m & ((1u << lane) - 1u))] = (uint32_t)i;
}

// Minimum eigenpair and flag of every matrix over the position (root
// formula).  A zero matrix (a Gaussian no pixel reached) gets (0, e_0), what
// the formula returns for it; the block's non-zero matrices are first packed
// into its leading threads through shared memory, so that the solve runs in
// full warps.  bcount[block] = the block's number of flags (the sums the
// compaction's scan starts from).
__global__ void __launch_bounds__(256) eig_direct_kernel(const float* __restrict__ S, int n, float inv_T,
                                                         float eps_split, const float* __restrict__ grad_norm,
                                                         float eps_grad, float* __restrict__ lam_out,
                                                         float* __restrict__ v_out, uint32_t* __restrict__ flags,
                                                         uint32_t* __restrict__ bcount) {
    pdl_wait_and_trigger();
    __shared__ float s_m[256][7];                     // packed matrices (6 floats, padded)
    __shared__ int s_idx[256];
    __shared__ uint32_t s_wcnt[8];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float s6[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    bool nz = false, f0 = false, f1 = false;
    if (i < n) {
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            s6[k] = S[(size_t)i * 6 + k];
            nz |= s6[k] != 0.0f;
        }
        if (!nz) {
            lam_out[i] = 0.0f;
            v_out[3 * (size_t)i] = 1.0f;
            v_out[3 * (size_t)i + 1] = 0.0f;
            v_out[3 * (size_t)i + 2] = 0.0f;
            f0 = write_flag(i, 0.0f, eps_split, grad_norm, eps_grad, flags);
        }
    }
    const unsigned m = __ballot_sync(0xffffffffu, nz);
    if (lane == 0) s_wcnt[warp] = (uint32_t)__popc(m);
    __syncthreads();
    uint32_t before = 0, count = 0;
#pragma unroll
    for (int w = 0; w < 8; ++w) {
        const uint32_t c = s_wcnt[w];
        before += w < warp ? c : 0u;
        count += c;
    }
    if (nz) {
        const uint32_t slot = before + (uint32_t)__popc(m & ((1u << lane) - 1u));
#pragma unroll
        for (int k = 0; k < 6; ++k) s_m[slot][k] = s6[k];
        s_idx[slot] = i;
    }
    __syncthreads();
    if (threadIdx.x < count) {
        float a6[6];
#pragma unroll
        for (int k = 0; k < 6; ++k) a6[k] = s_m[threadIdx.x][k];
        const int j = s_idx[threadIdx.x];
        const Eig e = eig3_min(a6, inv_T);
        lam_out[j] = e.lam;
#pragma unroll
        for (int k = 0; k < 3; ++k) v_out[3 * (size_t)j + k] = e.v[k];
        f1 = write_flag(j, e.lam, eps_split, grad_norm, eps_grad, flags);
    }
    const int c = __syncthreads_count(f0) + __syncthreads_count(f1);
    if (bcount && threadIdx.x == 0) bcount[blockIdx.x] = (uint32_t)c;
}

// Minimum eigenpair and flag of the listed (non-zero) matrices.
template <int N>
__global__ void __launch_bounds__(256) eig_solve_kernel(const float* __restrict__ S,
                                                              const float* __restrict__ S_po,
                                                              const float* __restrict__ S_ls, float inv_T,
                                                              float eps_split, const float* __restrict__ grad_norm,
                                                              float eps_grad, float* __restrict__ lam_out,
                                                              float* __restrict__ v_out, uint32_t* __restrict__ flags,
                                                              const uint32_t* __restrict__ work,
                                                              const uint32_t* __restrict__ n_work) {
    pdl_wait_and_trigger();
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= *n_work) return;
    const int i = (int)work[t];
    float s6[6], spo[3], sls[N == 7 ? 18 : 1];
    load_theta<N>(S, S_po, S_ls, i, s6, spo, sls);
    const EigN<N> e = jacobi_min<N>([&](int r, int c) { return theta_entry<N>(s6, spo, sls, r, c) * inv_T; });
    lam_out[i] = e.lam;
#pragma unroll
    for (int k = 0; k < N; ++k) v_out[N * (size_t)i + k] = e.v[k];
    write_flag(i, e.lam, eps_split, grad_norm, eps_grad, flags);
}

// ---------------------------------------------------------------------------
// Increment budget (the "Densification with Increment Budget" variant): when
// more than K Gaussians are flagged, keep the K with the least lambda_min,
// ties by index.  A 4-pass radix select (8-bit digits, most significant
// first) over order-preserving keys of lambda finds the K-th smallest key on
// the device; ties at that key are admitted in index order through a scan.
// ---------------------------------------------------------------------------
struct SelectState {
    uint32_t active;    // 1 when the budget binds
    uint32_t prefix;    // key digits fixed so far
    uint32_t k_rem;     // rank still sought among keys matching the prefix
    uint32_t pad;
    uint32_t hist[256];
};

__device__ __forceinline__ uint32_t order_key(float x) {
    const uint32_t u = __float_as_uint(x);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

__global__ void select_init_kernel(const uint32_t* __restrict__ total, int64_t K, SelectState* st) {
    pdl_wait_and_trigger();
    if (threadIdx.x == 0) {
        st->active = (int64_t)(*total) > K ? 1u : 0u;
        st->prefix = 0u;
        st->k_rem = (uint32_t)K;
    }
    for (int b = threadIdx.x; b < 256; b += blockDim.x) st->hist[b] = 0u;
}

__global__ void __launch_bounds__(256) select_hist_kernel(const float* __restrict__ lam,
                                                          const uint32_t* __restrict__ flags, int n, int shift,
                                                          SelectState* st) {
    pdl_wait_and_trigger();
    __shared__ uint32_t h[256];
    if (!st->active) return;
    h[threadIdx.x] = 0u;
    __syncthreads();
    const uint32_t hi_mask = shift + 8 >= 32 ? 0u : ~((1u << (shift + 8)) - 1u);
    const uint32_t prefix = st->prefix;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        if (!flags[i]) continue;
        const uint32_t k = order_key(lam[i]);
        if ((k & hi_mask) == (prefix & hi_mask)) atomicAdd(&h[(k >> shift) & 255u], 1u);
    }
    __syncthreads();
    if (h[threadIdx.x]) atomicAdd(&st->hist[threadIdx.x], h[threadIdx.x]);
}

__global__ void select_pick_kernel(int shift, SelectState* st) {
    pdl_wait_and_trigger();
    if (!st->active || threadIdx.x != 0) return;
    uint32_t before = 0u;
    int b = 0;
    for (; b < 255; ++b) {
        if (before + st->hist[b] >= st->k_rem) break;
        before += st->hist[b];
    }
    st->prefix |= (uint32_t)b << shift;
    st->k_rem -= before;
    for (int k = 0; k < 256; ++k) st->hist[k] = 0u;
}

__global__ void select_ties_kernel(const float* __restrict__ lam, const uint32_t* __restrict__ flags, int n,
                                   const SelectState* st, uint32_t* __restrict__ tie) {
    pdl_wait_and_trigger();
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    tie[i] = (st->active && flags[i] && order_key(lam[i]) == st->prefix) ? 1u : 0u;
}

__global__ void select_apply_kernel(const float* __restrict__ lam, uint32_t* __restrict__ flags, int n,
                                    const SelectState* st, const uint32_t* __restrict__ tie_rank) {
    pdl_wait_and_trigger();
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || !st->active || !flags[i]) return;
    const uint32_t k = order_key(lam[i]);
    flags[i] = (k < st->prefix || (k == st->prefix && tie_rank[i] < st->k_rem)) ? 1u : 0u;
}

// logit(sigmoid(x) / 2) = -log(1 + 2 exp(-x)), evaluated without overflow.
__device__ __forceinline__ float half_opacity_logit(float x) {
    return x > 0.0f ? -log1pf(2.0f * expf(-x)) : x - logf(expf(x) + 2.0f);
}

// Per-Gaussian fields of the output rows: mean, scales, rotation, opacity,
// parent index.  Row i holds Gaussian i (moved to p + eps v when flagged);
// row N + excl[i] holds the second offspring p - eps v.  DIM = 3: both
// offspring take o/2.  DIM = 4 (theta = (p, o)) and 7 (theta = (p, l, o)): v
// ends with an opacity component and the offspring take (o +- eps v_o) / 2,
// clamped to [1e-4, 1 - 1e-4]; DIM = 7 also moves the log-scales by
// +- eps v_l.
template <int DIM>
__device__ __forceinline__ void split_fields(
    int i, const float* __restrict__ means, const float* __restrict__ log_scales, const float* __restrict__ quats,
    const float* __restrict__ logit, int n, const float* __restrict__ v, const uint32_t* __restrict__ flags,
    const uint32_t* __restrict__ excl, float step_scale, int64_t cap, float* __restrict__ o_means,
    float* __restrict__ o_ls, float* __restrict__ o_quats, float* __restrict__ o_logit,
    int32_t* __restrict__ parent) {
    if (i >= n) return;
    const bool f = flags[i] != 0u;
    const float l0 = log_scales[3 * i], l1 = log_scales[3 * i + 1], l2 = log_scales[3 * i + 2];
    const float x = logit[i];
    const float p0 = means[3 * i], p1 = means[3 * i + 1], p2 = means[3 * i + 2];
    const float4 q = reinterpret_cast<const float4*>(quats)[i];
    float eps = 0.0f, lg = x;
    if (f) {
        eps = step_scale * expf(fmaxf(l0, fmaxf(l1, l2)));
        lg = half_opacity_logit(x);
    }
    const float v0 = f ? v[DIM * i] : 0.0f, v1 = f ? v[DIM * i + 1] : 0.0f, v2 = f ? v[DIM * i + 2] : 0.0f;
    const float vo = (DIM > 3 && f) ? v[DIM * i + DIM - 1] : 0.0f;
    const float w0 = (DIM == 7 && f) ? v[DIM * i + 3] : 0.0f, w1 = (DIM == 7 && f) ? v[DIM * i + 4] : 0.0f;
    const float w2 = (DIM == 7 && f) ? v[DIM * i + 5] : 0.0f;
    const float o = 1.0f / (1.0f + expf(-x));
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        const int64_t row = r == 0 ? (int64_t)i : (f ? (int64_t)n + (int64_t)excl[i] : -1);
        if (row < 0 || row >= cap) continue;
        const float sg = r == 0 ? eps : -eps;
        o_means[3 * row] = p0 + sg * v0;
        o_means[3 * row + 1] = p1 + sg * v1;
        o_means[3 * row + 2] = p2 + sg * v2;
        o_ls[3 * row] = l0 + sg * w0;
        o_ls[3 * row + 1] = l1 + sg * w1;
        o_ls[3 * row + 2] = l2 + sg * w2;
        reinterpret_cast<float4*>(o_quats)[row] = q;
        if (DIM > 3 && f) {
            const float oj = fminf(fmaxf(0.5f * (o + sg * vo), 1e-4f), 1.0f - 1e-4f);
            o_logit[row] = logf(oj) - log1pf(-oj);
        } else {
            o_logit[row] = lg;
        }
        if (parent) parent[row] = i;
    }
}

// SH rows of the output, one thread per vector unit of a row (U units of
// VEC floats): reads and the writes of row i are coalesced, and the second
// offspring of consecutive flagged Gaussians land in consecutive rows.
template <int VEC>
__device__ __forceinline__ void split_sh(int64_t first, int64_t stride, const float* __restrict__ sh, int n, int U,
                                         const uint32_t* __restrict__ flags, const uint32_t* __restrict__ excl,
                                         int64_t cap, float* __restrict__ o_sh) {
    using V = typename std::conditional<VEC == 4, float4, float>::type;
    const int64_t total = (int64_t)n * U;
    for (int64_t t = first; t < total; t += stride) {
        const int64_t i = t / U;
        const int u = (int)(t - i * U);
        const V val = reinterpret_cast<const V*>(sh)[t];
        reinterpret_cast<V*>(o_sh)[t] = val;
        if (flags[i]) {
            const int64_t row = (int64_t)n + (int64_t)excl[i];
            if (row < cap) reinterpret_cast<V*>(o_sh)[row * U + u] = val;
        }
    }
}

// The split in one launch: blocks [0, nbf) write the per-Gaussian fields (one
// thread per Gaussian; the first also writes n_out = n + number flagged), the
// other blocks copy the SH rows (grid-stride over the vector units), so the
// two streams of rows run side by side.
template <int DIM, int VEC>
__global__ void __launch_bounds__(256) split_kernel(
    const float* __restrict__ means, const float* __restrict__ log_scales, const float* __restrict__ quats,
    const float* __restrict__ logit, const float* __restrict__ sh, int n, int U, int nbf,
    const float* __restrict__ v, const uint32_t* __restrict__ flags, const uint32_t* __restrict__ excl,
    const uint32_t* __restrict__ total, float step_scale, int64_t cap, float* __restrict__ o_means,
    float* __restrict__ o_ls, float* __restrict__ o_quats, float* __restrict__ o_logit, float* __restrict__ o_sh,
    int32_t* __restrict__ parent, int32_t* __restrict__ d_n_out) {
    pdl_wait_and_trigger();
    if ((int)blockIdx.x < nbf) {
        if (blockIdx.x == 0 && threadIdx.x == 0) *d_n_out = n + (int32_t)(*total);
        split_fields<DIM>((int)blockIdx.x * 256 + (int)threadIdx.x, means, log_scales, quats, logit, n, v, flags,
                          excl, step_scale, cap, o_means, o_ls, o_quats, o_logit, parent);
    } else {
        split_sh<VEC>((int64_t)(blockIdx.x - nbf) * 256 + threadIdx.x, (int64_t)(gridDim.x - nbf) * 256, sh, n, U,
                      flags, excl, cap, o_sh);
    }
}

size_t densify_ws_bytes(int n) {
    Carver c{nullptr, 0};
    size_t nn = (size_t)(n > 0 ? n : 1);
    c.take<uint32_t>(nn);       // flags
    c.take<uint32_t>(nn);       // excl
    c.take<uint32_t>(1);        // total
    c.take<float>(nn);          // lam (when the caller passes none)
    c.take<float>(7 * nn);      // v (up to 7 components, theta = (p, l, o))
    c.take<char>(scan_tmp_bytes(n));
    c.take<uint32_t>(nn);       // ties at the budget threshold
    c.take<SelectState>(1);
    return c.off + 256;
}

cudaError_t launch_densify(const sgs_gaussians& in, const float* S, const float* S_po, const float* S_ls,
                           float inv_T, float eps_split,
                           float step_scale, const float* grad_norm, float eps_grad, int64_t max_splits,
                           const sgs_gaussians_mut& out, int64_t capacity, int32_t* d_n_out, int32_t* parent,
                           float* lam_out, float* v_out, void* ws, cudaStream_t stream) {
    const int n = in.n;
    Carver c{reinterpret_cast<char*>(ws), 0};
    size_t nn = (size_t)(n > 0 ? n : 1);
    uint32_t* flags = c.take<uint32_t>(nn);
    uint32_t* excl = c.take<uint32_t>(nn);
    uint32_t* total = c.take<uint32_t>(1);
    float* lam_ws = c.take<float>(nn);
    float* v_ws = c.take<float>(7 * nn);
    void* scan_tmp = c.take<char>(scan_tmp_bytes(n));
    uint32_t* tie = c.take<uint32_t>(nn);
    SelectState* sel = c.take<SelectState>(1);
    float* lam = lam_out ? lam_out : lam_ws;
    float* v = v_out ? v_out : v_ws;
    if (n == 0) return cudaMemsetAsync(d_n_out, 0, sizeof(int32_t), stream);
    const int nb = (n + 255) / 256;
    {
        // rotations: triage (zero matrices answered directly) then the solve
        // over the work list; excl and total serve as the list and its counter
        // until the scan
        if (S_po) {
            cudaError_t z = cudaMemsetAsync(total, 0, sizeof(uint32_t), stream);
            if (z != cudaSuccess) return z;
        }
        auto run = [&](auto dim) {
            constexpr int N = decltype(dim)::value;
            (void)launch_pdl(eig_triage_kernel<N>, dim3(nb), dim3(256), 0, stream, S, S_po, S_ls, n, eps_split,
                             grad_norm, eps_grad, lam, v, flags, excl, total);
            (void)launch_pdl(eig_solve_kernel<N>, dim3(nb), dim3(256), 0, stream, S, S_po, S_ls, inv_T, eps_split,
                             grad_norm, eps_grad, lam, v, flags, excl, total);
        };
        if (S_po && S_ls) {
            run(std::integral_constant<int, 7>{});
            note_launch(2);
        } else if (S_po) {
            run(std::integral_constant<int, 4>{});
            note_launch(2);
        } else {                                     // the root formula: short enough to run unsorted
            // its per-block flag counts go to `tie` (free until the budget's
            // tie ranks) and spare the scan its reduction pass
            (void)launch_pdl(eig_direct_kernel, dim3(nb), dim3(256), 0, stream, S, n, inv_T, eps_split, grad_norm,
                             eps_grad, lam, v, flags, tie);
            note_launch();
        }
    }
    cudaError_t e = S_po ? launch_exclusive_scan(flags, excl, total, n, nullptr, scan_tmp, stream)
                         : launch_exclusive_scan_counted(flags, excl, total, n, tie, scan_tmp, stream);
    if (e != cudaSuccess) return e;
    if (max_splits > 0) {
        (void)launch_pdl(select_init_kernel, dim3(1), dim3(256), 0, stream, total, max_splits, sel);
        note_launch();
        const int hb = nb < 152 * 4 ? nb : 152 * 4;
        for (int shift = 24; shift >= 0; shift -= 8) {
            (void)launch_pdl(select_hist_kernel, dim3(hb), dim3(256), 0, stream, lam, flags, n, shift, sel);
            note_launch();
            (void)launch_pdl(select_pick_kernel, dim3(1), dim3(32), 0, stream, shift, sel);
            note_launch();
        }
        (void)launch_pdl(select_ties_kernel, dim3(nb), dim3(256), 0, stream, lam, flags, n, sel, tie);
        note_launch();
        e = launch_exclusive_scan(tie, excl, nullptr, n, nullptr, scan_tmp, stream);
        if (e != cudaSuccess) return e;
        (void)launch_pdl(select_apply_kernel, dim3(nb), dim3(256), 0, stream, lam, flags, n, sel, excl);
        note_launch();
        e = launch_exclusive_scan(flags, excl, total, n, nullptr, scan_tmp, stream);
        if (e != cudaSuccess) return e;
    }
    const int K3 = (in.sh_degree + 1) * (in.sh_degree + 1) * 3;
    const bool vec4 = K3 % 4 == 0 && (reinterpret_cast<uintptr_t>(in.sh) % 16) == 0 &&
                      (reinterpret_cast<uintptr_t>(out.sh) % 16) == 0;
    const int U = vec4 ? K3 / 4 : K3;
    const int64_t units = (int64_t)n * U;
    const int sb = (int)std::min<int64_t>((units + 255) / 256, 152 * 16);
    auto pick = [&](auto vec) {
        constexpr int VEC = decltype(vec)::value;
        return S_po ? (S_ls ? split_kernel<7, VEC> : split_kernel<4, VEC>) : split_kernel<3, VEC>;
    };
    auto kern = vec4 ? pick(std::integral_constant<int, 4>{}) : pick(std::integral_constant<int, 1>{});
    (void)launch_pdl(kern, dim3(nb + sb), dim3(256), 0, stream, in.means, in.log_scales, in.quats,
                     in.opacity_logit, in.sh, n, U, nb, v, flags, excl, total, step_scale, capacity, out.means,
                     out.log_scales, out.quats, out.opacity_logit, out.sh, parent, d_n_out);
    note_launch();
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Adam update of one parameter array (the optimiser of the training loop
// around the splitting path), optionally accumulating the raw gradient into
// G (Algorithm 1's G <- G + grad).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) adam_kernel(float* __restrict__ p, const float* __restrict__ g,
                                                   float* __restrict__ m, float* __restrict__ v, int64_t count,
                                                   float lr, float b1, float b2, float eps, float bc1, float bc2,
                                                   float* __restrict__ G, const int32_t* __restrict__ d_step) {
    pdl_wait_and_trigger();
    if (d_step) {                                    // step count from device memory (graph replays)
        const float t = (float)*d_step;
        bc1 = 1.0f - powf(b1, t);
        bc2 = 1.0f - powf(b2, t);
    }
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < count;
         k += (int64_t)gridDim.x * blockDim.x) {
        const float gk = g[k];
        const float mk = b1 * m[k] + (1.0f - b1) * gk;
        const float vk = b2 * v[k] + (1.0f - b2) * gk * gk;
        m[k] = mk;
        v[k] = vk;
        p[k] -= lr * (mk / bc1) / (sqrtf(vk / bc2) + eps);
        if (G) G[k] += gk;
    }
}

cudaError_t launch_adam(float* p, const float* g, float* m, float* v, int64_t count, float lr, float b1, float b2,
                        float eps, int step, const int32_t* d_step, float* G, cudaStream_t stream) {
    if (count == 0) return cudaSuccess;
    const float bc1 = d_step ? 1.0f : 1.0f - powf(b1, (float)step);
    const float bc2 = d_step ? 1.0f : 1.0f - powf(b2, (float)step);
    int64_t blocks = (count + 255) / 256;
    if (blocks > 152 * 8) blocks = 152 * 8;
    (void)launch_pdl(adam_kernel, dim3((int)blocks), dim3(256), 0, stream, p, g, m, v, count, lr, b1, b2, eps, bc1,
                     bc2, G, d_step);
    note_launch();
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// L1 loss: loss += sum |C - Chat| / (3 H W V); dL/dC = sign(C - Chat) / (3 H W V)
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) l1_kernel(const float* __restrict__ image, const float* __restrict__ target,
                                                 int64_t count, float norm, float* __restrict__ dL,
                                                 float* __restrict__ loss) {
    pdl_wait_and_trigger();
    __shared__ float s_part[8];
    float acc = 0.0f;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < count;
         k += (int64_t)gridDim.x * blockDim.x) {
        const float r = image[k] - target[k];
        acc += fabsf(r);
        dL[k] = r > 0.0f ? norm : (r < 0.0f ? -norm : 0.0f);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) s_part[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        float s = 0.0f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += s_part[w];
        atomicAdd(loss, s * norm);
    }
}

// Several views concatenated at pixel offsets: per-view normalisation.
__global__ void __launch_bounds__(256) l1_views_kernel(const float* __restrict__ image,
                                                       const float* __restrict__ target, ViewsDev vd,
                                                       float* __restrict__ dL, float* __restrict__ loss) {
    pdl_wait_and_trigger();
    __shared__ float s_part[8];
    float acc = 0.0f;
    const long long count = 3 * vd.P_total;
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < count;
         k += (long long)gridDim.x * blockDim.x) {
        const int v = view_of_pixel(vd, k / 3);
        const float norm = 1.0f / (3.0f * (float)vd.cam[v].width * (float)vd.cam[v].height * (float)vd.nv);
        const float r = image[k] - target[k];
        acc += fabsf(r) * norm;
        dL[k] = r > 0.0f ? norm : (r < 0.0f ? -norm : 0.0f);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) s_part[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        float s = 0.0f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += s_part[w];
        atomicAdd(loss, s);
    }
}

cudaError_t launch_l1_views(const float* image, const float* target, const ViewsDev& vd, float* dL, float* loss,
                            cudaStream_t stream) {
    const long long count = 3 * vd.P_total;
    if (count == 0) return cudaSuccess;
    long long blocks = (count + 255) / 256;
    if (blocks > 152 * 8) blocks = 152 * 8;
    (void)launch_pdl(l1_views_kernel, dim3((int)blocks), dim3(256), 0, stream, image, target, vd, dL, loss);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_l1(const float* image, const float* target, int H, int W, int n_views, float* dL, float* loss,
                      cudaStream_t stream) {
    const int64_t count = (int64_t)H * W * 3;
    if (count == 0) return cudaSuccess;
    const float norm = (float)(1.0 / (3.0 * (double)H * (double)W * (double)n_views));
    int64_t blocks = (count + 255) / 256;
    if (blocks > 152 * 8) blocks = 152 * 8;
    (void)launch_pdl(l1_kernel, dim3((int)blocks), dim3(256), 0, stream, image, target, count, norm, dL, loss);
    note_launch();
    return cudaGetLastError();
}

}  // namespace sgs
