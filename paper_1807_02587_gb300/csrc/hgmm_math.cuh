// Small device-side numerics used by the build and registration kernels.
//
//  * two_sum        Knuth's error-free transformation a + b = s + e, the
//                   building block of the compensated (Kahan-style) moment
//                   sums of the precision form.
//  * jacobi_eig3    cyclic Jacobi eigen-decomposition of a symmetric 3x3
//                   matrix in FP64 (Jacobi's method with Rutishauser's
//                   rotation formulas), eigenvalues sorted descending
//                   (lambda_1 >= lambda_2 >= lambda_3, Sec. 4.1), each
//                   eigenvector signed so that its largest-magnitude entry is
//                   positive.
//  * chol3 / pack   FP64 Cholesky factor of a 3x3 covariance and the
//                   E-step constants of Eq. 2 in log2 units.
//  * chol_solve6    FP64 Cholesky (LL^T) solve of the 6x6 normal equations
//                   of Eq. 16.
//  * rodrigues      axis-angle to rotation matrix (FP64).
#pragma once

#include <cuda_runtime.h>
#include <math_constants.h>

#include "hgmm_internal.cuh"

namespace hgmm {

// ------------------------------------------------- FP32 special functions
// 2^x and 1/x by the multi-function unit's approximations (PTX ex2.approx /
// rcp.approx, .ftz): one instruction each.  The E-step and the descent take
// exponentials of max-subtracted log2 scores (x <= 0; a result below the
// smallest normal flushes to zero, a negligible posterior) and one
// reciprocal of a posterior sum in [1, 8]; the approximations' relative
// errors (about 2^-22 and 2^-23) are below the FP32 rounding that the
// moment sums carry anyway.
__device__ __forceinline__ float ex2_fast(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float rcp_fast(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float rsqrt_fast(float x) {
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// ---------------------------------------------------------------- FP32 sums
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bp = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bp)), __fsub_rn(b, bp));
}

// (s, c) += (s2, c2): compensated pair addition.
__device__ __forceinline__ void pair_add(float& s, float& c, float s2, float c2) {
    float t, e;
    two_sum(s, s2, t, e);
    s = t;
    c = __fadd_rn(c, __fadd_rn(c2, e));
}

// ---------------------------------------------------------------- FP64 helpers
// On sm_103 every FP64 warp instruction holds the SM sub-partition's FP64
// pipe ~64 cycles and the library FP64 division / square root take several
// hundred, so FP64 reciprocals and inverse square roots start from the
// multi-function unit's FP64 approximations (rcp.approx.ftz.f64 /
// rsqrt.approx.ftz.f64, relative error about 2^-20 on this part) and take one
// third-order correction step in FP64: for 1/x, r (1 + e + e^2) with
// e = 1 - x r; for 1/sqrt(x), y (1 + e/2 + 3 e^2/8) with e = 1 - x y^2 (the
// truncated binomial series of (1 - e)^-1 and (1 - e)^-1/2).  The remainder
// is O(e^3) < 2^-58, below FP64 rounding, in three and five FP64
// instructions.  Inputs outside [2^-1000, 2^1000] (and zero, negative
// square-root arguments, infinities, NaN) take the library routine.
__device__ __forceinline__ bool f64_normal_range(double x) {
    const int be = (__double2hiint(x) >> 20) & 0x7FF;
    return be >= 23 && be <= 2023;
}

__device__ __forceinline__ double rcp_f64(double x) {
    if (!f64_normal_range(x)) return 1.0 / x;
    double r;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(x));
    const double e = fma(-x, r, 1.0);
    return fma(r, fma(e, e, e), r);
}

__device__ __forceinline__ double rsqrt_f64(double x) {
    if (__double2hiint(x) < 0 || !f64_normal_range(x)) return rsqrt(x);
    double y;
    asm("rsqrt.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
    const double e = fma(-x * y, y, 1.0);
    return fma(y, e * fma(e, 0.375, 0.5), y);
}

// ---------------------------------------------------------------- FP64 3x3
// S packed xx xy xz yy yz zz.
__device__ inline void jacobi_eig3(const double S[6], double lam[3], double V[9]) {
    double a[3][3] = {{S[0], S[1], S[2]}, {S[1], S[3], S[4]}, {S[2], S[4], S[5]}};
    double v[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
    for (int sweep = 0; sweep < 40; ++sweep) {
        const double off = a[0][1] * a[0][1] + a[0][2] * a[0][2] + a[1][2] * a[1][2];
        const double dia = a[0][0] * a[0][0] + a[1][1] * a[1][1] + a[2][2] * a[2][2];
        if (!(off > 1e-34 * dia)) break;  // also stops on NaN
        for (int pq = 0; pq < 3; ++pq) {
            const int p = pq == 2 ? 1 : 0;
            const int q = pq == 0 ? 1 : 2;
            const double apq = a[p][q];
            if (apq == 0.0) continue;
            const double theta = (a[q][q] - a[p][p]) / (2.0 * apq);
            double t;
            if (fabs(theta) > 1e150) {
                t = 0.5 / theta;  // theta^2 would overflow: t ~ 1/(2 theta)
            } else {
                t = 1.0 / (fabs(theta) + sqrt(theta * theta + 1.0));
                if (theta < 0.0) t = -t;
            }
            const double c = 1.0 / sqrt(t * t + 1.0);
            const double s = t * c;
            a[p][p] -= t * apq;
            a[q][q] += t * apq;
            a[p][q] = a[q][p] = 0.0;
            const int r = 3 - p - q;
            const double arp = a[r][p], arq = a[r][q];
            a[r][p] = a[p][r] = c * arp - s * arq;
            a[r][q] = a[q][r] = s * arp + c * arq;
            for (int k = 0; k < 3; ++k) {
                const double vkp = v[k][p], vkq = v[k][q];
                v[k][p] = c * vkp - s * vkq;
                v[k][q] = s * vkp + c * vkq;
            }
        }
    }
    int idx[3] = {0, 1, 2};
    double d[3] = {a[0][0], a[1][1], a[2][2]};
    // sort descending (3 elements)
    if (d[idx[0]] < d[idx[1]]) { int x = idx[0]; idx[0] = idx[1]; idx[1] = x; }
    if (d[idx[1]] < d[idx[2]]) { int x = idx[1]; idx[1] = idx[2]; idx[2] = x; }
    if (d[idx[0]] < d[idx[1]]) { int x = idx[0]; idx[0] = idx[1]; idx[1] = x; }
    for (int c = 0; c < 3; ++c) {
        const int k = idx[c];
        lam[c] = d[k];
        int best = 0;
        for (int r = 1; r < 3; ++r)
            if (fabs(v[r][k]) > fabs(v[best][k])) best = r;
        const double sg = v[best][k] < 0.0 ? -1.0 : 1.0;
        for (int r = 0; r < 3; ++r) V[r * 3 + c] = sg * v[r][k];
    }
}

// Symmetric 3x3 eigen-decomposition accurate to FP64: cyclic Jacobi in FP32
// brings the matrix to within ~1e-7 of diagonal, the FP32 eigenvectors are
// re-orthonormalised in FP64 (Gram-Schmidt), the FP64 matrix is rotated into
// that basis and FP64 Jacobi sweeps (quadratically convergent) finish it.
// Eigenvalues descending, each eigenvector signed so that its largest-
// magnitude entry is positive.
__device__ inline void eig3(const double S[6], double lam[3], double V[9]) {
    double sc = fmax(fmax(fabs(S[0]), fabs(S[3])), fabs(S[5]));
    sc = fmax(sc, fmax(fmax(fabs(S[1]), fabs(S[2])), fabs(S[4])));
    if (!(sc > 0.0) || !isfinite(sc)) {
        jacobi_eig3(S, lam, V);  // zero or non-finite input: plain path
        return;
    }
    const double isc = rcp_f64(sc);
    // 1) FP32 cyclic Jacobi on S / sc
    float a[3][3] = {{float(S[0] * isc), float(S[1] * isc), float(S[2] * isc)},
                     {float(S[1] * isc), float(S[3] * isc), float(S[4] * isc)},
                     {float(S[2] * isc), float(S[4] * isc), float(S[5] * isc)}};
    float v[3][3] = {{1.f, 0.f, 0.f}, {0.f, 1.f, 0.f}, {0.f, 0.f, 1.f}};
    for (int sweep = 0; sweep < 12; ++sweep) {
        const float off = a[0][1] * a[0][1] + a[0][2] * a[0][2] + a[1][2] * a[1][2];
        if (!(off > 1e-18f)) break;
        for (int pq = 0; pq < 3; ++pq) {
            const int p = pq == 2 ? 1 : 0, q = pq == 0 ? 1 : 2;
            const float apq = a[p][q];
            if (apq == 0.f) continue;
            // the rotation from the multi-function unit's approximations
            // (relative errors ~2^-22): this phase only brings the matrix
            // near diagonal, and the FP64 sweeps below finish from whatever
            // orthonormal basis it reaches
            const float theta = (a[q][q] - a[p][p]) * rcp_fast(2.f * apq);
            const float h = fmaf(theta, theta, 1.f);
            float t = rcp_fast(fabsf(theta) + h * rsqrt_fast(h));  // 1 / (|theta| + sqrt(theta^2 + 1))
            if (theta < 0.f) t = -t;
            if (fabsf(theta) > 1e18f) t = 0.5f * rcp_fast(theta);
            const float c = rsqrt_fast(fmaf(t, t, 1.f)), s = t * c;
            a[p][p] -= t * apq;
            a[q][q] += t * apq;
            a[p][q] = a[q][p] = 0.f;
            const int r = 3 - p - q;
            const float arp = a[r][p], arq = a[r][q];
            a[r][p] = a[p][r] = c * arp - s * arq;
            a[r][q] = a[q][r] = s * arp + c * arq;
            for (int k = 0; k < 3; ++k) {
                const float vkp = v[k][p], vkq = v[k][q];
                v[k][p] = c * vkp - s * vkq;
                v[k][q] = s * vkp + c * vkq;
            }
        }
    }
    // 2) FP64 Gram-Schmidt of the FP32 columns
    double U[3][3];
    for (int c = 0; c < 3; ++c)
        for (int r = 0; r < 3; ++r) U[r][c] = v[r][c];
    for (int c = 0; c < 3; ++c) {
        for (int b = 0; b < c; ++b) {
            const double d = U[0][b] * U[0][c] + U[1][b] * U[1][c] + U[2][b] * U[2][c];
            for (int r = 0; r < 3; ++r) U[r][c] -= d * U[r][b];
        }
        const double nn = rsqrt_f64(U[0][c] * U[0][c] + U[1][c] * U[1][c] + U[2][c] * U[2][c]);
        for (int r = 0; r < 3; ++r) U[r][c] *= nn;
    }
    // 3) B = U^T S U in FP64 (unscaled S)
    const double Sm[3][3] = {{S[0], S[1], S[2]}, {S[1], S[3], S[4]}, {S[2], S[4], S[5]}};
    double SU[3][3], B[3][3];
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) SU[r][c] = Sm[r][0] * U[0][c] + Sm[r][1] * U[1][c] + Sm[r][2] * U[2][c];
    for (int r = 0; r < 3; ++r)
        for (int c = r; c < 3; ++c)
            B[r][c] = B[c][r] = U[0][r] * SU[0][c] + U[1][r] * SU[1][c] + U[2][r] * SU[2][c];
    // 4) FP64 Jacobi sweeps on the nearly diagonal B.  After the FP32 sweeps
    // the off-diagonal entries are ~1e-7 of the diagonal, so a rotation's
    // tan(phi) is apq / gap up to O(t^3) (t ~ 1e-7: far below FP64 rounding)
    // and cos(phi) = 1 - t^2 / 2 to O(t^4); one sweep leaves off-diagonals of
    // O(t^2).  The convergence test comes after the sweep: a second sweep
    // runs only where a pair with nearly equal eigenvalues took an exact
    // (large) rotation and refilled the others.  FP64 instructions hold this
    // part's FP64 pipe ~64 cycles each, so the common path is kept short.
    for (int sweep = 0; sweep < 3; ++sweep) {
        for (int pq = 0; pq < 3; ++pq) {
            const int p = pq == 2 ? 1 : 0, q = pq == 0 ? 1 : 2;
            const double apq = B[p][q];
            if (apq == 0.0) continue;
            const double gap = B[q][q] - B[p][p];
            double t, c;
            if (fabs(apq) < 1e-5 * fabs(gap)) {
                // small angle: t = tan(phi) ~ apq / gap to O(t^3) < 1e-15 t
                t = apq * rcp_f64(gap);
                c = 1.0 - 0.5 * t * t;
            } else {
                const double theta = gap * rcp_f64(2.0 * apq);
                if (fabs(theta) > 1e150) {
                    t = 0.5 * rcp_f64(theta);
                } else {
                    const double h = theta * theta + 1.0;
                    t = rcp_f64(fabs(theta) + h * rsqrt_f64(h));
                    if (theta < 0.0) t = -t;
                }
                c = rsqrt_f64(t * t + 1.0);
            }
            const double s = t * c;
            B[p][p] -= t * apq;
            B[q][q] += t * apq;
            B[p][q] = B[q][p] = 0.0;
            const int r = 3 - p - q;
            const double brp = B[r][p], brq = B[r][q];
            B[r][p] = B[p][r] = c * brp - s * brq;
            B[r][q] = B[q][r] = s * brp + c * brq;
            for (int k = 0; k < 3; ++k) {
                const double ukp = U[k][p], ukq = U[k][q];
                U[k][p] = c * ukp - s * ukq;
                U[k][q] = s * ukp + c * ukq;
            }
        }
        const double off = B[0][1] * B[0][1] + B[0][2] * B[0][2] + B[1][2] * B[1][2];
        const double dia = B[0][0] * B[0][0] + B[1][1] * B[1][1] + B[2][2] * B[2][2];
        if (!(off > 1e-26 * dia)) break;
    }
    int idx[3] = {0, 1, 2};
    const double d[3] = {B[0][0], B[1][1], B[2][2]};
    if (d[idx[0]] < d[idx[1]]) { int x = idx[0]; idx[0] = idx[1]; idx[1] = x; }
    if (d[idx[1]] < d[idx[2]]) { int x = idx[1]; idx[1] = idx[2]; idx[2] = x; }
    if (d[idx[0]] < d[idx[1]]) { int x = idx[0]; idx[0] = idx[1]; idx[1] = x; }
    for (int c = 0; c < 3; ++c) {
        const int k = idx[c];
        lam[c] = d[k];
        int best = 0;
        for (int r = 1; r < 3; ++r)
            if (fabs(U[r][k]) > fabs(U[best][k])) best = r;
        const double sg = U[best][k] < 0.0 ? -1.0 : 1.0;
        for (int r = 0; r < 3; ++r) V[r * 3 + c] = sg * U[r][k];
    }
}

// Cholesky Sigma = L L^T, returns false if not positive definite.
// L packed: L00 L10 L11 L20 L21 L22; R = 1 / (L00, L11, L22).
__device__ inline bool chol3(const double S[6], double L[6], double R[3]) {
    const double d0 = S[0];
    if (!(d0 > 0.0)) return false;
    const double r0 = rsqrt_f64(d0);
    const double l10 = S[1] * r0;
    const double l20 = S[2] * r0;
    const double d1 = S[3] - l10 * l10;
    if (!(d1 > 0.0)) return false;
    const double r1 = rsqrt_f64(d1);
    const double l21 = (S[4] - l20 * l10) * r1;
    const double d2 = S[5] - l20 * l20 - l21 * l21;
    if (!(d2 > 0.0)) return false;
    const double r2 = rsqrt_f64(d2);
    L[0] = d0 * r0; L[1] = l10; L[2] = d1 * r1; L[3] = l20; L[4] = l21; L[5] = d2 * r2;
    R[0] = r0; R[1] = r1; R[2] = r2;
    return true;
}

// E-step constants of a live node (see NodeEst): returns false when Sigma
// needed extra diagonal loading to become positive definite.
__device__ inline bool pack_est(double pi, const double mu[3], const double S_in[6],
                                double eps, float stop, NodeEst& out) {
    double S[6] = {S_in[0], S_in[1], S_in[2], S_in[3], S_in[4], S_in[5]};
    double L[6], R[3];
    bool clean = true;
    double boost = eps > 0.0 ? eps : 1e-30;
    bool ok = chol3(S, L, R);
    for (int tries = 0; tries < 8 && !ok; ++tries) {
        clean = false;
        S[0] += boost; S[3] += boost; S[5] += boost;
        boost *= 10.0;
        ok = chol3(S, L, R);
    }
    if (!ok) {  // hopeless (NaN input): make it an isotropic unit Gaussian
        L[0] = 1; L[1] = 0; L[2] = 1; L[3] = 0; L[4] = 0; L[5] = 1;
        R[0] = 1; R[1] = 1; R[2] = 1;
        clean = false;
    }
    // M = L^-1 (lower triangular)
    const double m00 = R[0], m11 = R[1], m22 = R[2];
    const double m10 = -L[1] * m00 * m11;
    const double m21 = -L[4] * m11 * m22;
    const double m20 = -(L[3] * m00 + L[4] * m10) * m22;
    const double k = sqrt(0.5 * 1.4426950408889634);  // sqrt(log2(e) / 2)
    // log-normaliser in FP32 (it is stored as FP32): log2 det(L) from the
    // FP64 product split into exponent and mantissa
    int ex = 0;
    const double mant = frexp(L[0] * L[2] * L[5], &ex);
    const float C = log2f(float(pi)) - 3.9547135f /* 1.5 log2(2 pi) */ -
                    (float(ex) + log2f(float(mant)));
    out.a = make_float4(float(mu[0]), float(mu[1]), float(mu[2]), C);
    out.b = make_float4(float(k * m00), float(k * m10), float(k * m11), float(k * m20));
    out.c = make_float4(float(k * m21), float(k * m22), stop, 0.f);
    return clean;
}

__device__ inline void dead_est(const double mu[3], NodeEst& out) {
    out.a = make_float4(float(mu[0]), float(mu[1]), float(mu[2]), -CUDART_INF_F);
    out.b = make_float4(0.f, 0.f, 0.f, 0.f);
    out.c = make_float4(0.f, 0.f, 0.f, 0.f);
}

// ---------------------------------------------------------------- FP64 6x6
// H packed upper row-major (21): (0,0..5),(1,1..5),...; solves H x = g.
__device__ inline bool chol_solve6(const double Hu[21], const double g[6], double x[6]) {
    double A[6][6];
    int k = 0;
    double dmax = 0.0;
    for (int i = 0; i < 6; ++i)
        for (int j = i; j < 6; ++j) {
            A[i][j] = A[j][i] = Hu[k++];
        }
    for (int i = 0; i < 6; ++i) dmax = fmax(dmax, fabs(A[i][i]));
    if (!(dmax > 0.0)) return false;
    // L L^T with one reciprocal per pivot (multiplications replace divisions)
    double L[6][6] = {};
    double inv[6];
    for (int j = 0; j < 6; ++j) {
        double d = A[j][j];
        for (int p = 0; p < j; ++p) d -= L[j][p] * L[j][p];
        if (!(d > 1e-15 * dmax)) return false;
        const double r = rsqrt_f64(d);  // 1 / L_jj
        L[j][j] = d * r;
        inv[j] = r;
        for (int i = j + 1; i < 6; ++i) {
            double s = A[i][j];
            for (int p = 0; p < j; ++p) s -= L[i][p] * L[j][p];
            L[i][j] = s * r;
        }
    }
    double y[6];
    for (int i = 0; i < 6; ++i) {
        double s = g[i];
        for (int p = 0; p < i; ++p) s -= L[i][p] * y[p];
        y[i] = s * inv[i];
    }
    for (int i = 5; i >= 0; --i) {
        double s = y[i];
        for (int p = i + 1; p < 6; ++p) s -= L[p][i] * x[p];
        x[i] = s * inv[i];
    }
    return true;
}

__device__ inline void rodrigues(const double w[3], double R[9]) {
    const double th2 = w[0] * w[0] + w[1] * w[1] + w[2] * w[2];
    const double th = sqrt(th2);
    double a, b;  // R = I + a K + b K^2
    if (th < 1e-8) {
        a = 1.0 - th2 / 6.0;
        b = 0.5 - th2 / 24.0;
    } else {
        a = sin(th) / th;
        b = (1.0 - cos(th)) / th2;
    }
    const double K[9] = {0, -w[2], w[1], w[2], 0, -w[0], -w[1], w[0], 0};
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double kk = 0.0;
            for (int m = 0; m < 3; ++m) kk += K[i * 3 + m] * K[m * 3 + j];
            R[i * 3 + j] = (i == j ? 1.0 : 0.0) + a * K[i * 3 + j] + b * kk;
        }
}

}  // namespace hgmm
