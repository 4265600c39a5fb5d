// proj_bwd.cuh -- chain rule of the EWA projection for one candidate
// Gaussian (3DGS preliminaries, Sec. III-A), shared by gs_project_bwd and the
// fused decode + projection reverse pass.
#pragma once

#include "cov2d_f2.cuh"

namespace gs {

// From d mean2d = (gmx, gmy) and d conic = (gka, gkb, gkc) of a splat to the
// gradients of its mean mu, scales s and quaternion q (w, x, y, z) under the
// camera cm of a W x H view: Sigma2 = J W Sigma3 W^T J^T + 0.3 I with the
// tangent clamp (no gradient through a clamped coordinate), conic =
// Sigma2^-1 (FP64 inverse derivative on the compensated covariance where
// det < 1e-3 a c, as the forward), mean2d = (fx x/z + cx, fy y/z + cy).
__device__ __forceinline__ void proj_bwd_one(const Cam &cm, float W, float H, float m0, float m1, float m2,
                                             const float s[3], const float q[4], float gmx, float gmy, float gka,
                                             float gkb, float gkc, float dmu[3], float ds[3], float dq[4])
{
    const float px = cm.R[0] * m0 + cm.R[1] * m1 + cm.R[2] * m2 + cm.t[0];
    const float py = cm.R[3] * m0 + cm.R[4] * m1 + cm.R[5] * m2 + cm.t[1];
    const float pz = cm.R[6] * m0 + cm.R[7] * m1 + cm.R[8] * m2 + cm.t[2];
    const float qw = q[0], qx = q[1], qy = q[2], qz = q[3];
    float Rq[9];
    Rq[0] = 1.f - 2.f * (qy * qy + qz * qz); Rq[1] = 2.f * (qx * qy - qw * qz); Rq[2] = 2.f * (qx * qz + qw * qy);
    Rq[3] = 2.f * (qx * qy + qw * qz); Rq[4] = 1.f - 2.f * (qx * qx + qz * qz); Rq[5] = 2.f * (qy * qz - qw * qx);
    Rq[6] = 2.f * (qx * qz - qw * qy); Rq[7] = 2.f * (qy * qz + qw * qx); Rq[8] = 1.f - 2.f * (qx * qx + qy * qy);
    float M[9];   // Rq diag(s)
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) M[3 * i + j] = Rq[3 * i + j] * s[j];
    float S3[9];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j)
            S3[3 * i + j] = M[3 * i] * M[3 * j] + M[3 * i + 1] * M[3 * j + 1] + M[3 * i + 2] * M[3 * j + 2];
    const float limx = kTanClamp * (W / (2.f * cm.fx)), limy = kTanClamp * (H / (2.f * cm.fy));
    const float iz = 1.f / pz;
    const float ux = px * iz, uy = py * iz;   // the forward's quotients (same clamp decisions)
    const bool inx = ux >= -limx && ux <= limx, iny = uy >= -limy && uy <= limy;
    const float txz = fminf(fmaxf(ux, -limx), limx), tyz = fminf(fmaxf(uy, -limy), limy);
    const float fx = cm.fx, fy = cm.fy, z = pz;
    const float J[6] = {fx * iz, 0.f, -fx * txz * iz, 0.f, fy * iz, -fy * tyz * iz};
    float T[6];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j)
            T[3 * i + j] = J[3 * i] * cm.R[j] + J[3 * i + 1] * cm.R[3 + j] + J[3 * i + 2] * cm.R[6 + j];
    float TS[6];   // T S3
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j)
            TS[3 * i + j] = T[3 * i] * S3[j] + T[3 * i + 1] * S3[3 + j] + T[3 * i + 2] * S3[6 + j];
    const float ca = TS[0] * T[0] + TS[1] * T[1] + TS[2] * T[2] + kLowpass;
    const float cb = TS[0] * T[3] + TS[1] * T[4] + TS[2] * T[5];
    const float cc = TS[3] * T[3] + TS[4] * T[4] + TS[5] * T[5] + kLowpass;
    float da, db, dcv;
    const float det = ca * cc - cb * cb;
    if (det < 1e-3f * ca * cc) {   // near-degenerate: the forward's compensated covariance, FP64 inverse
        double A, Bv, Cv;
        cov2d_compensated(cm, m0, m1, m2, qw, qx, qy, qz, s[0], s[1], s[2], limx, limy, &A, &Bv, &Cv);
        const double dd = A * Cv - Bv * Bv, d2 = dd * dd;
        da = (float)((gka * (-Cv * Cv) + gkb * (Bv * Cv) + gkc * (-Bv * Bv)) / d2);
        db = (float)((gka * (2 * Bv * Cv) + gkb * (-(A * Cv + Bv * Bv)) + gkc * (2 * A * Bv)) / d2);
        dcv = (float)((gka * (-Bv * Bv) + gkb * (A * Bv) + gkc * (-A * A)) / d2);
    } else {
        const float i2 = 1.f / (det * det);
        da = (gka * (-cc * cc) + gkb * (cb * cc) + gkc * (-cb * cb)) * i2;
        db = (gka * (2.f * cb * cc) + gkb * (-(ca * cc + cb * cb)) + gkc * (2.f * ca * cb)) * i2;
        dcv = (gka * (-cb * cb) + gkb * (ca * cb) + gkc * (-ca * ca)) * i2;
    }
    const float G2[4] = {da, 0.5f * db, 0.5f * db, dcv};
    // dS3 = T^T G2 T ; dT = 2 G2 T S3
    float GT[6];   // G2 T
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) GT[3 * i + j] = G2[2 * i] * T[j] + G2[2 * i + 1] * T[3 + j];
    float dS3[9];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) dS3[3 * i + j] = T[i] * GT[j] + T[3 + i] * GT[3 + j];
    float dT[6];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j)
            dT[3 * i + j] = 2.f * (G2[2 * i] * TS[j] + G2[2 * i + 1] * TS[3 + j]);
    float dJ[6];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j)
            dJ[3 * i + j] = dT[3 * i] * cm.R[3 * j] + dT[3 * i + 1] * cm.R[3 * j + 1] + dT[3 * i + 2] * cm.R[3 * j + 2];
    const float iz2 = iz * iz;
    float dp0 = 0.f, dp1 = 0.f, dp2 = 0.f;
    dp2 += dJ[0] * (-fx * iz2) + dJ[4] * (-fy * iz2);
    dp2 += dJ[2] * (fx * txz * iz2);
    if (inx) { dp0 += dJ[2] * (-fx * iz2); dp2 += dJ[2] * (fx * px * iz2 * iz); }
    dp2 += dJ[5] * (fy * tyz * iz2);
    if (iny) { dp1 += dJ[5] * (-fy * iz2); dp2 += dJ[5] * (fy * py * iz2 * iz); }
    dp0 += gmx * fx * iz;
    dp1 += gmy * fy * iz;
    dp2 += gmx * (-fx * px * iz2) + gmy * (-fy * py * iz2);
#pragma unroll
    for (int j = 0; j < 3; ++j) dmu[j] = cm.R[j] * dp0 + cm.R[3 + j] * dp1 + cm.R[6 + j] * dp2;
    // dM = 2 dS3 M ; dscale_j = sum_i dM_ij Rq_ij ; dRq_ij = dM_ij s_j
    float dRq[9];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        float acc = 0.f;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            const float dM = 2.f * (dS3[3 * i] * M[j] + dS3[3 * i + 1] * M[3 + j] + dS3[3 * i + 2] * M[6 + j]);
            acc += dM * Rq[3 * i + j];
            dRq[3 * i + j] = dM * s[j];
        }
        ds[j] = acc;
    }
    dq[0] = 2.f * (-qz * dRq[1] + qy * dRq[2] + qz * dRq[3] - qx * dRq[5] - qy * dRq[6] + qx * dRq[7]);
    dq[1] = 2.f * (qy * dRq[1] + qz * dRq[2] + qy * dRq[3] - 2.f * qx * dRq[4] - qw * dRq[5] +
                   qz * dRq[6] + qw * dRq[7] - 2.f * qx * dRq[8]);
    dq[2] = 2.f * (-2.f * qy * dRq[0] + qx * dRq[1] + qw * dRq[2] + qx * dRq[3] + qz * dRq[5] -
                   qw * dRq[6] + qz * dRq[7] - 2.f * qy * dRq[8]);
    dq[3] = 2.f * (-2.f * qz * dRq[0] - qw * dRq[1] + qx * dRq[2] + qw * dRq[3] - 2.f * qz * dRq[4] +
                   qy * dRq[5] + qx * dRq[6] + qy * dRq[7]);
}

}  // namespace gs
