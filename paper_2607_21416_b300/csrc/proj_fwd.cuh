// proj_fwd.cuh -- EWA projection of one candidate Gaussian to its 48-byte
// splat record (3DGS preliminaries, Sec. III-A), shared by gs_project and the
// fused decode + projection of the tensor-core decoder.
#pragma once

#include <cfloat>

#include "cov2d_f2.cuh"

namespace gs {

__device__ __forceinline__ void quat_rot(float w, float x, float y, float z, float R[9])
{
    R[0] = 1.f - 2.f * (y * y + z * z); R[1] = 2.f * (x * y - w * z);       R[2] = 2.f * (x * z + w * y);
    R[3] = 2.f * (x * y + w * z);       R[4] = 1.f - 2.f * (x * x + z * z); R[5] = 2.f * (y * z - w * x);
    R[6] = 2.f * (x * z - w * y);       R[7] = 2.f * (y * z + w * x);       R[8] = 1.f - 2.f * (x * x + y * y);
}

// Record of a candidate with mean (mx_, my_, mz_), scales sc, quaternion q,
// opacity op and colour col under camera cm of a Wv x Hv view (TXv x TYv
// tiles): p = R mu + t, culled if op <= 0 or p_z <= 0.2; Sigma2 = J R Sigma3
// R^T J^T + 0.3 I with the tangent clamp; culled if det <= 0; conic and
// radius (the near-degenerate branch in compensated covariance and FP64
// inverse); tile rectangle, culled if empty.  r0..r2 stay zero and *ntiles 0
// for a culled candidate.
__device__ __forceinline__ void project_one(const Cam &cm, float Wv, float Hv, int TXv, int TYv, float mx_, float my_,
                                            float mz_, const float sc[3], const float q[4], float op,
                                            const float col[3], float4 &r0, float4 &r1, float4 &r2, int &ntiles)
{
    const float pz = cm.R[6] * mx_ + cm.R[7] * my_ + cm.R[8] * mz_ + cm.t[2];
    if (op > 0.f && pz > kNear) {
        const float px = cm.R[0] * mx_ + cm.R[1] * my_ + cm.R[2] * mz_ + cm.t[0];
        const float py = cm.R[3] * mx_ + cm.R[4] * my_ + cm.R[5] * mz_ + cm.t[1];
        float Rq[9];
        quat_rot(q[0], q[1], q[2], q[3], Rq);
        const float s0 = sc[0], s1 = sc[1], s2 = sc[2];
        const float q0 = s0 * s0, q1 = s1 * s1, q2 = s2 * s2;
        // Sigma3 (symmetric)
        float S[6];
        S[0] = Rq[0] * Rq[0] * q0 + Rq[1] * Rq[1] * q1 + Rq[2] * Rq[2] * q2;
        S[1] = Rq[0] * Rq[3] * q0 + Rq[1] * Rq[4] * q1 + Rq[2] * Rq[5] * q2;
        S[2] = Rq[0] * Rq[6] * q0 + Rq[1] * Rq[7] * q1 + Rq[2] * Rq[8] * q2;
        S[3] = Rq[3] * Rq[3] * q0 + Rq[4] * Rq[4] * q1 + Rq[5] * Rq[5] * q2;
        S[4] = Rq[3] * Rq[6] * q0 + Rq[4] * Rq[7] * q1 + Rq[5] * Rq[8] * q2;
        S[5] = Rq[6] * Rq[6] * q0 + Rq[7] * Rq[7] * q1 + Rq[8] * Rq[8] * q2;
        const float W = Wv, H = Hv;
        const float limx = kTanClamp * (W / (2.f * cm.fx)), limy = kTanClamp * (H / (2.f * cm.fy));
        // one reciprocal of the depth (the reverse pass forms the same quotients for its clamp test)
        const float iz = 1.f / pz;
        const float ux = px * iz, uy = py * iz;
        const float txz = fminf(fmaxf(ux, -limx), limx);
        const float tyz = fminf(fmaxf(uy, -limy), limy);
        const float j00 = cm.fx * iz, j02 = -cm.fx * txz * iz;
        const float j11 = cm.fy * iz, j12 = -cm.fy * tyz * iz;
        // T = J R (2x3)
        float T0[3], T1[3];
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            T0[j] = j00 * cm.R[j] + j02 * cm.R[6 + j];
            T1[j] = j11 * cm.R[3 + j] + j12 * cm.R[6 + j];
        }
        // Sigma2 = T Sigma3 T^T
        float U0[3], U1[3];
        U0[0] = S[0] * T0[0] + S[1] * T0[1] + S[2] * T0[2];
        U0[1] = S[1] * T0[0] + S[3] * T0[1] + S[4] * T0[2];
        U0[2] = S[2] * T0[0] + S[4] * T0[1] + S[5] * T0[2];
        U1[0] = S[0] * T1[0] + S[1] * T1[1] + S[2] * T1[2];
        U1[1] = S[1] * T1[0] + S[3] * T1[1] + S[4] * T1[2];
        U1[2] = S[2] * T1[0] + S[4] * T1[1] + S[5] * T1[2];
        const float ca = T0[0] * U0[0] + T0[1] * U0[1] + T0[2] * U0[2] + kLowpass;
        const float cb = T0[0] * U1[0] + T0[1] * U1[1] + T0[2] * U1[2];
        const float cc = T1[0] * U1[0] + T1[1] * U1[1] + T1[2] * U1[2] + kLowpass;
        float det = ca * cc - cb * cb;
        float ka, kb, kc;
        if (det < 1e-3f * ca * cc) {
            double da, db, dc;
            cov2d_compensated(cm, mx_, my_, mz_, q[0], q[1], q[2], q[3], s0, s1, s2,
                              kTanClamp * (W / (2.f * cm.fx)), kTanClamp * (H / (2.f * cm.fy)), &da, &db, &dc);
            const double dd = da * dc - db * db;
            det = (float)dd;
            if (dd > 0.0) {
                ka = (float)(dc / dd);
                kb = (float)(-db / dd);
                kc = (float)(da / dd);
                if (!(det > 0.f)) det = FLT_MIN;   // positive, below FP32's normal range
            }
            if (!(dd > 0.0)) det = 0.f;
        } else {
            const float inv = 1.f / det;
            ka = cc * inv; kb = -cb * inv; kc = ca * inv;
        }
        if (det > 0.f) {
            const float mid = 0.5f * (ca + cc);
            const float lam = mid + sqrtf(fmaxf(0.1f, mid * mid - det));
            const float rad = ceilf(3.f * sqrtf(lam));
            const float mx = fmaf(cm.fx, ux, cm.cx);
            const float my = fmaf(cm.fy, uy, cm.cy);
            const float TX = (float)TXv, TY = (float)TYv;
            const float fx0 = fminf(fmaxf(floorf((mx - rad) * (1.f / kTile)), 0.f), TX);
            const float fx1 = fminf(fmaxf(floorf((mx + rad) * (1.f / kTile)) + 1.f, 0.f), TX);
            const float fy0 = fminf(fmaxf(floorf((my - rad) * (1.f / kTile)), 0.f), TY);
            const float fy1 = fminf(fmaxf(floorf((my + rad) * (1.f / kTile)) + 1.f, 0.f), TY);
            const int x0 = (int)fx0, x1 = (int)fx1, y0 = (int)fy0, y1 = (int)fy1;
            ntiles = (x1 - x0) * (y1 - y0);
            if (ntiles > 0) {
                // exponent coefficients in base 2: power * log2(e) = A dx^2 + B dx dy + C dy^2
                const float l2e = 1.4426950408889634f;
                r0 = make_float4(mx, my, -0.5f * l2e * ka, -l2e * kb);
                r1 = make_float4(-0.5f * l2e * kc, log2f(op), col[0], col[1]);
                r2 = make_float4(col[2], pz,
                                 __uint_as_float((uint32_t)x0 | ((uint32_t)x1 << 16)),
                                 __uint_as_float((uint32_t)y0 | ((uint32_t)y1 << 16)));
            }
        }
    }
}

}  // namespace gs
