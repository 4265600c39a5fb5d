// project.cu -- EWA projection of candidate Gaussians to 2D splat records.
//
// One thread per candidate (grid-stride over the device-side candidate count).
// Each writes a 48-byte record (mean, conic, opacity, colour, depth, tile
// rectangle) and its tile count; culled candidates get an empty rectangle.
// Near-degenerate splats (det < 1e-3 a c from the FP32 covariance) have
// their covariance formed again in compensated single precision
// (cov2d_f2.cuh) and its determinant and conic taken in FP64; everything
// else is FP32.
#include <cfloat>

#include "cov2d_f2.cuh"

namespace gs {

struct ProjectArgs {
    const float *mu, *scale, *quat, *opacity, *colour;
    const int32_t *view_start;
    const gs_camera *cams;
    int k, V;
    long long cap_cand;
    float4 *rec;
    int32_t *tiles;
    const gs_status *st;
};

__device__ __forceinline__ void quat_rot(float w, float x, float y, float z, float R[9])
{
    R[0] = 1.f - 2.f * (y * y + z * z); R[1] = 2.f * (x * y - w * z);       R[2] = 2.f * (x * z + w * y);
    R[3] = 2.f * (x * y + w * z);       R[4] = 1.f - 2.f * (x * x + z * z); R[5] = 2.f * (y * z - w * x);
    R[6] = 2.f * (x * z - w * y);       R[7] = 2.f * (y * z + w * x);       R[8] = 1.f - 2.f * (x * x + y * y);
}

__global__ void __launch_bounds__(256) project_kernel(ProjectArgs a, ViewTable vt)
{
    if (has_error(a.st)) return;
    const long long rows = __ldg(a.view_start + a.V);
    const long long C = std::min<long long>(rows * a.k, a.cap_cand);
    for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < C;
         c += (long long)gridDim.x * blockDim.x) {
        float4 r0 = make_float4(0.f, 0.f, 0.f, 0.f), r1 = r0, r2 = r0;
        int ntiles = 0;
        const float op = __ldg(a.opacity + c);
        const int v = view_of_row(a.view_start, a.V, (int)(c / a.k));
        const Cam cm = load_cam(a.cams, v);
        const float mx_ = __ldg(a.mu + 3 * c), my_ = __ldg(a.mu + 3 * c + 1), mz_ = __ldg(a.mu + 3 * c + 2);
        const float pz = cm.R[6] * mx_ + cm.R[7] * my_ + cm.R[8] * mz_ + cm.t[2];
        if (op > 0.f && pz > kNear) {
            const float px = cm.R[0] * mx_ + cm.R[1] * my_ + cm.R[2] * mz_ + cm.t[0];
            const float py = cm.R[3] * mx_ + cm.R[4] * my_ + cm.R[5] * mz_ + cm.t[1];
            float Rq[9];
            quat_rot(__ldg(a.quat + 4 * c), __ldg(a.quat + 4 * c + 1), __ldg(a.quat + 4 * c + 2),
                     __ldg(a.quat + 4 * c + 3), Rq);
            const float s0 = __ldg(a.scale + 3 * c), s1 = __ldg(a.scale + 3 * c + 1), s2 = __ldg(a.scale + 3 * c + 2);
            const float q0 = s0 * s0, q1 = s1 * s1, q2 = s2 * s2;
            // Sigma3 (symmetric)
            float S[6];
            S[0] = Rq[0] * Rq[0] * q0 + Rq[1] * Rq[1] * q1 + Rq[2] * Rq[2] * q2;
            S[1] = Rq[0] * Rq[3] * q0 + Rq[1] * Rq[4] * q1 + Rq[2] * Rq[5] * q2;
            S[2] = Rq[0] * Rq[6] * q0 + Rq[1] * Rq[7] * q1 + Rq[2] * Rq[8] * q2;
            S[3] = Rq[3] * Rq[3] * q0 + Rq[4] * Rq[4] * q1 + Rq[5] * Rq[5] * q2;
            S[4] = Rq[3] * Rq[6] * q0 + Rq[4] * Rq[7] * q1 + Rq[5] * Rq[8] * q2;
            S[5] = Rq[6] * Rq[6] * q0 + Rq[7] * Rq[7] * q1 + Rq[8] * Rq[8] * q2;
            const float W = (float)vt.W[v], H = (float)vt.H[v];
            const float limx = kTanClamp * (W / (2.f * cm.fx)), limy = kTanClamp * (H / (2.f * cm.fy));
            const float txz = fminf(fmaxf(px / pz, -limx), limx);
            const float tyz = fminf(fmaxf(py / pz, -limy), limy);
            const float j00 = cm.fx / pz, j02 = -cm.fx * txz / pz;
            const float j11 = cm.fy / pz, j12 = -cm.fy * tyz / pz;
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
                cov2d_compensated(cm, mx_, my_, mz_, __ldg(a.quat + 4 * c), __ldg(a.quat + 4 * c + 1),
                                  __ldg(a.quat + 4 * c + 2), __ldg(a.quat + 4 * c + 3), s0, s1, s2,
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
                const float mx = cm.fx * px / pz + cm.cx;
                const float my = cm.fy * py / pz + cm.cy;
                const float TX = (float)vt.TX[v], TY = (float)vt.TY[v];
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
                    r1 = make_float4(-0.5f * l2e * kc, log2f(op), __ldg(a.colour + 3 * c), __ldg(a.colour + 3 * c + 1));
                    r2 = make_float4(__ldg(a.colour + 3 * c + 2), pz,
                                     __uint_as_float((uint32_t)x0 | ((uint32_t)x1 << 16)),
                                     __uint_as_float((uint32_t)y0 | ((uint32_t)y1 << 16)));
                }
            }
        }
        a.rec[3 * c] = r0;
        a.rec[3 * c + 1] = r1;
        a.rec[3 * c + 2] = r2;
        a.tiles[c] = ntiles;
    }
}

int launch_project(const gs_gauss3d *g, const gs_camera *cams, const ViewTable &vt, gs_splats *out,
                   gs_status *st, cudaStream_t s)
{
    ProjectArgs a;
    a.mu = g->mu; a.scale = g->scale; a.quat = g->quat; a.opacity = g->opacity; a.colour = g->colour;
    a.view_start = g->view_start; a.cams = cams; a.k = g->k; a.V = vt.V;
    a.cap_cand = g->cap_rows * (long long)g->k;
    a.rec = reinterpret_cast<float4 *>(out->rec); a.tiles = out->tiles; a.st = st;
    const long long need = (a.cap_cand + 255) / 256;
    const int grid = (int)std::max<long long>(1, std::min<long long>(need, (long long)sm_count() * 16));
    project_kernel<<<grid, 256, 0, s>>>(a, vt);
    count_launches(1);
    return cudaPeekAtLastError() == cudaSuccess ? GS_OK : GS_ERR_CUDA;
}

}  // namespace gs
