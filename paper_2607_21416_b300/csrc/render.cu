// render.cu -- tile compositing (Eq. 1) forward and backward, the L1 term of
// Eq. 3, and the chain rule of the projection.
//
// One CTA of 256 threads per 16x16 tile (one thread per pixel), all views in
// one launch (tiles numbered view-major).  The tile's sorted splat list is
// staged through shared memory 256 records at a time; every thread reads the
// same record at the same time (broadcast, no bank conflicts).
//
// The power / alpha arithmetic is written with explicit fmaf / __fmul_rn so
// the forward pass, the recomputation inside the backward pass and any stored
// forward state take bit-identical skip / stop decisions.
#include "gs_internal.cuh"

namespace gs {

constexpr int kRT = kTilePix;   // 256 threads per tile

__device__ __forceinline__ float splat_power(float4 a, float cc, float px, float py, float *dx, float *dy)
{
    const float x = __fsub_rn(a.x, px), y = __fsub_rn(a.y, py);
    *dx = x; *dy = y;
    // -0.5 (ca x^2 + cc y^2) - cb x y
    const float q = fmaf(a.z, __fmul_rn(x, x), __fmul_rn(cc, __fmul_rn(y, y)));
    return fmaf(-0.5f, q, -__fmul_rn(a.w, __fmul_rn(x, y)));
}

__device__ __forceinline__ float splat_gauss(float power) { return __expf(power); }

struct TileCoord {
    int v, px, py;
    bool inside;
};
__device__ __forceinline__ TileCoord tile_coord(const ViewTable &vt, int t)
{
    TileCoord c;
    c.v = view_of_tile(vt, t);
    const int local = t - vt.tile_base[c.v];
    const int tx = local % vt.TX[c.v], ty = local / vt.TX[c.v];
    c.px = tx * kTile + (threadIdx.x & (kTile - 1));
    c.py = ty * kTile + (threadIdx.x >> 4);
    c.inside = c.px < vt.W[c.v] && c.py < vt.H[c.v];
    return c;
}

template <bool COUNT>
__global__ void __launch_bounds__(kRT) render_fwd_kernel(const float4 *__restrict__ rec,
                                                         const uint32_t *__restrict__ vals,
                                                         const uint32_t *__restrict__ ranges, ViewTable vt,
                                                         float bg0, float bg1, float bg2, float *__restrict__ image,
                                                         float *__restrict__ T_final, int32_t *__restrict__ last,
                                                         unsigned long long *__restrict__ n_eval,
                                                         const uint32_t *__restrict__ n_pairs, long long cap_cand,
                                                         const gs_status *st)
{
    if (has_error(st)) return;
    __shared__ float4 s_a[kRT];
    __shared__ float4 s_b[kRT];
    __shared__ float s_c[kRT];
    const int t = blockIdx.x;
    const TileCoord tc = tile_coord(vt, t);
    const float fpx = (float)tc.px, fpy = (float)tc.py;
    uint32_t start = ranges[2 * t], end = ranges[2 * t + 1];
    if (end < start || (end > start && !idx_ok(st, (long long)end - 1, (long long)*n_pairs, 41))) end = start;
    float T = 1.f, C0 = 0.f, C1 = 0.f, C2 = 0.f;
    int lastc = 0;
    bool done = !tc.inside;
    unsigned long long nev = 0, ncomp = 0;
    for (uint32_t b0 = start; b0 < end; b0 += kRT) {
        if (__syncthreads_count(done) == kRT) break;
        const uint32_t i = b0 + threadIdx.x;
        if (i < end) {
            size_t id = vals[i];
            if (!idx_ok(st, (long long)id, cap_cand, 42)) id = 0;
            const float4 r0 = __ldg(&rec[3 * id]);
            const float4 r1 = __ldg(&rec[3 * id + 1]);
            const float4 r2 = __ldg(&rec[3 * id + 2]);
            s_a[threadIdx.x] = r0;
            s_b[threadIdx.x] = r1;
            s_c[threadIdx.x] = r2.x;
        }
        __syncthreads();
        const int n = (int)min((uint32_t)kRT, end - b0);
        if (!done) {
            for (int j = 0; j < n; ++j) {
                if (COUNT) ++nev;
                const float4 a = s_a[j];
                const float4 bb = s_b[j];
                float dx, dy;
                const float power = splat_power(a, bb.x, fpx, fpy, &dx, &dy);
                if (power > 0.f) continue;
                const float alpha = fminf(kAlphaMax, __fmul_rn(bb.y, splat_gauss(power)));
                if (alpha < kAlphaMin) continue;
                const float Tn = __fmul_rn(T, 1.f - alpha);
                if (Tn < kTMin) { done = true; break; }
                const float w = __fmul_rn(alpha, T);
                C0 = fmaf(bb.z, w, C0);
                C1 = fmaf(bb.w, w, C1);
                C2 = fmaf(s_c[j], w, C2);
                T = Tn;
                lastc = (int)(b0 - start) + j + 1;
                if (COUNT) ++ncomp;
            }
        }
    }
    if (COUNT) {
        // warp-reduce the evaluation counts, one atomic per warp and counter
        for (int o = 16; o > 0; o >>= 1) {
            nev += __shfl_down_sync(0xffffffffu, nev, o);
            ncomp += __shfl_down_sync(0xffffffffu, ncomp, o);
        }
        if ((threadIdx.x & 31) == 0 && nev) atomicAdd(n_eval, nev);
        if ((threadIdx.x & 31) == 0 && ncomp) atomicAdd(n_eval + 1, ncomp);
    }
    if (!tc.inside) return;
    const int v = tc.v;
    const long long W = vt.W[v], H = vt.H[v];
    const long long pix = (long long)tc.py * W + tc.px;
    float *img = image + 3 * vt.pix_base[v];
    img[pix] = fmaf(T, bg0, C0);
    img[W * H + pix] = fmaf(T, bg1, C1);
    img[2 * W * H + pix] = fmaf(T, bg2, C2);
    if (T_final) T_final[vt.pix_base[v] + pix] = T;
    if (last) last[vt.pix_base[v] + pix] = lastc;
}

// ------------------------------------------------------------------- L1
__global__ void __launch_bounds__(256) l1_kernel(const float *__restrict__ image, const float *__restrict__ target,
                                                 ViewTable vt, float *__restrict__ loss, float *__restrict__ d_image)
{
    const long long n = 3 * vt.total_pixels;
    float acc = 0.f;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        int v = 0;
        while (v + 1 < vt.V && 3 * vt.pix_base[v + 1] <= i) ++v;
        const float inv = 1.f / (float)(3 * vt.pix_base[v + 1] - 3 * vt.pix_base[v]);
        const float d = image[i] - target[i];
        acc += fabsf(d) * inv;
        d_image[i] = d > 0.f ? inv : (d < 0.f ? -inv : 0.f);
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(loss, acc);
}

// ------------------------------------------------------------ backward
__device__ __forceinline__ float warp_sum(float x)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

__global__ void __launch_bounds__(kRT) render_bwd_kernel(
    const float4 *__restrict__ rec, const uint32_t *__restrict__ vals, const uint32_t *__restrict__ ranges,
    ViewTable vt, float bg0, float bg1, float bg2, const float *__restrict__ d_image,
    const float *__restrict__ T_final_in, const int32_t *__restrict__ last_in, float *__restrict__ sgrad,
    const uint32_t *__restrict__ n_pairs, long long cap_cand, const gs_status *st)
{
    if (has_error(st)) return;
    __shared__ float4 s_a[kRT];
    __shared__ float4 s_b[kRT];
    __shared__ float s_c[kRT];
    __shared__ uint32_t s_id[kRT];
    __shared__ int s_maxlast;
    const int t = blockIdx.x;
    const TileCoord tc = tile_coord(vt, t);
    const float fpx = (float)tc.px, fpy = (float)tc.py;
    uint32_t start = ranges[2 * t], end = ranges[2 * t + 1];
    if (end < start || (end > start && !idx_ok(st, (long long)end - 1, (long long)*n_pairs, 51))) end = start;
    const int v = tc.v;
    const long long W = vt.W[v], H = vt.H[v];
    const long long pix = (long long)tc.py * W + tc.px;
    float T = 1.f;
    int lastc = 0;
    if (threadIdx.x == 0) s_maxlast = 0;
    if (T_final_in) {
        if (tc.inside) {
            T = T_final_in[vt.pix_base[v] + pix];
            lastc = min(last_in[vt.pix_base[v] + pix], (int)(end - start));
        }
    } else {
        // recompute the forward transmittance and the last composited position
        bool done = !tc.inside;
        for (uint32_t b0 = start; b0 < end; b0 += kRT) {
            if (__syncthreads_count(done) == kRT) break;
            const uint32_t i = b0 + threadIdx.x;
            if (i < end) {
                size_t id = vals[i];
                if (!idx_ok(st, (long long)id, cap_cand, 52)) id = 0;
                s_a[threadIdx.x] = __ldg(&rec[3 * id]);
                s_b[threadIdx.x] = __ldg(&rec[3 * id + 1]);
            }
            __syncthreads();
            const int n = (int)min((uint32_t)kRT, end - b0);
            if (!done) {
                for (int j = 0; j < n; ++j) {
                    const float4 a = s_a[j];
                    const float4 bb = s_b[j];
                    float dx, dy;
                    const float power = splat_power(a, bb.x, fpx, fpy, &dx, &dy);
                    if (power > 0.f) continue;
                    const float alpha = fminf(kAlphaMax, __fmul_rn(bb.y, splat_gauss(power)));
                    if (alpha < kAlphaMin) continue;
                    const float Tn = __fmul_rn(T, 1.f - alpha);
                    if (Tn < kTMin) { done = true; break; }
                    T = Tn;
                    lastc = (int)(b0 - start) + j + 1;
                }
            }
        }
    }
    __syncthreads();
    atomicMax(&s_maxlast, lastc);
    float g0 = 0.f, g1 = 0.f, g2 = 0.f;
    if (tc.inside) {
        const float *dimg = d_image + 3 * vt.pix_base[v];
        g0 = dimg[pix]; g1 = dimg[W * H + pix]; g2 = dimg[2 * W * H + pix];
    }
    float B0 = T * bg0, B1 = T * bg1, B2 = T * bg2;
    __syncthreads();
    const int maxlast = min(s_maxlast, (int)(end - start));
    const int lane = threadIdx.x & 31;
    // back to front over list positions [0, maxlast)
    for (int hi = maxlast; hi > 0; hi -= kRT) {
        const int lo = max(0, hi - kRT);
        __syncthreads();
        {
            const int p = hi - 1 - (int)threadIdx.x;   // smem slot j <-> position hi-1-j
            if (p >= lo) {
                uint32_t id = vals[start + p];
                if (!idx_ok(st, (long long)id, cap_cand, 53)) id = 0;
                s_id[threadIdx.x] = id;
                s_a[threadIdx.x] = __ldg(&rec[3 * (size_t)id]);
                s_b[threadIdx.x] = __ldg(&rec[3 * (size_t)id + 1]);
                s_c[threadIdx.x] = __ldg(&rec[3 * (size_t)id + 2]).x;
            }
        }
        __syncthreads();
        const int n = hi - lo;
        for (int j = 0; j < n; ++j) {
            const int p = hi - 1 - j;
            float gmx = 0.f, gmy = 0.f, gca = 0.f, gcb = 0.f, gcc = 0.f, gop = 0.f, gr = 0.f, gg = 0.f, gb = 0.f;
            bool contrib = false;
            if (p < lastc) {
                const float4 a = s_a[j];
                const float4 bb = s_b[j];
                float dx, dy;
                const float power = splat_power(a, bb.x, fpx, fpy, &dx, &dy);
                if (power <= 0.f) {
                    const float G = splat_gauss(power);
                    const float ag = __fmul_rn(bb.y, G);
                    const float alpha = fminf(kAlphaMax, ag);
                    if (alpha >= kAlphaMin) {
                        contrib = true;
                        const float om = 1.f - alpha;
                        T = T / om;                      // transmittance in front of this splat
                        const float w = alpha * T;
                        gr = w * g0; gg = w * g1; gb = w * g2;
                        const float cr = bb.z, cg = bb.w, cbl = s_c[j];
                        const float dal = g0 * (cr * T - B0 / om) + g1 * (cg * T - B1 / om) +
                                          g2 * (cbl * T - B2 / om);
                        B0 = fmaf(cr, w, B0); B1 = fmaf(cg, w, B1); B2 = fmaf(cbl, w, B2);
                        if (ag < kAlphaMax) {
                            gop = dal * G;
                            const float dp = dal * alpha;
                            gmx = -dp * (a.z * dx + a.w * dy);
                            gmy = -dp * (bb.x * dy + a.w * dx);
                            gca = -0.5f * dp * dx * dx;
                            gcb = -dp * dx * dy;
                            gcc = -0.5f * dp * dy * dy;
                        }
                    }
                }
            }
            if (__any_sync(0xffffffffu, contrib)) {
                gmx = warp_sum(gmx); gmy = warp_sum(gmy); gca = warp_sum(gca); gcb = warp_sum(gcb);
                gcc = warp_sum(gcc); gop = warp_sum(gop); gr = warp_sum(gr); gg = warp_sum(gg); gb = warp_sum(gb);
                if (lane == 0) {
                    float *o = sgrad + 9 * (size_t)s_id[j];
                    atomicAdd(o + 0, gmx); atomicAdd(o + 1, gmy); atomicAdd(o + 2, gca);
                    atomicAdd(o + 3, gcb); atomicAdd(o + 4, gcc); atomicAdd(o + 5, gop);
                    atomicAdd(o + 6, gr); atomicAdd(o + 7, gg); atomicAdd(o + 8, gb);
                }
            }
        }
    }
}

// Projection chain rule, one thread per candidate.
struct ProjBwdArgs {
    const float *mu, *scale, *quat;
    const int32_t *view_start;
    const int32_t *tiles;
    const gs_camera *cams;
    const float *sgrad;
    int k, V;
    long long cap_cand;
    float *dmu, *dscale, *dquat, *dopacity, *dcolour;
    const gs_status *st;
};

__global__ void __launch_bounds__(256) project_bwd_kernel(ProjBwdArgs a, ViewTable vt)
{
    if (has_error(a.st)) return;
    const long long rows = __ldg(a.view_start + a.V);
    const long long C = std::min<long long>(rows * a.k, a.cap_cand);
    for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < C;
         c += (long long)gridDim.x * blockDim.x) {
        float dmu[3] = {0.f, 0.f, 0.f}, ds[3] = {0.f, 0.f, 0.f}, dq[4] = {0.f, 0.f, 0.f, 0.f};
        float dop = 0.f, dc0 = 0.f, dc1 = 0.f, dc2 = 0.f;
        if (__ldg(a.tiles + c) > 0) {
            const float *sg = a.sgrad + 9 * c;
            const float gmx = sg[0], gmy = sg[1], gka = sg[2], gkb = sg[3], gkc = sg[4];
            dop = sg[5]; dc0 = sg[6]; dc1 = sg[7]; dc2 = sg[8];
            const int v = view_of_row(a.view_start, a.V, (int)(c / a.k));
            const Cam cm = load_cam(a.cams, v);
            const float m0 = __ldg(a.mu + 3 * c), m1 = __ldg(a.mu + 3 * c + 1), m2 = __ldg(a.mu + 3 * c + 2);
            const float px = cm.R[0] * m0 + cm.R[1] * m1 + cm.R[2] * m2 + cm.t[0];
            const float py = cm.R[3] * m0 + cm.R[4] * m1 + cm.R[5] * m2 + cm.t[1];
            const float pz = cm.R[6] * m0 + cm.R[7] * m1 + cm.R[8] * m2 + cm.t[2];
            const float qw = __ldg(a.quat + 4 * c), qx = __ldg(a.quat + 4 * c + 1),
                        qy = __ldg(a.quat + 4 * c + 2), qz = __ldg(a.quat + 4 * c + 3);
            float Rq[9];
            Rq[0] = 1.f - 2.f * (qy * qy + qz * qz); Rq[1] = 2.f * (qx * qy - qw * qz); Rq[2] = 2.f * (qx * qz + qw * qy);
            Rq[3] = 2.f * (qx * qy + qw * qz); Rq[4] = 1.f - 2.f * (qx * qx + qz * qz); Rq[5] = 2.f * (qy * qz - qw * qx);
            Rq[6] = 2.f * (qx * qz - qw * qy); Rq[7] = 2.f * (qy * qz + qw * qx); Rq[8] = 1.f - 2.f * (qx * qx + qy * qy);
            const float s[3] = {__ldg(a.scale + 3 * c), __ldg(a.scale + 3 * c + 1), __ldg(a.scale + 3 * c + 2)};
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
            const float W = (float)vt.W[v], H = (float)vt.H[v];
            const float limx = kTanClamp * (W / (2.f * cm.fx)), limy = kTanClamp * (H / (2.f * cm.fy));
            const float ux = px / pz, uy = py / pz;
            const bool inx = ux >= -limx && ux <= limx, iny = uy >= -limy && uy <= limy;
            const float txz = fminf(fmaxf(ux, -limx), limx), tyz = fminf(fmaxf(uy, -limy), limy);
            const float fx = cm.fx, fy = cm.fy, z = pz;
            const float J[6] = {fx / z, 0.f, -fx * txz / z, 0.f, fy / z, -fy * tyz / z};
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
            if (det < 1e-3f * ca * cc) {
                const double A = ca, Bv = cb, Cv = cc;
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
            const float iz2 = 1.f / (z * z);
            float dp0 = 0.f, dp1 = 0.f, dp2 = 0.f;
            dp2 += dJ[0] * (-fx * iz2) + dJ[4] * (-fy * iz2);
            dp2 += dJ[2] * (fx * txz * iz2);
            if (inx) { dp0 += dJ[2] * (-fx * iz2); dp2 += dJ[2] * (fx * px * iz2 / z); }
            dp2 += dJ[5] * (fy * tyz * iz2);
            if (iny) { dp1 += dJ[5] * (-fy * iz2); dp2 += dJ[5] * (fy * py * iz2 / z); }
            dp0 += gmx * fx / z;
            dp1 += gmy * fy / z;
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
#pragma unroll
        for (int j = 0; j < 3; ++j) { a.dmu[3 * c + j] = dmu[j]; a.dscale[3 * c + j] = ds[j]; }
#pragma unroll
        for (int j = 0; j < 4; ++j) a.dquat[4 * c + j] = dq[j];
        a.dopacity[c] = dop;
        a.dcolour[3 * c] = dc0; a.dcolour[3 * c + 1] = dc1; a.dcolour[3 * c + 2] = dc2;
    }
}

// ------------------------------------------------------------ launchers
int launch_render_fwd(const gs_splats *sp, const gs_bins *bins, const ViewTable &vt, const float bg[3],
                      float *image, float *T_final, int32_t *last, long long *n_eval, gs_status *st,
                      cudaStream_t s)
{
    if (vt.total_tiles == 0) return GS_OK;
    const float4 *rec = reinterpret_cast<const float4 *>(sp->rec);
    if (n_eval) {
        cudaMemsetAsync(n_eval, 0, 2 * sizeof(long long), s);
        render_fwd_kernel<true><<<vt.total_tiles, kRT, 0, s>>>(rec, bins->vals, bins->ranges, vt, bg[0], bg[1],
                                                               bg[2], image, T_final, last,
                                                               reinterpret_cast<unsigned long long *>(n_eval),
                                                               bins->n_pairs, sp->cap, st);
    } else {
        render_fwd_kernel<false><<<vt.total_tiles, kRT, 0, s>>>(rec, bins->vals, bins->ranges, vt, bg[0], bg[1],
                                                                bg[2], image, T_final, last, nullptr,
                                                                bins->n_pairs, sp->cap, st);
    }
    count_launches(1);
    return cudaPeekAtLastError() == cudaSuccess ? GS_OK : GS_ERR_CUDA;
}

int launch_l1(const float *image, const float *target, const ViewTable &vt, float *loss, float *d_image,
              cudaStream_t s)
{
    cudaMemsetAsync(loss, 0, sizeof(float), s);
    const long long n = 3 * vt.total_pixels;
    const int grid = (int)std::max<long long>(1, std::min<long long>((n + 255) / 256, (long long)sm_count() * 8));
    l1_kernel<<<grid, 256, 0, s>>>(image, target, vt, loss, d_image);
    count_launches(1);
    return cudaPeekAtLastError() == cudaSuccess ? GS_OK : GS_ERR_CUDA;
}

int launch_render_bwd(const gs_gauss3d *g, const gs_camera *cams, const gs_splats *sp, const gs_bins *bins,
                      const ViewTable &vt, const float bg[3], const float *d_image, const float *T_final,
                      const int32_t *last, gs_splat_grad *sgrad, gs_gauss3d_grad *out, gs_status *st,
                      cudaStream_t s)
{
    const long long cap_cand = g->cap_rows * (long long)g->k;
    cudaMemsetAsync(sgrad->g, 0, sizeof(float) * 9 * (size_t)cap_cand, s);
    const float4 *rec = reinterpret_cast<const float4 *>(sp->rec);
    if (vt.total_tiles > 0) {
        render_bwd_kernel<<<vt.total_tiles, kRT, 0, s>>>(rec, bins->vals, bins->ranges, vt, bg[0], bg[1], bg[2],
                                                          d_image, T_final, last, sgrad->g, bins->n_pairs,
                                                          std::min<long long>(sp->cap, cap_cand), st);
        count_launches(1);
    }
    ProjBwdArgs a;
    a.mu = g->mu; a.scale = g->scale; a.quat = g->quat; a.view_start = g->view_start; a.tiles = sp->tiles;
    a.cams = cams; a.sgrad = sgrad->g; a.k = g->k; a.V = vt.V; a.cap_cand = cap_cand;
    a.dmu = out->dmu; a.dscale = out->dscale; a.dquat = out->dquat; a.dopacity = out->dopacity;
    a.dcolour = out->dcolour; a.st = st;
    const int grid = (int)std::max<long long>(1, std::min<long long>((cap_cand + 255) / 256, (long long)sm_count() * 16));
    project_bwd_kernel<<<grid, 256, 0, s>>>(a, vt);
    count_launches(1);
    return cudaPeekAtLastError() == cudaSuccess ? GS_OK : GS_ERR_CUDA;
}

}  // namespace gs
