// render_bwd.cu -- reverse of the tile compositing (Eq. 1) over chunked work
// items, and the chain rule of the projection.
//
// Per item and pixel the reverse traversal starts from the transmittance after
// the item's last composited splat and the colour composited behind it, and
// walks the chunk's list back to front.  Single-chunk tiles take those from the
// forward's optional per-pixel output or recompute them (one extra front-to-back
// pass over the tile); multi-chunk tiles read them from the per-chunk state the
// forward left in the render workspace.  Per-splat sums are reduced across the
// warp (shuffles) before one global atomicAdd per warp and quantity.
#include "render_common.cuh"

namespace gs {

__device__ __forceinline__ float warp_sum(float x)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

__global__ void __launch_bounds__(kRT) render_bwd_kernel(
    const float4 *__restrict__ rec, const uint32_t *__restrict__ vals, const uint32_t *__restrict__ ranges,
    ViewTable vt, RenderPlan plan, float bg0, float bg1, float bg2, const float *__restrict__ d_image,
    const float *__restrict__ T_final_in, const int32_t *__restrict__ last_in, float *__restrict__ sgrad,
    long long cap_cand, const gs_status *st)
{
    if (has_error(st)) return;
    Item it;
    if (!item_of(blockIdx.x, plan.item_base, vt.total_tiles, ranges, plan.L, &it)) return;
    __shared__ Staged S;
    __shared__ int s_maxlast;
    const TileCoord tc = tile_coord(vt, it.t);
    const float fpx = (float)tc.px, fpy = (float)tc.py;
    const int v = tc.v;
    const long long W = vt.W[v], H = vt.H[v];
    const long long pix = (long long)tc.py * W + tc.px;
    const int n_items = (int)(it.s1 - it.s0);
    float T = 1.f, B0 = 0.f, B1 = 0.f, B2 = 0.f;
    int lastc = 0;
    if (threadIdx.x == 0) s_maxlast = 0;
    if (it.nk > 1) {
        // state of the forward: start transmittance, end state, colour behind
        float T0 = 1.f, Tf = 1.f;
        for (int j = 0; j < it.nk; ++j) {
            if (!(T0 >= kTMin)) break;
            const int item = it.base + j;
            if (j > it.k) {
                B0 += state_plane(plan.state, item, 2)[threadIdx.x];
                B1 += state_plane(plan.state, item, 3)[threadIdx.x];
                B2 += state_plane(plan.state, item, 4)[threadIdx.x];
            }
            Tf = state_plane(plan.state, item, 1)[threadIdx.x];
            if (j == it.k) {
                T = Tf;
                lastc = reinterpret_cast<const int *>(state_plane(plan.state, item, 5))[threadIdx.x];
            }
            T0 = __fmul_rn(T0, state_plane(plan.state, item, 0)[threadIdx.x]);
        }
        if (!tc.inside) lastc = 0;
        B0 = fmaf(Tf, bg0, B0); B1 = fmaf(Tf, bg1, B1); B2 = fmaf(Tf, bg2, B2);
    } else if (T_final_in) {
        if (tc.inside) {
            T = T_final_in[vt.pix_base[v] + pix];
            lastc = min(last_in[vt.pix_base[v] + pix], n_items);
        }
        B0 = T * bg0; B1 = T * bg1; B2 = T * bg2;
    } else {
        // recompute the forward transmittance and the last composited position
        bool done = !tc.inside;
        for (uint32_t b0 = it.s0; b0 < it.s1; b0 += kRT) {
            if (__syncthreads_count(done) == kRT) break;
            stage(S, rec, vals, b0 + threadIdx.x, b0 + threadIdx.x < it.s1, cap_cand, st, 52, false);
            __syncthreads();
            const int n = (int)min((uint32_t)kRT, it.s1 - b0);
            if (!done) {
                for (int j = 0; j < n; ++j) {
                    const float4 a = S.a[j];
                    const float4 bb = S.b[j];
                    float dx, dy;
                    const float power = splat_power(a, bb.x, fpx, fpy, &dx, &dy);
                    if (power > 0.f) continue;
                    const float alpha = fminf(kAlphaMax, __fmul_rn(bb.y, splat_gauss(power)));
                    if (alpha < kAlphaMin) continue;
                    const float Tn = __fmul_rn(T, 1.f - alpha);
                    if (Tn < kTMin) { done = true; break; }
                    T = Tn;
                    lastc = (int)(b0 - it.s0) + j + 1;
                }
            }
        }
        B0 = T * bg0; B1 = T * bg1; B2 = T * bg2;
    }
    __syncthreads();
    atomicMax(&s_maxlast, lastc);
    float g0 = 0.f, g1 = 0.f, g2 = 0.f;
    if (tc.inside) {
        const float *dimg = d_image + 3 * vt.pix_base[v];
        g0 = dimg[pix]; g1 = dimg[W * H + pix]; g2 = dimg[2 * W * H + pix];
    }
    __syncthreads();
    const int maxlast = min(s_maxlast, n_items);
    const int lane = threadIdx.x & 31;
    // back to front over chunk positions [0, maxlast)
    for (int hi = maxlast; hi > 0; hi -= kRT) {
        const int lo = max(0, hi - kRT);
        __syncthreads();
        {
            const int p = hi - 1 - (int)threadIdx.x;   // smem slot j <-> position hi-1-j
            stage(S, rec, vals, it.s0 + (uint32_t)max(p, 0), p >= lo, cap_cand, st, 53, true);
        }
        __syncthreads();
        const int n = hi - lo;
        for (int j = 0; j < n; ++j) {
            const int p = hi - 1 - j;
            float gmx = 0.f, gmy = 0.f, gca = 0.f, gcb = 0.f, gcc = 0.f, gop = 0.f, gr = 0.f, gg = 0.f, gb = 0.f;
            bool contrib = false;
            if (p < lastc) {
                const float4 a = S.a[j];
                const float4 bb = S.b[j];
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
                        const float cr = bb.z, cg = bb.w, cbl = S.c[j];
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
                    float *o = sgrad + 9 * (size_t)S.id[j];
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

// ------------------------------------------------------------ launcher
int launch_render_bwd(const gs_gauss3d *g, const gs_camera *cams, const gs_splats *sp, const gs_bins *bins,
                      const ViewTable &vt, const float bg[3], int L, void *ws, const float *d_image,
                      const float *T_final, const int32_t *last, gs_splat_grad *sgrad, gs_gauss3d_grad *out,
                      gs_status *st, cudaStream_t s)
{
    const long long cap_cand = g->cap_rows * (long long)g->k;
    cudaMemsetAsync(sgrad->g, 0, sizeof(float) * 9 * (size_t)cap_cand, s);
    const float4 *rec = reinterpret_cast<const float4 *>(sp->rec);
    if (vt.total_tiles > 0) {
        const RenderPlan plan = render_plan(vt, bins->cap_pairs, L, ws);
        render_bwd_kernel<<<plan.max_items, kRT, 0, s>>>(rec, bins->vals, bins->ranges, vt, plan, bg[0], bg[1],
                                                          bg[2], d_image, T_final, last, sgrad->g,
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
