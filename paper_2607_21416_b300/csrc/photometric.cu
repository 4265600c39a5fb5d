// photometric.cu -- the full photometric objective of Eq. 3 over a batch of
// views: L = lambda L1 + (1 - lambda) L_SSIM, L_SSIM = 1 - SSIM, and dL/dimage.
//
// SSIM as in the 3DGS objective the paper cites for Eq. 3: per view and
// channel, 11x11 Gaussian window (sigma 1.5, normalised), zero padding outside
// the image, C1 = 0.01^2, C2 = 0.03^2; each term is the per-view mean over
// pixels and channels, summed over the views.
//
// One fused pass.  A warp owns a work unit: 32 output columns (one per lane)
// by 64 output rows of one (view, channel), and slides down it one input row
// at a time, keeping in shared memory the last 11 input rows (52 columns: the
// strip and two window radii each side), so every image value is read from
// HBM about once (52/32 columns, 84/64 rows, plus L2 hits).  For each input
// row r it
//   1. sums the window down the columns (moments x, y, x^2, y^2, x y) and
//      then along the row, giving mu_x, mu_y, s_xx, s_yy, s_xy of moment row
//      r - 5 at 42 columns (the strip and one radius each side);
//   2. forms there the SSIM value S and its partials dS/dmu_x, dS/ds_xx,
//      dS/ds_xy, scaled by -(1 - lambda) / (3 H W) and zero outside the image
//      (the adjoint of the zero-padded window sum is the same window sum,
//      since the window is symmetric);
//   3. windows the partials along the row (32 columns) into a second 11-row
//      ring, and down the columns for output row r - 10:
//        dL/dx = lambda sign(x - y) / (3 H W) + W*P_mu + 2 x W*P_xx + y W*P_xy.
// Each unit adds its sums of S and |x - y| into one partial; a one-block
// finalize step sums them per view in double and writes the loss.
#include <cmath>

#include "gs_internal.cuh"

namespace gs {

constexpr int kSR = 5;                  // window radius (11 taps)
constexpr int kRing = 2 * kSR + 1;      // rows kept
constexpr int kSW = 32;                 // output columns per unit (one per lane)
constexpr int kSegRows = 64;            // output rows per unit
constexpr int kIn = kSW + 4 * kSR;      // input columns kept (52)
constexpr int kMo = kSW + 2 * kSR;      // moment / partial columns (42)
constexpr int kSsimWarps = 4;           // units per CTA
constexpr float kC1 = 0.01f * 0.01f, kC2 = 0.03f * 0.03f;

struct SsimTaps {
    float g[kRing];
};

static SsimTaps ssim_taps()
{
    double g[kRing], s = 0;
    for (int i = -kSR; i <= kSR; ++i) {
        g[i + kSR] = std::exp(-(double)(i * i) / (2.0 * 1.5 * 1.5));
        s += g[i + kSR];
    }
    SsimTaps t;
    for (int i = 0; i < kRing; ++i) t.g[i] = (float)(g[i] / s);
    return t;
}

// Work units: per view, 3 channels x row segments x column strips.
struct SsimPlan {
    int V, units;
    int strips[GS_MAX_VIEWS], segs[GS_MAX_VIEWS];
    int unit_base[GS_MAX_VIEWS + 1];
};

static SsimPlan ssim_plan(const ViewTable &vt)
{
    SsimPlan p;
    p.V = vt.V;
    int u = 0;
    for (int v = 0; v < vt.V; ++v) {
        p.strips[v] = (vt.W[v] + kSW - 1) / kSW;
        p.segs[v] = (vt.H[v] + kSegRows - 1) / kSegRows;
        p.unit_base[v] = u;
        u += 3 * p.strips[v] * p.segs[v];
    }
    p.unit_base[vt.V] = u;
    p.units = u;
    return p;
}

struct SsimWarpSmem {
    float rx[kRing][kIn], ry[kRing][kIn];   // input rows ri - 10 .. ri (ring by row)
    float vm[5][kIn];                        // column sums of the five moments, moment row ri - 5
    float pm[3][kMo];                        // scaled partials of moment row ri - 5
    float rc[kRing][3][kSW];                 // partials windowed along rows (ring by row)
};

__device__ __forceinline__ int ring_of(int r) { return (r + 8 * kRing) % kRing; }   // r >= -2 kSR

__global__ void __launch_bounds__(32 * kSsimWarps) ssim_kernel(const float *__restrict__ image,
                                                               const float *__restrict__ target, ViewTable vt,
                                                               SsimPlan plan, SsimTaps taps, float lam,
                                                               float *__restrict__ d_image,
                                                               float2 *__restrict__ partial)
{
    __shared__ SsimWarpSmem sm_all[kSsimWarps];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int u = blockIdx.x * kSsimWarps + warp;
    if (u >= plan.units) return;   // warp-uniform; the kernel has no block barrier
    SsimWarpSmem &sm = sm_all[warp];
    int v = 0;
    while (v + 1 < plan.V && plan.unit_base[v + 1] <= u) ++v;
    const int local = u - plan.unit_base[v];
    const int per_ch = plan.strips[v] * plan.segs[v];
    const int ch = local / per_ch, rem = local - ch * per_ch;
    const int seg = rem / plan.strips[v], strip = rem - seg * plan.strips[v];
    const int W = vt.W[v], H = vt.H[v];
    const int x0 = strip * kSW, r0 = seg * kSegRows, r1 = min(H, r0 + kSegRows);
    const long long plane = 3 * vt.pix_base[v] + (long long)ch * W * H;
    const float *X = image + plane, *Y = target + plane;
    const float inv_n = 1.f / (3.f * (float)W * (float)H);
    const float wv = -(1.f - lam) * inv_n, wl = lam * inv_n;
    const int ci0 = x0 - 2 * kSR + lane, ci1 = ci0 + 32;   // this lane's input columns
    const bool has1 = lane < kIn - 32;
    auto load_row = [&](int r, float &a0, float &b0, float &a1, float &b1) {
        a0 = b0 = a1 = b1 = 0.f;
        if (r >= 0 && r < H) {
            const long long base = (long long)r * W;
            if (ci0 >= 0 && ci0 < W) { a0 = __ldg(X + base + ci0); b0 = __ldg(Y + base + ci0); }
            if (has1 && ci1 >= 0 && ci1 < W) { a1 = __ldg(X + base + ci1); b1 = __ldg(Y + base + ci1); }
        }
    };
    float ca0, cb0, ca1, cb1, na0, nb0, na1, nb1;   // rows ri and ri + 1, loaded ahead
    load_row(r0 - 2 * kSR, ca0, cb0, ca1, cb1);
    load_row(r0 - 2 * kSR + 1, na0, nb0, na1, nb1);
    float s_sum = 0.f, l1_sum = 0.f;
    const int steps = (r1 - r0) + 4 * kSR;
    for (int i = 0; i < steps; ++i) {
        const int ri = r0 - 2 * kSR + i;
        float fa0, fb0, fa1, fb1;
        load_row(ri + 2, fa0, fb0, fa1, fb1);
        {
            const int sl = ring_of(ri);
            sm.rx[sl][lane] = ca0;
            sm.ry[sl][lane] = cb0;
            if (has1) { sm.rx[sl][lane + 32] = ca1; sm.ry[sl][lane + 32] = cb1; }
        }
        __syncwarp();
        if (i >= 2 * kSR) {
            const int rm = ri - kSR;   // moment row
            // 1a. column sums of the moments over input rows rm - 5 .. rm + 5
#pragma unroll
            for (int slot = 0; slot < 2; ++slot) {
                const int c = lane + 32 * slot;
                if (slot == 1 && !has1) break;
                float m0 = 0.f, m1 = 0.f, m2 = 0.f, m3 = 0.f, m4 = 0.f;
#pragma unroll
                for (int k = 0; k < kRing; ++k) {
                    const int sl = ring_of(rm - kSR + k);
                    const float a = sm.rx[sl][c], b = sm.ry[sl][c], w = taps.g[k];
                    const float wa = w * a, wb = w * b;
                    m0 += wa;
                    m1 += wb;
                    m2 = fmaf(wa, a, m2);
                    m3 = fmaf(wb, b, m3);
                    m4 = fmaf(wa, b, m4);
                }
                sm.vm[0][c] = m0; sm.vm[1][c] = m1; sm.vm[2][c] = m2; sm.vm[3][c] = m3; sm.vm[4][c] = m4;
            }
            __syncwarp();
            // 1b + 2. row sums -> moments at 42 columns; S and the scaled partials
#pragma unroll
            for (int slot = 0; slot < 2; ++slot) {
                const int j = lane + 32 * slot;
                if (slot == 1 && j >= kMo) break;
                const int gc = x0 - kSR + j;
                float p0 = 0.f, p1 = 0.f, p2 = 0.f;
                if (rm >= 0 && rm < H && gc >= 0 && gc < W) {
                    float mx = 0.f, my = 0.f, sxx = 0.f, syy = 0.f, sxy = 0.f;
#pragma unroll
                    for (int k = 0; k < kRing; ++k) {
                        const float w = taps.g[k];
                        mx = fmaf(w, sm.vm[0][j + k], mx);
                        my = fmaf(w, sm.vm[1][j + k], my);
                        sxx = fmaf(w, sm.vm[2][j + k], sxx);
                        syy = fmaf(w, sm.vm[3][j + k], syy);
                        sxy = fmaf(w, sm.vm[4][j + k], sxy);
                    }
                    const float vx = sxx - mx * mx, vy = syy - my * my, cv = sxy - mx * my;
                    const float A1 = 2.f * mx * my + kC1, A2 = 2.f * cv + kC2;
                    const float B1 = mx * mx + my * my + kC1, B2 = vx + vy + kC2;
                    const float iB1 = 1.f / B1, iB2 = 1.f / B2, iB12 = iB1 * iB2;
                    const float S = A1 * A2 * iB12;
                    p0 = wv * (2.f * my * A2 * iB12 - 2.f * mx * S * iB1 + 2.f * mx * S * iB2 - 2.f * my * A1 * iB12);
                    p1 = wv * (-S * iB2);
                    p2 = wv * (2.f * A1 * iB12);
                    if (rm >= r0 && rm < r1 && j >= kSR && j < kSR + kSW) {   // this unit's own pixel
                        const int sl = ring_of(rm);
                        s_sum += S;
                        l1_sum += fabsf(sm.rx[sl][j + kSR] - sm.ry[sl][j + kSR]);
                    }
                }
                sm.pm[0][j] = p0; sm.pm[1][j] = p1; sm.pm[2][j] = p2;
            }
            __syncwarp();
            // 3a. partials windowed along the row, output column x0 + lane
            {
                float h0 = 0.f, h1 = 0.f, h2 = 0.f;
#pragma unroll
                for (int k = 0; k < kRing; ++k) {
                    const float w = taps.g[k];
                    h0 = fmaf(w, sm.pm[0][lane + k], h0);
                    h1 = fmaf(w, sm.pm[1][lane + k], h1);
                    h2 = fmaf(w, sm.pm[2][lane + k], h2);
                }
                const int sl = ring_of(rm);
                sm.rc[sl][0][lane] = h0; sm.rc[sl][1][lane] = h1; sm.rc[sl][2][lane] = h2;
            }
            __syncwarp();
            // 3b. down the columns for output row rm - 5, and the gradient
            if (i >= 4 * kSR) {
                const int ro = rm - kSR;
                float b0 = 0.f, b1 = 0.f, b2 = 0.f;
#pragma unroll
                for (int k = 0; k < kRing; ++k) {
                    const int sl = ring_of(ro - kSR + k);
                    const float w = taps.g[k];
                    b0 = fmaf(w, sm.rc[sl][0][lane], b0);
                    b1 = fmaf(w, sm.rc[sl][1][lane], b1);
                    b2 = fmaf(w, sm.rc[sl][2][lane], b2);
                }
                const int gc = x0 + lane;
                if (gc < W) {
                    const int sl = ring_of(ro);
                    const float x = sm.rx[sl][lane + 2 * kSR], y = sm.ry[sl][lane + 2 * kSR];
                    const float d = x - y;
                    const float sgn = d > 0.f ? 1.f : (d < 0.f ? -1.f : 0.f);
                    d_image[plane + (long long)ro * W + gc] = fmaf(wl, sgn, b0 + 2.f * x * b1 + y * b2);
                }
            }
        }
        __syncwarp();   // the next row overwrites the oldest ring slot
        ca0 = na0; cb0 = nb0; ca1 = na1; cb1 = nb1;
        na0 = fa0; nb0 = fb0; na1 = fa1; nb1 = fb1;
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        s_sum += __shfl_xor_sync(0xffffffffu, s_sum, off);
        l1_sum += __shfl_xor_sync(0xffffffffu, l1_sum, off);
    }
    if (lane == 0) partial[u] = make_float2(s_sum, l1_sum);
}

// One block: per view, the sums of S and |x - y| over its units (double),
// then loss[0] = lambda L1 + (1 - lambda) L_SSIM, loss[1] = L1, loss[2] = L_SSIM.
__global__ void __launch_bounds__(1024) photometric_finalize(const float2 *__restrict__ partial, ViewTable vt,
                                                             SsimPlan plan, float lam, float *__restrict__ loss)
{
    __shared__ double s_a[32], s_b[32];
    double L1 = 0.0, Ls = 0.0;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int v = 0; v < vt.V; ++v) {
        double a = 0.0, b = 0.0;
        for (int i = plan.unit_base[v] + threadIdx.x; i < plan.unit_base[v + 1]; i += blockDim.x) {
            const float2 p = partial[i];
            a += p.x;
            b += p.y;
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            a += __shfl_xor_sync(0xffffffffu, a, off);
            b += __shfl_xor_sync(0xffffffffu, b, off);
        }
        if (lane == 0) { s_a[warp] = a; s_b[warp] = b; }
        __syncthreads();
        if (threadIdx.x == 0) {
            double sa = 0.0, sb = 0.0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { sa += s_a[w]; sb += s_b[w]; }
            const double n = 3.0 * (double)vt.W[v] * (double)vt.H[v];
            Ls += 1.0 - sa / n;
            L1 += sb / n;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        loss[0] = (float)((double)lam * L1 + (1.0 - (double)lam) * Ls);
        loss[1] = (float)L1;
        loss[2] = (float)Ls;
    }
}

size_t photometric_workspace_bytes(const ViewTable &vt)
{
    return align_up(sizeof(float2) * (size_t)std::max(1, ssim_plan(vt).units), 256);
}

int launch_photometric(const float *image, const float *target, const ViewTable &vt, float lam, void *ws,
                       float *loss, float *d_image, cudaStream_t s)
{
    const SsimPlan plan = ssim_plan(vt);
    float2 *partial = reinterpret_cast<float2 *>(ws);
    const SsimTaps taps = ssim_taps();
    const int grid = (plan.units + kSsimWarps - 1) / kSsimWarps;
    ssim_kernel<<<grid, 32 * kSsimWarps, 0, s>>>(image, target, vt, plan, taps, lam, d_image, partial);
    photometric_finalize<<<1, 1024, 0, s>>>(partial, vt, plan, lam, loss);
    count_launches(2);
    return cudaPeekAtLastError() == cudaSuccess ? GS_OK : GS_ERR_CUDA;
}

}  // namespace gs
