// photometric.cu -- the full photometric objective of Eq. 3 over a batch of
// views: L = lambda L1 + (1 - lambda) L_SSIM, L_SSIM = 1 - SSIM, and dL/dimage.
//
// SSIM as in the 3DGS objective the paper cites for Eq. 3: per view and
// channel, 11x11 Gaussian window (sigma 1.5, normalised), zero padding outside
// the image, C1 = 0.01^2, C2 = 0.03^2; each term is the per-view mean over
// pixels and channels, summed over the views.
//
// Two passes over 16x16 pixel tiles, one CTA per (tile, channel), each with
// its 26x26 neighbourhood staged in shared memory and the window applied as
// two 11-tap passes (rows, then columns):
//   ssim_fwd_kernel  windowed moments mu_x, mu_y, s_xx, s_yy, s_xy of the
//                    tile; per pixel the SSIM value S and the three partials
//                    dS/dmu_x, dS/ds_xx, dS/ds_xy (already scaled by
//                    -(1 - lambda) / (3 H W)), written to the workspace; the
//                    tile's sums of S and |x - y| as one partial per CTA;
//   ssim_bwd_kernel  the same window applied to the three partial maps (the
//                    window is symmetric, so the adjoint of the zero-padded
//                    window sum is the window sum itself, restricted to the
//                    image): dL/dx = lambda sign(x - y) / (3 H W) + W*P_mu +
//                    2 x W*P_xx + y W*P_xy;
//   photometric_finalize  per-view sums of the partials in double, the loss.
#include <cmath>

#include "gs_internal.cuh"

namespace gs {

constexpr int kSR = 5;                      // window radius (11 taps)
constexpr int kSReg = kTile + 2 * kSR;      // staged neighbourhood side (26)
constexpr float kC1 = 0.01f * 0.01f, kC2 = 0.03f * 0.03f;

struct SsimTaps {
    float g[2 * kSR + 1];
};

static SsimTaps ssim_taps()
{
    double g[2 * kSR + 1], s = 0;
    for (int i = -kSR; i <= kSR; ++i) {
        g[i + kSR] = std::exp(-(double)(i * i) / (2.0 * 1.5 * 1.5));
        s += g[i + kSR];
    }
    SsimTaps t;
    for (int i = 0; i < 2 * kSR + 1; ++i) t.g[i] = (float)(g[i] / s);
    return t;
}

struct TileOf {
    int v, x0, y0, W, H;
    long long plane;   // offset of the view's channel plane in the batch image
};
__device__ __forceinline__ TileOf tile_of(const ViewTable &vt, int t, int ch)
{
    TileOf o;
    o.v = view_of_tile(vt, t);
    const int local = t - vt.tile_base[o.v];
    o.W = vt.W[o.v];
    o.H = vt.H[o.v];
    o.x0 = (local % vt.TX[o.v]) * kTile;
    o.y0 = (local / vt.TX[o.v]) * kTile;
    o.plane = 3 * vt.pix_base[o.v] + (long long)ch * o.W * o.H;
    return o;
}

__global__ void __launch_bounds__(kTile *kTile) ssim_fwd_kernel(const float *__restrict__ image,
                                                                const float *__restrict__ target, ViewTable vt,
                                                                SsimTaps taps, float lam, float *__restrict__ maps,
                                                                float2 *__restrict__ partial)
{
    __shared__ float sx[kSReg][kSReg + 1], sy[kSReg][kSReg + 1];
    __shared__ float hm[5][kSReg][kTile + 1];
    __shared__ float s_red[2][kTile * kTile / 32];
    const int t = blockIdx.x, ch = blockIdx.y;
    const TileOf o = tile_of(vt, t, ch);
    const float *X = image + o.plane, *Y = target + o.plane;
    for (int i = threadIdx.x; i < kSReg * kSReg; i += blockDim.x) {
        const int ry = i / kSReg, rx = i - ry * kSReg;
        const int gx = o.x0 - kSR + rx, gy = o.y0 - kSR + ry;
        float a = 0.f, b = 0.f;
        if (gx >= 0 && gx < o.W && gy >= 0 && gy < o.H) {
            a = X[(long long)gy * o.W + gx];
            b = Y[(long long)gy * o.W + gx];
        }
        sx[ry][rx] = a;
        sy[ry][rx] = b;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kSReg * kTile; i += blockDim.x) {   // along rows
        const int ry = i / kTile, c = i - ry * kTile;
        float m0 = 0.f, m1 = 0.f, m2 = 0.f, m3 = 0.f, m4 = 0.f;
#pragma unroll
        for (int k = 0; k < 2 * kSR + 1; ++k) {
            const float a = sx[ry][c + k], b = sy[ry][c + k], w = taps.g[k];
            const float wa = w * a, wb = w * b;
            m0 += wa;
            m1 += wb;
            m2 = fmaf(wa, a, m2);
            m3 = fmaf(wb, b, m3);
            m4 = fmaf(wa, b, m4);
        }
        hm[0][ry][c] = m0; hm[1][ry][c] = m1; hm[2][ry][c] = m2; hm[3][ry][c] = m3; hm[4][ry][c] = m4;
    }
    __syncthreads();
    const int ty = threadIdx.x / kTile, tx = threadIdx.x - ty * kTile;
    float mx = 0.f, my = 0.f, sxx = 0.f, syy = 0.f, sxy = 0.f;   // along columns
#pragma unroll
    for (int k = 0; k < 2 * kSR + 1; ++k) {
        const float w = taps.g[k];
        mx = fmaf(w, hm[0][ty + k][tx], mx);
        my = fmaf(w, hm[1][ty + k][tx], my);
        sxx = fmaf(w, hm[2][ty + k][tx], sxx);
        syy = fmaf(w, hm[3][ty + k][tx], syy);
        sxy = fmaf(w, hm[4][ty + k][tx], sxy);
    }
    const int px = o.x0 + tx, py = o.y0 + ty;
    const bool in = px < o.W && py < o.H;
    float S = 0.f, l1 = 0.f;
    if (in) {
        const float vx = sxx - mx * mx, vy = syy - my * my, cv = sxy - mx * my;
        const float A1 = 2.f * mx * my + kC1, A2 = 2.f * cv + kC2;
        const float B1 = mx * mx + my * my + kC1, B2 = vx + vy + kC2;
        const float iB1 = 1.f / B1, iB2 = 1.f / B2, iB12 = iB1 * iB2;
        S = A1 * A2 * iB12;
        const float wv = -(1.f - lam) / (3.f * (float)o.W * (float)o.H);
        const float d_mu = 2.f * my * A2 * iB12 - 2.f * mx * S * iB1 + 2.f * mx * S * iB2 - 2.f * my * A1 * iB12;
        const long long n3 = 3 * vt.total_pixels, at = o.plane + (long long)py * o.W + px;
        maps[at] = wv * d_mu;
        maps[n3 + at] = wv * (-S * iB2);
        maps[2 * n3 + at] = wv * (2.f * A1 * iB12);
        l1 = fabsf(sx[ty + kSR][tx + kSR] - sy[ty + kSR][tx + kSR]);
    }
    // tile sums (one partial per CTA, summed per view in double by the finalize step)
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        S += __shfl_xor_sync(0xffffffffu, S, off);
        l1 += __shfl_xor_sync(0xffffffffu, l1, off);
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) { s_red[0][warp] = S; s_red[1][warp] = l1; }
    __syncthreads();
    if (threadIdx.x == 0) {
        float a = 0.f, b = 0.f;
        for (int w = 0; w < kTile * kTile / 32; ++w) { a += s_red[0][w]; b += s_red[1][w]; }
        partial[(long long)ch * vt.total_tiles + t] = make_float2(a, b);
    }
}

__global__ void __launch_bounds__(kTile *kTile) ssim_bwd_kernel(const float *__restrict__ image,
                                                                const float *__restrict__ target, ViewTable vt,
                                                                SsimTaps taps, float lam,
                                                                const float *__restrict__ maps,
                                                                float *__restrict__ d_image)
{
    __shared__ float sm[3][kSReg][kSReg + 1];
    __shared__ float hb[3][kSReg][kTile + 1];
    const int t = blockIdx.x, ch = blockIdx.y;
    const TileOf o = tile_of(vt, t, ch);
    const long long n3 = 3 * vt.total_pixels;
    for (int i = threadIdx.x; i < kSReg * kSReg; i += blockDim.x) {
        const int ry = i / kSReg, rx = i - ry * kSReg;
        const int gx = o.x0 - kSR + rx, gy = o.y0 - kSR + ry;
        float a = 0.f, b = 0.f, c = 0.f;   // the partial maps are zero outside the image
        if (gx >= 0 && gx < o.W && gy >= 0 && gy < o.H) {
            const long long at = o.plane + (long long)gy * o.W + gx;
            a = maps[at];
            b = maps[n3 + at];
            c = maps[2 * n3 + at];
        }
        sm[0][ry][rx] = a;
        sm[1][ry][rx] = b;
        sm[2][ry][rx] = c;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kSReg * kTile; i += blockDim.x) {
        const int ry = i / kTile, c = i - ry * kTile;
        float m0 = 0.f, m1 = 0.f, m2 = 0.f;
#pragma unroll
        for (int k = 0; k < 2 * kSR + 1; ++k) {
            const float w = taps.g[k];
            m0 = fmaf(w, sm[0][ry][c + k], m0);
            m1 = fmaf(w, sm[1][ry][c + k], m1);
            m2 = fmaf(w, sm[2][ry][c + k], m2);
        }
        hb[0][ry][c] = m0; hb[1][ry][c] = m1; hb[2][ry][c] = m2;
    }
    __syncthreads();
    const int ty = threadIdx.x / kTile, tx = threadIdx.x - ty * kTile;
    const int px = o.x0 + tx, py = o.y0 + ty;
    if (px >= o.W || py >= o.H) return;
    float b0 = 0.f, b1 = 0.f, b2 = 0.f;
#pragma unroll
    for (int k = 0; k < 2 * kSR + 1; ++k) {
        const float w = taps.g[k];
        b0 = fmaf(w, hb[0][ty + k][tx], b0);
        b1 = fmaf(w, hb[1][ty + k][tx], b1);
        b2 = fmaf(w, hb[2][ty + k][tx], b2);
    }
    const long long at = o.plane + (long long)py * o.W + px;
    const float x = image[at], y = target[at];
    const float d = x - y;
    const float sgn = d > 0.f ? 1.f : (d < 0.f ? -1.f : 0.f);
    d_image[at] = lam * sgn / (3.f * (float)o.W * (float)o.H) + b0 + 2.f * x * b1 + y * b2;
}

// One block: per view, the sums of S and |x - y| over its tiles and channels
// (double), then loss[0] = lambda L1 + (1 - lambda) L_SSIM, loss[1] = L1,
// loss[2] = L_SSIM.
__global__ void __launch_bounds__(1024) photometric_finalize(const float2 *__restrict__ partial, ViewTable vt,
                                                             float lam, float *__restrict__ loss)
{
    __shared__ double s_a[32], s_b[32];
    double L1 = 0.0, Ls = 0.0;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int v = 0; v < vt.V; ++v) {
        const int t0 = vt.tile_base[v], t1 = vt.tile_base[v + 1], nt = t1 - t0;
        double a = 0.0, b = 0.0;
        for (int i = threadIdx.x; i < 3 * nt; i += blockDim.x) {
            const int ch = i / nt, t = t0 + (i - ch * nt);
            const float2 p = partial[(long long)ch * vt.total_tiles + t];
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

struct PhotoLayout {
    size_t maps, partial, total;
};
static PhotoLayout photo_layout(const ViewTable &vt)
{
    PhotoLayout L;
    size_t o = 0;
    auto take = [&](size_t bytes) { size_t at = o; o = align_up(o + bytes, 256); return at; };
    L.maps = take(sizeof(float) * 9 * (size_t)vt.total_pixels);
    L.partial = take(sizeof(float2) * 3 * (size_t)vt.total_tiles);
    L.total = o;
    return L;
}

size_t photometric_workspace_bytes(const ViewTable &vt) { return photo_layout(vt).total; }

int launch_photometric(const float *image, const float *target, const ViewTable &vt, float lam, void *ws,
                       float *loss, float *d_image, cudaStream_t s)
{
    const PhotoLayout L = photo_layout(vt);
    char *w = reinterpret_cast<char *>(ws);
    float *maps = reinterpret_cast<float *>(w + L.maps);
    float2 *partial = reinterpret_cast<float2 *>(w + L.partial);
    const SsimTaps taps = ssim_taps();
    const dim3 grid((unsigned)vt.total_tiles, 3);
    ssim_fwd_kernel<<<grid, kTile * kTile, 0, s>>>(image, target, vt, taps, lam, maps, partial);
    ssim_bwd_kernel<<<grid, kTile * kTile, 0, s>>>(image, target, vt, taps, lam, maps, d_image);
    photometric_finalize<<<1, 1024, 0, s>>>(partial, vt, lam, loss);
    count_launches(3);
    return cudaPeekAtLastError() == cudaSuccess ? GS_OK : GS_ERR_CUDA;
}

}  // namespace gs
