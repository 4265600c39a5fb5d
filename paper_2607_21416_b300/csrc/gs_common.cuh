// gs_common.cuh -- shared device-side definitions of libgs (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "gs.h"

namespace gs {

// Method constants (3DGS rasterizer conventions the paper builds on; see the
// comments on each call in gs.h).
constexpr float kNear = 0.2f;
constexpr float kMargin = 0.15f;
constexpr float kLowpass = 0.3f;
constexpr float kTanClamp = 1.3f;
constexpr float kAlphaMax = 0.99f;
constexpr float kAlphaMin = 1.0f / 255.0f;
constexpr float kTMin = 1e-4f;
constexpr int kTile = GS_TILE;
constexpr int kTilePix = kTile * kTile;

// Per-view layout, passed by value to kernels (resolution is host data).
struct ViewTable {
    int V;
    int total_tiles;
    long long total_pixels;
    int W[GS_MAX_VIEWS];
    int H[GS_MAX_VIEWS];
    int TX[GS_MAX_VIEWS];
    int TY[GS_MAX_VIEWS];
    int tile_base[GS_MAX_VIEWS + 1];
    long long pix_base[GS_MAX_VIEWS + 1];
};

// Builds the table; returns false on invalid resolution / too many views.
bool make_view_table(const gs_view *views, int V, ViewTable *vt);

__device__ __forceinline__ int view_of_tile(const ViewTable &vt, int t)
{
    int lo = 0, hi = vt.V - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (vt.tile_base[mid] <= t) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// View of a row: the last v with view_start[v] <= row (view_start is [V+1]).
__device__ __forceinline__ int view_of_row(const int32_t *__restrict__ view_start, int V, int row)
{
    int lo = 0, hi = V - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (__ldg(view_start + mid) <= row) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Status word helpers.  The first error wins; `needed` keeps the maximum.
__device__ __forceinline__ void set_error(gs_status *st, int code, int where)
{
    if (atomicCAS(&st->code, 0, code) == 0) st->where = where;
}
__device__ __forceinline__ void set_needed(gs_status *st, long long n)
{
    atomicMax(reinterpret_cast<unsigned long long *>(&st->needed), (unsigned long long)n);
}
// Defensive index check: records GS_ERR_INVALID_ARG with the site id and the
// offending index in the status word and tells the caller to skip the access.
__device__ __forceinline__ bool idx_ok(const gs_status *st, long long idx, long long lim, int site)
{
    if (idx >= 0 && idx < lim) return true;
    gs_status *w = const_cast<gs_status *>(st);
    if (atomicCAS(&w->code, 0, GS_ERR_INVALID_ARG) == 0) {
        w->where = site;
        w->needed = idx;
    }
    return false;
}

__device__ __forceinline__ bool has_error(const gs_status *st)
{
    return *((volatile const int32_t *)&st->code) != 0;
}

// Camera in registers.
struct Cam {
    float fx, fy, cx, cy, R[9], t[3];
};
__device__ __forceinline__ Cam load_cam(const gs_camera *__restrict__ cams, int v)
{
    Cam c;
    const float *p = reinterpret_cast<const float *>(cams + v);
    c.fx = __ldg(p + 0); c.fy = __ldg(p + 1); c.cx = __ldg(p + 2); c.cy = __ldg(p + 3);
#pragma unroll
    for (int i = 0; i < 9; ++i) c.R[i] = __ldg(p + 4 + i);
#pragma unroll
    for (int i = 0; i < 3; ++i) c.t[i] = __ldg(p + 13 + i);
    return c;
}

__device__ __forceinline__ float sigmoidf_(float x) { return 1.0f / (1.0f + expf(-x)); }

// SFU activations of the BF16 decoding path: tanh.approx (max relative error
// about 2^-11, below the BF16 rounding of the MMA inputs) and
// sigmoid(x) = (1 + tanh(x / 2)) / 2.
__device__ __forceinline__ float tanh_fast(float x)
{
    float y;
    asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float sigmoid_fast(float x) { return fmaf(0.5f, tanh_fast(0.5f * x), 0.5f); }

inline int div_up(long long a, long long b) { return (int)((a + b - 1) / b); }

// Number of SMs of the current device (cached per device).
int sm_count();

// Host-side count of kernels this library has launched (gs_kernel_launches).
void count_launches(int n);

// Limit in nanoseconds of the tensor-core kernels' waits for their MMAs
// (gs_set_wait_limit; 1 s unless changed).
constexpr unsigned long long kDefaultWaitNs = 1000000000ull;
unsigned long long wait_limit_ns();

// Launch shapes of gs_set_tuning (0: the library's choice).
gs_tuning tuning();

}  // namespace gs
