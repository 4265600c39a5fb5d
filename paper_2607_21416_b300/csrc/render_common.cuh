// render_common.cuh -- shared pieces of the tile compositing kernels.
//
// Work decomposition.  Each 16x16 tile's sorted splat list [start, end) is
// cut into chunks of at most L splats; chunk k of tile t is one work item and
// one CTA of 256 threads (one thread per pixel).  item_base[t] (exclusive scan
// of the per-tile chunk counts, built on the device) numbers the items; the
// item of block b is found by binary search.  A tile with one chunk is
// composited directly.  A tile with several chunks keeps per-chunk, per-pixel
// state in the render workspace:
//   Tprod  product of (1 - alpha) over the chunk's splats (no stop rule; it
//          may stop early once below 1e-4, which decides every later chunk)
//   Tend   transmittance after the chunk's compositing (stop rule applied)
//   C[3]   the chunk's colour contribution
//   last   1-based position (in the chunk) of its last composited splat
// so that compositing Eq. 1 front to back over the whole list is reproduced
// exactly: chunk k starts from T0_k = prod_{j<k} Tprod_j (it is active iff
// T0_k >= 1e-4, i.e. iff no earlier splat stopped the pixel), and the
// backward pass of chunk k needs only T0_k, its own Tend/last and the colour
// of the chunks behind it.
#pragma once

#include "gs_internal.cuh"

namespace gs {

constexpr int kRT = kTilePix;      // 256 threads per tile / work item
constexpr int kStateWords = 6;     // Tprod, Tend, C0, C1, C2, last  (x 256 pixels)

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

struct Item {
    int t;            // tile
    int k, nk;        // chunk index, chunks of the tile
    int base;         // first item of the tile
    uint32_t start;   // tile list start (positions are counted from here)
    uint32_t s0, s1;  // this chunk's list range
};

// Item of block b; returns false when b is past the last item.
__device__ __forceinline__ bool item_of(int b, const int32_t *__restrict__ item_base, int T,
                                        const uint32_t *__restrict__ ranges, int L, Item *it)
{
    if (b >= __ldg(item_base + T)) return false;
    int lo = 0, hi = T - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(item_base + mid) <= b) lo = mid; else hi = mid - 1;
    }
    it->t = lo;
    it->base = __ldg(item_base + lo);
    it->k = b - it->base;
    it->nk = __ldg(item_base + lo + 1) - it->base;
    const uint32_t start = ranges[2 * lo], end = ranges[2 * lo + 1];
    it->start = start;
    it->s0 = start + (uint32_t)it->k * (uint32_t)L;
    it->s1 = min(end, it->s0 + (uint32_t)L);
    if (it->s0 > it->s1) it->s0 = it->s1;
    return true;
}

// Per-item state planes (only items of multi-chunk tiles use them).
__device__ __forceinline__ float *state_plane(float *state, int item, int plane)
{
    return state + ((size_t)item * kStateWords + plane) * kRT;
}

// Transmittance in front of chunk k: the product of the earlier chunks' Tprod.
__device__ __forceinline__ float chunk_T0(const float *state, const Item &it)
{
    float T = 1.f;
    for (int j = 0; j < it.k; ++j) T = __fmul_rn(T, state_plane(const_cast<float *>(state), it.base + j, 0)[threadIdx.x]);
    return T;
}

// Stage list positions [b0, b0 + n) of vals into shared memory records.
struct Staged {
    float4 a[kRT];    // mean x, mean y, conic a, conic b
    float4 b[kRT];    // conic c, opacity, r, g
    float c[kRT];     // b
    uint32_t id[kRT];
};

__device__ __forceinline__ void stage(Staged &S, const float4 *__restrict__ rec,
                                      const uint32_t *__restrict__ vals, uint32_t pos, bool valid,
                                      long long cap_cand, const gs_status *st, int site, bool with_colour)
{
    if (!valid) return;
    uint32_t id = vals[pos];
    if (!idx_ok(st, (long long)id, cap_cand, site)) id = 0;
    S.id[threadIdx.x] = id;
    S.a[threadIdx.x] = __ldg(&rec[3 * (size_t)id]);
    S.b[threadIdx.x] = __ldg(&rec[3 * (size_t)id + 1]);
    if (with_colour) S.c[threadIdx.x] = __ldg(&rec[3 * (size_t)id + 2]).x;
}

struct RenderPlan {
    const int32_t *item_base;   // [T+1]
    float *state;               // [max_items][6][256]
    int L;
    int max_items;
};

RenderPlan render_plan(const ViewTable &vt, long long cap_pairs, int L, void *ws);

}  // namespace gs
