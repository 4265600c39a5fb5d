// render_common.cuh -- shared pieces of the tile compositing kernels.
//
// Work decomposition.  Each 16x16 tile's sorted splat list [start, end) is
// cut into chunks of at most L splats; chunk k of tile t is one work item,
// and each of its four 16x4 pixel blocks is a work unit that one warp of a
// persistent kernel takes from a device counter (two pixels per lane,
// lane_pixels).  item_base[t] (exclusive scan of the per-tile chunk counts,
// built on the device) numbers the items; the item of unit u is found by
// binary search.  A tile with one chunk is composited directly.  Chunk 0 of a multi-chunk tile is composited exactly (it starts
// at T = 1); every later chunk is composited with its own transmittance
// starting at 1 and no stop rule, and the combine step scales it by the
// transmittance in front of it.  That is Eq. 1 exactly unless a pixel's stop
// (T' < 1e-4) falls inside the chunk; those (chunk, pixel) pairs are
// composited again from the now known entering transmittance (fix-up).
// After the forward, each item k of a multi-chunk tile holds per pixel:
//   T0     transmittance in front of the chunk: the running product of the
//          chunks' own products; the chunk is active iff T0 >= 1e-4 (0 for
//          the chunks behind the pixel's stop)
//   Tend   transmittance after the chunk's compositing (stop rule applied)
//   P[3]   colour composited up to and including this chunk (prefix)
//   last   1-based position (in the chunk) of its last composited splat
// so the reverse pass of chunk k starts from Tend, last and the colour behind
// the chunk, F - P_k (F the pixel's final colour, the forward's image), in
// O(1).
#pragma once

#include "gs_internal.cuh"

namespace gs {

constexpr int kRT = kTilePix;      // pixels per tile / work item
constexpr int kRThreads = 128;     // threads per CTA of the compositing kernels (4 warps, one 16x4 block each)
constexpr int kStateWords = 7;     // T0 (Tprod during the forward), Tend, P0..2 (C during the forward), last,
                                   // composited count (x 256 pixels)

// 2^x on the special-function unit (ex2.approx, max relative error ~2^-22).
__device__ __forceinline__ float ex2_approx(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// power * log2(e) of a splat record (a = mean x, mean y, A, B; C) at pixel
// (px, py): (A dx + B dy) dx + C dy^2 with (dx, dy) = mean - pixel.  Explicit
// rounding so that every pass that re-evaluates a pair decides identically.
__device__ __forceinline__ float splat_q(float4 a, float C, float px, float py, float *dx, float *dy)
{
    const float x = __fsub_rn(a.x, px), y = __fsub_rn(a.y, py);
    *dx = x; *dy = y;
    const float t = fmaf(a.z, x, __fmul_rn(a.w, y));
    return fmaf(t, x, __fmul_rn(__fmul_rn(C, y), y));
}

// Unclamped alpha o exp(power) = 2^(q + L).
__device__ __forceinline__ float splat_alpha(float q, float L) { return ex2_approx(__fadd_rn(q, L)); }

// Tile coordinates of tile t (view, origin), and for the combine step, where
// tile thread `tid` (0..127) owns pixels (px, py) and (px, py + 1): px = x0 +
// (tid & 15), py = y0 + 2 (tid >> 4), tile-local pixel ids pid0 = (py - y0)
// 16 + (px - x0) and pid0 + 16.  The persistent compositing kernels use only
// the view and origin: their warp w plays the 16x4 block of rows 4w..4w+3 of
// its work unit's item, its lanes taking pixels as lane_pixels says.
struct TileCoord {
    int v, x0, y0, px, py, pid0;
    bool in0, in1;
};
__device__ __forceinline__ TileCoord tile_coord(const ViewTable &vt, int t, int tid)
{
    TileCoord c;
    c.v = view_of_tile(vt, t);
    const int local = t - vt.tile_base[c.v];
    const int tx = local % vt.TX[c.v], ty = local / vt.TX[c.v];
    c.x0 = tx * kTile;
    c.y0 = ty * kTile;
    c.px = c.x0 + (tid & (kTile - 1));
    c.py = c.y0 + 2 * (tid >> 4);
    c.pid0 = 2 * (tid >> 4) * kTile + (tid & (kTile - 1));
    c.in0 = c.px < vt.W[c.v] && c.py < vt.H[c.v];
    c.in1 = c.px < vt.W[c.v] && c.py + 1 < vt.H[c.v];
    return c;
}

// The two pixels a lane composites in its warp's 16x4 block: (x0 + c, y) and
// (x0 + c + 8, y) with c = lane & 7 and y = y0 + 4 w + (lane >> 3).  A splat
// narrower than 9 pixels is composited by at most one pixel of each lane, so
// the two per-pixel steps rarely both run their compositing branch.
struct LanePix {
    int px0, py, pid0;     // first pixel (image coordinates) and its tile-local id; the second is +8
    bool in0, in1;         // inside the image
};
__device__ __forceinline__ LanePix lane_pixels(const TileCoord &tc, int warp, int lane, int W, int H)
{
    LanePix lp;
    const int col = lane & 7, row = 4 * warp + (lane >> 3);
    lp.px0 = tc.x0 + col;
    lp.py = tc.y0 + row;
    lp.pid0 = row * kTile + col;
    lp.in0 = lp.px0 < W && lp.py < H;
    lp.in1 = lp.px0 + 8 < W && lp.py < H;
    return lp;
}

struct Item {
    int t;            // tile
    int k, nk;        // chunk index, chunks of the tile
    int base;         // first item of the tile
    uint32_t start;   // tile list start (positions are counted from here)
    uint32_t s0, s1;  // this chunk's list range
};

// Item b (its tile from the plan's item -> tile table); returns false when b
// is past the last item.
__device__ __forceinline__ bool item_of(int b, const int32_t *__restrict__ item_base,
                                        const int32_t *__restrict__ item_tile, int T,
                                        const uint32_t *__restrict__ ranges, int L, Item *it)
{
    if (b >= __ldg(item_base + T)) return false;
    const int lo = __ldg(item_tile + b);
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

// Per-warp record stage: a warp walks its item's list 32 positions at a
// time; lane l reads position base + l and the warp keeps, in list order,
// the splats whose alpha >= 1/255 region meets its 16x4 block.
struct WarpStage {
    float4 a[32];      // mean x, mean y, A, B
    float4 b[32];      // C, L, r, g
    float c[32];       // b
    uint32_t id[32];   // candidate id
    int pos[32];       // list position within the item (0-based)
    int half[32];      // forward: bit 0 / 1 = the alpha box meets the left / right 8 columns of the block
};

// Whether the alpha >= 1/255 region of a splat record meets the pixel block
// [bx0, bx1] x [by0, by1].  The region {2^(q + L) >= 1/255} is an ellipse
// since q is a negative-definite quadratic form in (dx, dy): with Q = -[[A,
// B/2], [B/2, C]] and s = log2(255) + L > 0 it is d^T Q d <= s, with
// half-extents sqrt(s (Q^-1)_xx), sqrt(s (Q^-1)_yy).  Its bounding box, grown
// by 0.1 % + 0.01 px (far beyond the FP32 error of q, so every pixel outside
// also fails the alpha test as the kernels evaluate it: skipping is exact), is
// tested against the block without a square root: with d the distance from
// the mean to the block along an axis, less 0.01 px, d <= 1.001 sqrt(s
// (Q^-1)_axis) reads d^2 det Q <= 1.002001 s (-C) for x and (-A) for y.
__device__ __forceinline__ bool meets_block(float4 a, float4 b, float bx0, float bx1, float by0, float by1)
{
    const float s = b.y + 7.994353436858858f;   // L + log2(255)
    if (!(s > 0.f)) return false;
    const float det = a.z * b.x - 0.25f * a.w * a.w;
    if (!(det > 0.f)) return true;
    const float dx = fmaxf(fmaxf(bx0 - a.x, a.x - bx1) - 0.01f, 0.f);
    const float dy = fmaxf(fmaxf(by0 - a.y, a.y - by1) - 0.01f, 0.f);
    return dx * dx * det <= 1.002001f * s * (-b.x) && dy * dy * det <= 1.002001f * s * (-a.z);
}

// Reads list position `pos` of the item (when valid) and tests it against the
// warp's block; the hits are compacted into the warp's stage in list order
// (lane order).  Returns the number of hits.
// HALF: also stage which 8-column halves of the block the splat's alpha box
// meets.
template <bool HALF>
__device__ __forceinline__ int warp_stage(WarpStage &W, const float4 *__restrict__ rec,
                                          const uint32_t *__restrict__ vals, uint32_t pos, uint32_t s0, bool valid,
                                          long long cap_cand, const gs_status *st, int site,
                                          float bx0, float bx1, float by0, float by1)
{
    const int lane = threadIdx.x & 31;
    float4 a = make_float4(0.f, 0.f, 0.f, 0.f), b = a;
    uint32_t id = 0;
    bool hit = false;
    if (valid) {
        id = vals[pos];
        if (!idx_ok(st, (long long)id, cap_cand, site)) id = 0;
        a = __ldg(&rec[3 * (size_t)id]);
        b = __ldg(&rec[3 * (size_t)id + 1]);
        hit = meets_block(a, b, bx0, bx1, by0, by1);
    }
    const unsigned m = __ballot_sync(0xffffffffu, hit);
    if (hit) {
        unsigned lt;
        asm("mov.u32 %0, %%lanemask_lt;" : "=r"(lt));
        const int slot = __popc(m & lt);
        W.a[slot] = a;
        W.b[slot] = b;
        W.c[slot] = __ldg(reinterpret_cast<const float *>(&rec[3 * (size_t)id + 2]));
        W.id[slot] = id;
        W.pos[slot] = (int)(pos - s0);
        // which 8-column half of the block the box meets.  A lane's first pixel lies in the left
        // half and its second in the right one (lane_pixels), so a pixel of a half the box misses
        // fails the alpha test as the kernels evaluate it and is skipped (same test as above).
        if (HALF)
            W.half[slot] = (meets_block(a, b, bx0, bx0 + 7.f, by0, by1) ? 1 : 0) |
                           (meets_block(a, b, bx0 + 8.f, bx1, by0, by1) ? 2 : 0);
    }
    __syncwarp();
    (void)lane;
    return __popc(m);
}

// The 16x4 block w of tile coordinates tc: [bx0, bx1] x [by0, by1].
struct BlockRect {
    float x0, x1, y0, y1;
};
__device__ __forceinline__ BlockRect block_rect(const TileCoord &tc, int w)
{
    BlockRect r;
    r.x0 = (float)tc.x0;
    r.x1 = r.x0 + (float)(kTile - 1);
    r.y0 = (float)(tc.y0 + 4 * w);
    r.y1 = r.y0 + 3.f;
    return r;
}

// Next work unit of the calling warp from a device counter (lane 0 takes it).
__device__ __forceinline__ int next_unit(int32_t *counter)
{
    int u = 0;
    if ((threadIdx.x & 31) == 0) u = atomicAdd(counter, 1);
    return __shfl_sync(0xffffffffu, u, 0);
}

struct RenderPlan {
    const int32_t *item_base;   // [T+1]
    int32_t *counters;          // [8] work-unit counters: forward, fix-up, backward, fix count, block lists,
                                //     long multi-chunk tiles, combine, other multi-chunk tiles
    int32_t *fix;               // [max_items] flags: items with pixels to composite again
    int32_t *fix_list;          // [max_items] those items, counters[3] of them
    float *state;               // [max_items][kStateWords][256]
    // Block lists of the items of tiles cut into several chunks: for item i
    // (list positions [s0, s1)) and pixel block w, the positions (relative to
    // s0, ascending) of the splats whose alpha box meets the block, at
    // blist[4 s0 + w (s1 - s0) ...], bcnt[4 i + w] of them.
    uint32_t *blist;            // [4 cap_pairs]
    int32_t *bcnt;              // [max_items][4]
    int32_t *item_tile;         // [max_items] tile of each item
    int32_t *multi_list;        // [T] tiles cut into several chunks: counters[5] long ones from the front,
                                //     counters[7] others from the back
    int L;
    int max_items;
};

RenderPlan render_plan(const ViewTable &vt, long long cap_pairs, int L, void *ws);

// CTAs of 128 threads of a persistent compositing kernel that fit on the
// device at once (registers, shared memory, warps), at most cap_per_sm per
// SM when cap_per_sm > 0, times the SM count.
int persistent_grid(const void *kernel, int cap_per_sm = 0);

}  // namespace gs
