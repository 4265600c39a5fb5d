// render_bwd.cu -- reverse of the tile compositing (Eq. 1) over chunked work
// items, and the chain rule of the projection.
//
// A tile whose splat list is one work item is reversed front to back, like
// the forward: the traversal recomputes the transmittance in front of each
// splat and the colour composited so far with the forward's own arithmetic
// (so it takes the forward's skip and stop decisions), and gets the colour
// behind a splat as the pixel's final colour (the forward's image) minus that
// prefix -- no per-pixel state is stored by the forward or recomputed in a
// separate pass.  A chunk of a longer list starts from the per-chunk state
// the forward left in the render workspace and is reversed back to front.
// Per-splat sums are reduced across the warp (shuffles) before one global
// atomicAdd per warp and quantity.
#include "proj_bwd.cuh"
#include "render_common.cuh"

namespace gs {

__device__ __forceinline__ float warp_sum(float x)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

// Warp sum of eight values at once (transpose-style halving: 9 shuffles instead
// of 40).  Lane L returns the total of value ((L >> 4) & 1) * 4 + ((L >> 3) & 1)
// * 2 + ((L >> 2) & 1); lanes with (L & 3) == 0 hold the eight totals.
__device__ __forceinline__ float warp_sum8(const float v[8])
{
    const int lane = threadIdx.x & 31;
    float r4[4], r2[2];
    const bool u16 = lane & 16, u8 = lane & 8, u4 = lane & 4;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const float send = u16 ? v[i] : v[i + 4];
        const float keep = u16 ? v[i + 4] : v[i];
        r4[i] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
    }
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const float send = u8 ? r4[i] : r4[i + 2];
        const float keep = u8 ? r4[i + 2] : r4[i];
        r2[i] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
    }
    const float send = u4 ? r2[0] : r2[1];
    float r = (u4 ? r2[1] : r2[0]) + __shfl_xor_sync(0xffffffffu, send, 4);
    r += __shfl_xor_sync(0xffffffffu, r, 2);
    r += __shfl_xor_sync(0xffffffffu, r, 1);
    return r;
}

// Reverse state of one pixel, carried front to back: T the transmittance in
// front of the current splat, Sp = g . (colour composited up to and including
// it), GC = g . (the pixel's final colour, background included) with g =
// dL/dC of the pixel, so that g . B_i = GC - Sp_i is the colour behind splat i.
// lim: last list position (1-based, in the item) the pixel may composite;
// done: nothing left for the pixel in this item.
struct PixBwd {
    float T, Sp, GC, g0, g1, g2;
    int lim;
    bool done;
};

// The alpha decision of Eq. 1 for one pixel (the forward's, operation for
// operation): true iff the splat passes the skip tests at (px, py), with the
// offset and the unclamped alpha o exp(power).
__device__ __forceinline__ bool alpha_test(const float4 a, const float4 bb, float px, float py, float *dx, float *dy,
                                           float *ag)
{
    const float q = splat_q(a, bb.x, px, py, dx, dy);
    if (q > 0.f) return false;
    *ag = splat_alpha(q, bb.y);
    return fminf(kAlphaMax, *ag) >= kAlphaMin;
}

// Gradient terms of one pixel for a splat it composites, added to the
// per-splat sums acc[9] = (m_x, m_y, m_xx, m_xy, m_yy, sum dal exp(power),
// d r, d g, d b) with dp = dL/dpower and the moments m_x = sum dp dx, m_y =
// sum dp dy, m_xx = sum dp dx^2, m_xy = sum dp dx dy, m_yy = sum dp dy^2 over
// the pixels; after the warp reduction they become d mean2d and d conic
// (conic_grads) and the opacity sum is divided by the opacity.  Eq. 1 gives,
// for splat i with transmittance T_i in front of it, dC/dalpha_i = T_i c_i -
// B_i / (1 - alpha_i) (B_i: colour behind i, background included).
//
// Front to back: T = T_i and Sp = g . (colour up to splat i - 1) on entry; g .
// B_i = GC - Sp_i with GC = g . (the pixel's final colour); T and Sp advance
// past the splat (T' = T (1 - alpha) rounded as the forward rounds it).
__device__ __forceinline__ void bwd_composite_f2b(float &T, float &Sp, float GC, float g0, float g1, float g2,
                                                  const float4 bb, float cb, float dx, float dy, float ag, float acc[9])
{
    const float alpha = fminf(kAlphaMax, ag);
    float inv;                             // 1 / (1 - alpha) on the SFU (relative error ~2^-23; the
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(inv) : "f"(1.f - alpha));   // operand lies in [0.01, 1))
    const float w = alpha * T;
    acc[6] = fmaf(w, g0, acc[6]);
    acc[7] = fmaf(w, g1, acc[7]);
    acc[8] = fmaf(w, g2, acc[8]);
    const float gc = fmaf(g0, bb.z, fmaf(g1, bb.w, g2 * cb));
    Sp = fmaf(gc, w, Sp);
    const float dal = fmaf(gc, T, -(GC - Sp) * inv);
    T = __fmul_rn(T, 1.f - alpha);
    if (ag < kAlphaMax) {                  // the clamped branch passes no gradient to o exp(power)
        acc[5] = fmaf(dal, ag, acc[5]);
        const float dp = dal * alpha;      // d power (alpha = o exp(power))
        const float t = dp * dx, u = dp * dy;
        acc[0] += t;
        acc[1] += u;
        acc[2] = fmaf(t, dx, acc[2]);
        acc[3] = fmaf(t, dy, acc[3]);
        acc[4] = fmaf(u, dy, acc[4]);
    }
}

// Back to front: T = T_(i+1) (transmittance behind the splat) and S = g . B_i
// on entry; T becomes T_i = T_(i+1) / (1 - alpha_i) and S takes the splat in.
__device__ __forceinline__ void bwd_composite_b2f(float &T, float &S, float g0, float g1, float g2, const float4 bb,
                                                  float cb, float dx, float dy, float ag, float acc[9])
{
    const float alpha = fminf(kAlphaMax, ag);
    float inv;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(inv) : "f"(1.f - alpha));
    T = T * inv;                           // transmittance in front of this splat
    const float w = alpha * T;
    acc[6] = fmaf(w, g0, acc[6]);
    acc[7] = fmaf(w, g1, acc[7]);
    acc[8] = fmaf(w, g2, acc[8]);
    const float gc = fmaf(g0, bb.z, fmaf(g1, bb.w, g2 * cb));
    const float dal = fmaf(gc, T, -S * inv);
    S = fmaf(gc, w, S);
    if (ag < kAlphaMax) {
        acc[5] = fmaf(dal, ag, acc[5]);
        const float dp = dal * alpha;
        const float t = dp * dx, u = dp * dy;
        acc[0] += t;
        acc[1] += u;
        acc[2] = fmaf(t, dx, acc[2]);
        acc[3] = fmaf(t, dy, acc[3]);
        acc[4] = fmaf(u, dy, acc[4]);
    }
}

// Per-splat gradient from the reduced sums for the calling lane's value index
// vi (warp_sum8 layout; `other` is the total of index vi ^ 1).  power = ln 2
// ((A dx + B dy) dx + C dy^2) with the record's A, B, C, and power = -(c_a
// dx^2 + c_c dy^2) / 2 - c_b dx dy with the conic (c_a, c_b, c_c), so
//   d mean x = ln 2 (2 A m_x + B m_y),  d mean y = ln 2 (2 C m_y + B m_x),
//   d c_a = -m_xx / 2,  d c_b = -m_xy,  d c_c = -m_yy / 2,
// and d opacity = (sum dal exp(power)) / opacity.  The lane's role is fixed,
// so the selection is branch-free: g = cs total + co other.
struct LaneRole {
    bool mx, my, op, mean;
    float k;   // constant factor of the other indices
};
__device__ __forceinline__ LaneRole lane_role(int vi)
{
    LaneRole r;
    r.mx = vi == 0;
    r.my = vi == 1;
    r.op = vi == 5;
    r.mean = vi < 2;
    r.k = (vi == 2 || vi == 4) ? -0.5f : (vi == 3 ? -1.f : 1.f);
    return r;
}
__device__ __forceinline__ float conic_grads(const LaneRole &r, float total, float other, float4 a, float4 bb,
                                             float io)
{
    constexpr float ln2 = 0.6931471805599453f;
    const float cs = r.mx ? (2.f * ln2) * a.z : (r.my ? (2.f * ln2) * bb.x : (r.op ? io : r.k));
    const float co = r.mean ? ln2 * a.w : 0.f;
    return fmaf(cs, total, co * other);
}

// Where the splat gradients go: candidate-major [C][9], or in row tiles
// [tile of 128 rows][i < k][9][128] (GS_SGRAD_ROW_TILES).  The row of a
// candidate id = row k + i comes from a multiply-high division by the
// invariant k (Granlund and Montgomery, "Division by invariant integers using
// multiplication", PLDI 1994, Fig. 4.1): t = umulhi(m, id), row = (t + ((id -
// t) >> s1)) >> s2, with m, s1, s2 from the host.
struct SgOut {
    float *g;
    int tiled;
    uint32_t k, m, s1, s2;
};
__device__ __forceinline__ uint32_t sg_offset(const SgOut &o, uint32_t id)
{
    if (!o.tiled) return 9u * id;
    const uint32_t t = __umulhi(o.m, id);
    const uint32_t row = (t + ((id - t) >> o.s1)) >> o.s2, i = id - row * o.k;
    return ((row >> 7) * o.k + i) * 9u * 128u + (row & 127u);
}
// The staged splats' ids become the offsets of their gradient entries.
__device__ __forceinline__ void stage_offsets(WarpStage &W, int cnt, const SgOut &o)
{
    const int lane = threadIdx.x & 31;
    if (lane < cnt) W.id[lane] = sg_offset(o, W.id[lane]);
    __syncwarp();
}

// The 9 per-splat sums of a staged splat: reduced across the warp, turned
// into the splat's gradient and added to its entry (one atomic per value).
__device__ __forceinline__ void splat_sums_out(const float acc[9], const LaneRole &role, int vi, float4 a, float4 bb,
                                               uint32_t off, const SgOut &sg)
{
    const int lane = threadIdx.x & 31;
    const float io = ex2_approx(-bb.y);   // 1 / opacity from the record's log2 opacity
    const float t8 = warp_sum8(acc);
    const float t9 = warp_sum(acc[8]);
    const float other = __shfl_xor_sync(0xffffffffu, t8, 4);
    const float g = conic_grads(role, t8, other, a, bb, io);
    float *o = sg.g + off;
    const uint32_t stride = sg.tiled ? 128u : 1u;
    if ((lane & 3) == 0) atomicAdd(o + stride * vi, g);
    if (lane == 1) atomicAdd(o + stride * 8u, t9);
}

// Reverse pass of one work unit (block `warp` of item b).
//
// A tile whose list is one work item is walked front to back: per pixel the
// traversal recomputes, splat by splat, the transmittance in front of it and
// the colour composited so far -- the forward's own arithmetic, so every
// skip / stop decision is the forward's -- and takes the colour behind a
// splat as the pixel's final colour (the forward's image) minus that prefix.
// Nothing per pixel is stored by the forward, and no separate pass
// recomputes its state.
//
// A chunk of a longer list starts from the state the forward left for it --
// the transmittance after its last composited splat, that position, and the
// colour prefix up to its end (the colour behind the chunk is the final
// colour minus it) -- and is walked back to front from the last composited
// position, recovering the transmittance in front of each splat by dividing
// by 1 - alpha.
__device__ __forceinline__ void bwd_unit(const float4 *__restrict__ rec, const uint32_t *__restrict__ vals,
                                         const uint32_t *__restrict__ ranges, const ViewTable &vt,
                                         const RenderPlan &plan, const float *__restrict__ image,
                                         const float *__restrict__ d_image, const int32_t *__restrict__ last_in,
                                         const SgOut &sg, long long cap_cand, const gs_status *st, int b,
                                         int warp, WarpStage &WSw)
{
    Item it;
    if (!item_of(b, plan.item_base, plan.item_tile, vt.total_tiles, ranges, plan.L, &it)) return;
    const int lane = threadIdx.x & 31, tid = warp * 32 + lane;
    const TileCoord tc = tile_coord(vt, it.t, tid);
    const int v = tc.v;
    const long long W = vt.W[v], H = vt.H[v];
    const LanePix lpx = lane_pixels(tc, warp, lane, (int)W, (int)H);
    const int px0 = lpx.px0, py = lpx.py;
    const int pid0 = lpx.pid0;
    const float fx0 = (float)px0, fx1 = (float)(px0 + 8), fy = (float)py;
    const float bx0 = (float)tc.x0, bx1 = bx0 + (float)(kTile - 1);
    const float by0 = (float)(tc.y0 + 4 * warp), by1 = by0 + 3.f;
    const long long pix0 = (long long)py * W + px0;
    const int n_items = (int)(it.s1 - it.s0);
    const bool multi = it.nk > 1;
    // per pixel: g = dL/dC and GC = g . (final colour)
    PixBwd p0, p1;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        PixBwd &ps = h ? p1 : p0;
        const bool in = h ? lpx.in1 : lpx.in0;
        const long long pix = pix0 + 8 * h;
        ps.T = 1.f;
        ps.Sp = ps.GC = ps.g0 = ps.g1 = ps.g2 = 0.f;
        ps.lim = 0;
        ps.done = true;
        if (!in) continue;
        const float *dimg = d_image + 3 * vt.pix_base[v];
        const float *img = image + 3 * vt.pix_base[v];
        ps.g0 = dimg[pix];
        ps.g1 = dimg[W * H + pix];
        ps.g2 = dimg[2 * W * H + pix];
        ps.GC = fmaf(ps.g0, img[pix], fmaf(ps.g1, img[W * H + pix], ps.g2 * img[2 * W * H + pix]));
        ps.lim = last_in ? min(last_in[vt.pix_base[v] + pix], n_items) : n_items;
        ps.done = ps.lim <= 0;
    }
    const int vi = ((lane >> 4) & 1) * 4 + ((lane >> 3) & 1) * 2 + ((lane >> 2) & 1);
    const LaneRole role = lane_role(vi);
    if (multi) {
        // ---- a chunk of a longer list, back to front from its last composited splat
        const int item = it.base + it.k;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            PixBwd &ps = h ? p1 : p0;
            const int pid = pid0 + 8 * h;
            ps.lim = 0;
            if (!(h ? lpx.in1 : lpx.in0)) continue;
            const float T0 = state_plane(plan.state, item, 0)[pid];
            if (!(T0 >= kTMin)) continue;   // behind the pixel's stop
            ps.T = state_plane(plan.state, item, 1)[pid];
            ps.lim = min(reinterpret_cast<const int *>(state_plane(plan.state, item, 5))[pid], n_items);
            // g . (colour behind the chunk) = GC - g . (colour up to and including it)
            ps.Sp = ps.GC - fmaf(ps.g0, state_plane(plan.state, item, 2)[pid],
                                 fmaf(ps.g1, state_plane(plan.state, item, 3)[pid],
                                      ps.g2 * state_plane(plan.state, item, 4)[pid]));
        }
        const int maxlast = __reduce_max_sync(0xffffffffu, max(p0.lim, p1.lim));
        // the block's list (ascending positions): its entries in front of maxlast, back to front
        const uint32_t *bl = plan.blist + 4ull * it.s0 + (size_t)warp * (it.s1 - it.s0);
        int je = 0;   // entries with position < maxlast (binary search, every lane the same)
        {
            int lo = 0, hi = plan.bcnt[4 * b + warp];
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if ((int)__ldg(bl + mid) < maxlast) lo = mid + 1; else hi = mid;
            }
            je = lo;
        }
        for (int hj = je; hj > 0; hj -= 32) {
            const int jl = hj - 1 - lane;   // lane l <-> entry hj - 1 - l: hits come back to front
            const uint32_t pos = it.s0 + (jl >= 0 ? __ldg(bl + jl) : 0u);
            const int cnt = warp_stage<false>(WSw, rec, vals, pos, it.s0, jl >= 0,
                                                    cap_cand, st, 53, bx0, bx1, by0, by1);
            stage_offsets(WSw, cnt, sg);
            for (int e = 0; e < cnt; ++e) {
                const int p = WSw.pos[e];
                const float4 a = WSw.a[e];
                const float4 bb = WSw.b[e];
                float dx0 = 0.f, dy0 = 0.f, ag0 = 0.f, dx1 = 0.f, dy1 = 0.f, ag1 = 0.f;
                const bool c0 = p < p0.lim && alpha_test(a, bb, fx0, fy, &dx0, &dy0, &ag0);
                const bool c1 = p < p1.lim && alpha_test(a, bb, fx1, fy, &dx1, &dy1, &ag1);
                const bool contrib = c0 || c1;
                if (!__any_sync(0xffffffffu, contrib)) continue;
                float acc[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
                const float cb = WSw.c[e];
                {   // pixel 0 where it composites the splat, else pixel 1
                    const bool u1 = !c0;
                    float T = u1 ? p1.T : p0.T, S = u1 ? p1.Sp : p0.Sp;
                    if (contrib) {
                        bwd_composite_b2f(T, S, u1 ? p1.g0 : p0.g0, u1 ? p1.g1 : p0.g1, u1 ? p1.g2 : p0.g2, bb, cb,
                                          u1 ? dx1 : dx0, u1 ? dy1 : dy0, u1 ? ag1 : ag0, acc);
                        if (u1) { p1.T = T; p1.Sp = S; } else { p0.T = T; p0.Sp = S; }
                    }
                }
                if (__any_sync(0xffffffffu, c0 && c1) && c0 && c1)   // a lane that composites it at both pixels
                    bwd_composite_b2f(p1.T, p1.Sp, p1.g0, p1.g1, p1.g2, bb, cb, dx1, dy1, ag1, acc);
                splat_sums_out(acc, role, vi, a, bb, WSw.id[e], sg);
            }
            __syncwarp();
        }
        return;
    }
    // ---- a tile whose list is one work item, front to back (the forward's stop rule decided again
    // unless `last` is given)
    const int maxlim = __reduce_max_sync(0xffffffffu, max(p0.done ? 0 : p0.lim, p1.done ? 0 : p1.lim));
    const bool stop_rule = !last_in;
    for (int b0 = 0; b0 < maxlim; b0 += 32) {
        if (__all_sync(0xffffffffu, p0.done && p1.done)) break;
        const int pl = b0 + lane;
        const int cnt = warp_stage<true>(WSw, rec, vals, it.s0 + (uint32_t)pl, it.s0, pl < maxlim, cap_cand,
                                               st, 53, bx0, bx1, by0, by1);
        stage_offsets(WSw, cnt, sg);
        for (int e = 0; e < cnt; ++e) {
            const int q1 = WSw.pos[e] + 1;
            const float4 a = WSw.a[e];
            const float4 bb = WSw.b[e];
            const int hm = WSw.half[e];
            float dx0 = 0.f, dy0 = 0.f, ag0 = 0.f, dx1 = 0.f, dy1 = 0.f, ag1 = 0.f;
            bool c0 = (hm & 1) && !p0.done && q1 <= p0.lim && alpha_test(a, bb, fx0, fy, &dx0, &dy0, &ag0);
            bool c1 = (hm & 2) && !p1.done && q1 <= p1.lim && alpha_test(a, bb, fx1, fy, &dx1, &dy1, &ag1);
            if (stop_rule) {   // T (1 - alpha) < 1e-4 stops the pixel before the splat, as in the forward
                if (c0 && __fmul_rn(p0.T, 1.f - fminf(kAlphaMax, ag0)) < kTMin) { p0.done = true; c0 = false; }
                if (c1 && __fmul_rn(p1.T, 1.f - fminf(kAlphaMax, ag1)) < kTMin) { p1.done = true; c1 = false; }
            }
            const bool contrib = c0 || c1;
            if (!__any_sync(0xffffffffu, contrib)) continue;
            float acc[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
            const float cb = WSw.c[e];
            {   // pixel 0 where it composites the splat, else pixel 1
                const bool u1 = !c0;
                float T = u1 ? p1.T : p0.T, Sp = u1 ? p1.Sp : p0.Sp;
                if (contrib) {
                    bwd_composite_f2b(T, Sp, u1 ? p1.GC : p0.GC, u1 ? p1.g0 : p0.g0, u1 ? p1.g1 : p0.g1,
                                      u1 ? p1.g2 : p0.g2, bb, cb, u1 ? dx1 : dx0, u1 ? dy1 : dy0, u1 ? ag1 : ag0,
                                      acc);
                    if (u1) { p1.T = T; p1.Sp = Sp; } else { p0.T = T; p0.Sp = Sp; }
                }
            }
            if (__any_sync(0xffffffffu, c0 && c1) && c0 && c1)   // a lane that composites it at both pixels
                bwd_composite_f2b(p1.T, p1.Sp, p1.GC, p1.g0, p1.g1, p1.g2, bb, cb, dx1, dy1, ag1, acc);
            splat_sums_out(acc, role, vi, a, bb, WSw.id[e], sg);
        }
        __syncwarp();
        // pixels whose last position lies in this batch are finished
        if (p0.lim <= b0 + 32) p0.done = true;
        if (p1.lim <= b0 + 32) p1.done = true;
    }
}

// Persistent reverse pass: each warp takes work units u = 4 i + w from the
// counter and runs block w of item i.
__global__ void __launch_bounds__(kRThreads) render_bwd_kernel(
    const float4 *__restrict__ rec, const uint32_t *__restrict__ vals, const uint32_t *__restrict__ ranges,
    ViewTable vt, RenderPlan plan, const float *__restrict__ image, const float *__restrict__ d_image,
    const int32_t *__restrict__ last_in, SgOut sg, long long cap_cand, const gs_status *st)
{
    if (has_error(st)) return;
    __shared__ WarpStage WS[kRThreads / 32];
    WarpStage &W = WS[threadIdx.x >> 5];
    const int n_units = 4 * __ldg(plan.item_base + vt.total_tiles);
    int32_t *counter = plan.counters + 2;
    for (int u = next_unit(counter); u < n_units; u = next_unit(counter))
        bwd_unit(rec, vals, ranges, vt, plan, image, d_image, last_in, sg, cap_cand, st, u >> 2, u & 3, W);
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
            const float s[3] = {__ldg(a.scale + 3 * c), __ldg(a.scale + 3 * c + 1), __ldg(a.scale + 3 * c + 2)};
            const float q[4] = {__ldg(a.quat + 4 * c), __ldg(a.quat + 4 * c + 1), __ldg(a.quat + 4 * c + 2),
                                __ldg(a.quat + 4 * c + 3)};
            proj_bwd_one(cm, (float)vt.W[v], (float)vt.H[v], m0, m1, m2, s, q, gmx, gmy, gka, gkb, gkc, dmu, ds, dq);
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
// Zeroes the splat gradients of every candidate up to the row count (the
// reverse pass adds into those that cover a tile).  Whole 16-byte pieces:
// zeroing only the covering candidates would leave sectors shared with a
// non-covering neighbour partly written, which costs DRAM read-modify-writes.
__global__ void __launch_bounds__(256) zero_sgrad_kernel(const int32_t *__restrict__ view_start, int V, int k,
                                                         long long cap_rows, int tiled, float *__restrict__ sgrad,
                                                         const gs_status *st)
{
    if (has_error(st)) return;
    long long rows = std::min<long long>(__ldg(view_start + V), cap_rows);
    if (tiled) rows = (rows + 127) / 128 * 128;   // the whole last tile of rows
    const long long n = 9 * rows * k;
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long t0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if ((reinterpret_cast<uintptr_t>(sgrad) & 15) == 0) {
        float4 *v = reinterpret_cast<float4 *>(sgrad);
        for (long long i = t0; i < n / 4; i += stride) v[i] = make_float4(0.f, 0.f, 0.f, 0.f);
        for (long long i = 4 * (n / 4) + t0; i < n; i += stride) sgrad[i] = 0.f;
    } else {
        for (long long i = t0; i < n; i += stride) sgrad[i] = 0.f;
    }
}

int launch_render_bwd(const gs_gauss3d *g, const gs_camera *cams, const gs_splats *sp, const gs_bins *bins,
                      const ViewTable &vt, int L, void *ws, const float *image, const float *d_image,
                      const int32_t *last, gs_splat_grad *sgrad, gs_gauss3d_grad *out, gs_status *st,
                      cudaStream_t s)
{
    const long long cap_cand = g->cap_rows * (long long)g->k;
    const bool tiled = sgrad->layout == GS_SGRAD_ROW_TILES;
    if (9ll * ((g->cap_rows + 127) / 128 * 128) * g->k >= (1ll << 32)) return GS_ERR_UNSUPPORTED;   // 32-bit offsets
    SgOut sg;
    sg.g = sgrad->g;
    sg.tiled = tiled ? 1 : 0;
    sg.k = (uint32_t)g->k;
    {   // multiply-high division by k (see SgOut)
        int l = 0;
        while ((1u << l) < sg.k) ++l;
        sg.m = (uint32_t)(((1ull << 32) * ((1ull << l) - sg.k)) / sg.k + 1);
        sg.s1 = l > 0 ? 1u : 0u;
        sg.s2 = l > 0 ? (uint32_t)(l - 1) : 0u;
    }
    const int zgrid = (int)std::max<long long>(1, std::min<long long>((cap_cand + 255) / 256,
                                                                      (long long)sm_count() * 16));
    zero_sgrad_kernel<<<zgrid, 256, 0, s>>>(g->view_start, vt.V, g->k, g->cap_rows, sg.tiled, sgrad->g, st);
    count_launches(1);
    const float4 *rec = reinterpret_cast<const float4 *>(sp->rec);
    if (vt.total_tiles > 0) {
        const RenderPlan plan = render_plan(vt, bins->cap_pairs, L, ws);
        cudaMemsetAsync(plan.counters + 2, 0, sizeof(int32_t), s);
        render_bwd_kernel<<<persistent_grid((const void *)render_bwd_kernel, tuning().bwd_ctas_per_sm), kRThreads, 0, s>>>(
            rec, bins->vals, bins->ranges, vt, plan, image, d_image, last, sg,
            std::min<long long>(sp->cap, cap_cand), st);
        count_launches(1);
    }
    if (!out) return cudaPeekAtLastError() == cudaSuccess ? GS_OK : GS_ERR_CUDA;
    return launch_project_bwd(g, cams, sp, vt, sgrad, out, st, s);
}

int launch_project_bwd(const gs_gauss3d *g, const gs_camera *cams, const gs_splats *sp, const ViewTable &vt,
                       const gs_splat_grad *sgrad, gs_gauss3d_grad *out, gs_status *st, cudaStream_t s)
{
    const long long cap_cand = g->cap_rows * (long long)g->k;
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
