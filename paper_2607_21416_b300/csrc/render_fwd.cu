// render_fwd.cu -- front-to-back tile compositing (Eq. 1) over chunked work
// items, and the L1 term of Eq. 3.
//
// Kernels (all views in every launch, tiles numbered view-major; 128 threads
// per work item, each owning pixels (x, y) and (x, y + 1) of the 16x16 tile, so
// every splat read from shared memory serves two evaluations; each warp walks
// only the splats whose alpha >= 1/255 box meets its 16x4 block):
//   plan_kernel     per-tile chunk counts -> item_base (one CTA scan)
//   chunk_kernel    compositing of every item: single-chunk tiles write the
//                   image directly; chunk 0 of a multi-chunk tile composites
//                   exactly, later chunks on their own transmittance (see
//                   render_common.cuh); multi-chunk tiles write per-chunk state
//   combine_kernel  multi-chunk tiles: scales each chunk by the transmittance
//                   in front of it and writes the image, or marks the chunk
//                   that holds the pixel's stop for the fix-up
//   chunk_kernel<fix-up>  composites the marked chunks again from their
//                   entering transmittance, with the stop rule
// The power / alpha arithmetic is pinned (explicit fmaf / __fmul_rn) so every
// pass that re-evaluates a pair takes bit-identical skip / stop decisions.
#include "render_common.cuh"

namespace gs {

__global__ void __launch_bounds__(1024) plan_kernel(const uint32_t *__restrict__ ranges, int T, int L,
                                                    int max_items, int32_t *__restrict__ item_base,
                                                    int32_t *__restrict__ fix, int32_t *__restrict__ counters,
                                                    const gs_status *st)
{
    for (int i = threadIdx.x; i < max_items; i += blockDim.x) fix[i] = 0;
    if (threadIdx.x < 8) counters[threadIdx.x] = 0;
    __shared__ int s_warp[32];
    __shared__ long long s_carry;
    if (threadIdx.x == 0) s_carry = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const bool err = __syncthreads_or(has_error(st));   // one decision for the block
    for (int base = 0; base < T; base += 1024) {
        const int t = base + threadIdx.x;
        int x = 0;
        if (t < T) {
            const uint32_t n = err ? 0u : ranges[2 * t + 1] - ranges[2 * t];
            x = n > (uint32_t)L ? (int)((n + L - 1) / L) : 1;
        }
        int v = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, v, o);
            if (lane >= o) v += y;
        }
        if (lane == 31) s_warp[warp] = v;
        __syncthreads();
        if (warp == 0) {
            int w = s_warp[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, w, o);
                if (lane >= o) w += y;
            }
            s_warp[lane] = w;
        }
        __syncthreads();
        const long long excl = s_carry + v - x + (warp > 0 ? s_warp[warp - 1] : 0);
        if (t < T) item_base[t] = (int32_t)excl;
        __syncthreads();
        if (threadIdx.x == 0) s_carry += s_warp[31];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const long long total = s_carry;
        if (total > max_items) {   // cannot happen for pairs within capacity
            idx_ok(st, total, max_items, 40);
            item_base[T] = 0;
        } else {
            item_base[T] = (int32_t)total;
        }
    }
}

constexpr int kLongTile = 32;   // chunks above which the combine takes a tile first

// The tile of every item (one thread per tile writes its items' entries), so
// that a work unit finds its tile without a search.
__global__ void __launch_bounds__(256) item_tiles_kernel(const int32_t *__restrict__ item_base, int T,
                                                         int max_items, int32_t *__restrict__ item_tile,
                                                         int32_t *__restrict__ multi_list, int32_t *__restrict__ counters)
{
    const int n = min(item_base[T], max_items);   // 0 when the plan overflowed (no item runs)
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < T; t += gridDim.x * blockDim.x) {
        const int b0 = item_base[t], b1 = t + 1 < T ? min(item_base[t + 1], n) : n;
        for (int b = max(b0, 0); b < b1; ++b) item_tile[b] = t;
        // tiles cut into several chunks: the long ones from the front of the list, the others from the
        // back, so that the combine starts the longest walks first
        if (b1 - b0 > kLongTile) multi_list[atomicAdd(counters + 5, 1)] = t;
        else if (b1 - b0 > 1) multi_list[T - 1 - atomicAdd(counters + 7, 1)] = t;
    }
}

// Front-to-back state of one pixel.
struct PixFwd {
    float T, C0, C1, C2;
    int last;      // position of the last composited splat (1-based, in the chunk)
    int stop;      // position of the splat that stopped the pixel (0: not stopped)
    int ncomp;     // splats composited
    bool done;
};

// Eq. 1 step of one pixel over a staged splat at chunk position pos (1-based).
// STOP: the stop rule of the method (the pixel's entering transmittance is
// known).  Otherwise (a later chunk on its own transmittance) every splat is
// composited; once the chunk's own product is below 1e-4 the pixel is stopped
// in any case and the pass ends for it.
template <bool STOP>
__device__ __forceinline__ void fwd_step(PixFwd &ps, const float4 a, const float4 bb, float cb, float px, float py,
                                         int pos)
{
    float dx, dy;
    const float q = splat_q(a, bb.x, px, py, &dx, &dy);
    if (q > 0.f) return;
    const float alpha = fminf(kAlphaMax, splat_alpha(q, bb.y));
    if (alpha < kAlphaMin) return;
    const float Tn = __fmul_rn(ps.T, 1.f - alpha);
    if (STOP && Tn < kTMin) { ps.done = true; ps.stop = pos; return; }
    const float w = __fmul_rn(alpha, ps.T);
    ps.C0 = fmaf(bb.z, w, ps.C0);
    ps.C1 = fmaf(bb.w, w, ps.C1);
    ps.C2 = fmaf(cb, w, ps.C2);
    ps.T = Tn;
    ps.last = pos;
    ++ps.ncomp;
    if (!STOP && Tn < kTMin) ps.done = true;
}

// Image (and optional T_final / last) of one pixel; lastg < 0 leaves `last`.
__device__ __forceinline__ void write_image(const ViewTable &vt, int v, int px, int py, float C0, float C1, float C2,
                                            float T, int lastg, float bg0, float bg1, float bg2, float *image,
                                            float *T_final, int32_t *last)
{
    const long long W = vt.W[v], H = vt.H[v];
    const long long p = (long long)py * W + px;
    float *img = image + 3 * vt.pix_base[v];
    img[p] = fmaf(T, bg0, C0);
    img[W * H + p] = fmaf(T, bg1, C1);
    img[2 * W * H + p] = fmaf(T, bg2, C2);
    if (T_final) T_final[vt.pix_base[v] + p] = T;
    if (last && lastg >= 0) last[vt.pix_base[v] + p] = lastg;
}

// Warp totals of the examined / composited pair counts into n_eval[0..1]
// (and [2..3] for a tile whose list is a single work item).
__device__ __forceinline__ void count_add(unsigned long long *n_eval, unsigned long long nev, unsigned long long ncomp,
                                          bool single = false)
{
    for (int o = 16; o > 0; o >>= 1) {
        nev += __shfl_down_sync(0xffffffffu, nev, o);
        ncomp += __shfl_down_sync(0xffffffffu, ncomp, o);
    }
    if ((threadIdx.x & 31) == 0 && nev) {
        atomicAdd(n_eval, nev);
        if (single) atomicAdd(n_eval + 2, nev);
    }
    if ((threadIdx.x & 31) == 0 && ncomp) {
        atomicAdd(n_eval + 1, ncomp);
        if (single) atomicAdd(n_eval + 3, ncomp);
    }
}

// Block lists of the items of tiles cut into several chunks (persistent
// warps, one item at a time): the item's list is read once, each splat's
// alpha box tested against the four 16x4 blocks of the tile (the test of
// warp_stage, so a block's list holds exactly the splats its walk would
// stage), and the hits appended to the blocks' lists in list order.  The
// compositing walks of those items then read only their block's list instead
// of the whole chunk, four times over.
__global__ void __launch_bounds__(kRThreads) block_lists_kernel(const float4 *__restrict__ rec,
                                                                const uint32_t *__restrict__ vals,
                                                                const uint32_t *__restrict__ ranges, ViewTable vt,
                                                                RenderPlan plan, long long cap_cand,
                                                                const gs_status *st)
{
    if (has_error(st)) return;
    const int lane = threadIdx.x & 31;
    unsigned lt;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(lt));
    const int n_items = __ldg(plan.item_base + vt.total_tiles);
    int32_t *counter = plan.counters + 4;
    for (int b = next_unit(counter); b < n_items; b = next_unit(counter)) {
        Item it;
        if (!item_of(b, plan.item_base, plan.item_tile, vt.total_tiles, ranges, plan.L, &it) || it.nk <= 1) continue;
        const TileCoord tc = tile_coord(vt, it.t, 0);
        const uint32_t n = it.s1 - it.s0;
        uint32_t *bl = plan.blist + 4ull * it.s0;
        int cnt[4] = {0, 0, 0, 0};
        constexpr int kAhead = 4;   // 32-position batches whose loads are issued together
        for (uint32_t b0 = it.s0; b0 < it.s1; b0 += 32 * kAhead) {
            uint32_t id[kAhead];
            float4 a[kAhead], bb[kAhead];
#pragma unroll
            for (int u = 0; u < kAhead; ++u) {
                const uint32_t pos = b0 + 32 * u + lane;
                id[u] = pos < it.s1 ? vals[pos] : 0u;
            }
#pragma unroll
            for (int u = 0; u < kAhead; ++u) {
                const uint32_t pos = b0 + 32 * u + lane;
                if (pos < it.s1 && !idx_ok(st, (long long)id[u], cap_cand, 44)) id[u] = 0;
                a[u] = pos < it.s1 ? __ldg(&rec[3 * (size_t)id[u]]) : make_float4(0.f, 0.f, 0.f, 0.f);
                bb[u] = pos < it.s1 ? __ldg(&rec[3 * (size_t)id[u] + 1]) : make_float4(0.f, 0.f, 0.f, 0.f);
            }
#pragma unroll
            for (int u = 0; u < kAhead; ++u) {
                const uint32_t pos = b0 + 32 * u + lane;
#pragma unroll
                for (int w = 0; w < 4; ++w) {
                    const BlockRect r = block_rect(tc, w);
                    const bool hit = pos < it.s1 && meets_block(a[u], bb[u], r.x0, r.x1, r.y0, r.y1);
                    const unsigned m = __ballot_sync(0xffffffffu, hit);
                    if (hit) bl[w * n + cnt[w] + __popc(m & lt)] = pos - it.s0;
                    cnt[w] += __popc(m);
                }
            }
        }
        if (lane < 4) plan.bcnt[4 * b + lane] = lane == 0 ? cnt[0] : (lane == 1 ? cnt[1] : (lane == 2 ? cnt[2] : cnt[3]));
    }
}

// Compositing of one work item (FIX: the fix-up pass over marked chunks).
// Each warp walks only the staged splats whose alpha box meets its pixel
// block.  With COUNT, the pairs the method examines (every list position up to
// the stop) and the pairs composited are counted for the chunks whose activity
// is decided here; the combine step counts the others.
template <bool COUNT, bool FIX>
__device__ __forceinline__ void chunk_unit(const float4 *__restrict__ rec, const uint32_t *__restrict__ vals,
                                           const uint32_t *__restrict__ ranges, const ViewTable &vt,
                                           const RenderPlan &plan, float bg0, float bg1, float bg2,
                                           float *__restrict__ image, float *__restrict__ T_final,
                                           int32_t *__restrict__ last, unsigned long long *__restrict__ n_eval,
                                           long long cap_cand, const gs_status *st, int b, int warp, WarpStage &W)
{
    if (FIX && plan.fix[b] == 0) return;
    Item it;
    if (!item_of(b, plan.item_base, plan.item_tile, vt.total_tiles, ranges, plan.L, &it)) return;
    const int lane = threadIdx.x & 31, tid = warp * 32 + lane;
    const TileCoord tc = tile_coord(vt, it.t, tid);
    const LanePix lp = lane_pixels(tc, warp, lane, vt.W[tc.v], vt.H[tc.v]);
    const float fx0 = (float)lp.px0, fx1 = (float)(lp.px0 + 8), fy = (float)lp.py;
    const float bx0 = (float)tc.x0, bx1 = bx0 + (float)(kTile - 1);
    const float by0 = (float)(tc.y0 + 4 * warp), by1 = by0 + 3.f;
    const bool multi = it.nk > 1;
    const bool exact = !multi || it.k == 0 || FIX;
    const int item = it.base + it.k;
    PixFwd p0, p1;
    p0.T = p1.T = 1.f;
    p0.C0 = p0.C1 = p0.C2 = p1.C0 = p1.C1 = p1.C2 = 0.f;
    p0.last = p1.last = p0.stop = p1.stop = p0.ncomp = p1.ncomp = 0;
    p0.done = !lp.in0;
    p1.done = !lp.in1;
    if (FIX) {   // the marked pixels start from their entering transmittance
        const int *lst = reinterpret_cast<const int *>(state_plane(plan.state, item, 5));
        const float *tp = state_plane(plan.state, item, 1);
        p0.done = p0.done || lst[lp.pid0] != -1;
        p1.done = p1.done || lst[lp.pid0 + 8] != -1;
        if (!p0.done) p0.T = tp[lp.pid0];
        if (!p1.done) p1.T = tp[lp.pid0 + 8];
    }
    const bool act0 = !p0.done, act1 = !p1.done;
    // the warp walks the item's list on its own, 32 entries at a time: every position of a
    // single-chunk tile's list, or its block's list in a tile cut into several chunks
    const uint32_t *bl = plan.blist + 4ull * it.s0 + (size_t)warp * (it.s1 - it.s0);
    const uint32_t n_walk = multi ? (uint32_t)plan.bcnt[4 * b + warp] : it.s1 - it.s0;
    for (uint32_t j0 = 0; j0 < n_walk; j0 += 32) {
        if (__all_sync(0xffffffffu, p0.done && p1.done)) break;
        const uint32_t j = j0 + lane;
        const bool valid = j < n_walk;
        const uint32_t pos = it.s0 + (multi ? (valid ? bl[j] : 0u) : j);
        const int cnt = warp_stage<true>(W, rec, vals, pos, it.s0, valid, cap_cand, st, 42, bx0, bx1,
                                                 by0, by1);
        if (exact) {
            for (int e = 0; e < cnt; ++e) {
                const float4 a = W.a[e];
                const float4 bb = W.b[e];
                const float cb = W.c[e];
                const int q = W.pos[e] + 1, hm = W.half[e];
                if ((hm & 1) && !p0.done) fwd_step<true>(p0, a, bb, cb, fx0, fy, q);
                if ((hm & 2) && !p1.done) fwd_step<true>(p1, a, bb, cb, fx1, fy, q);
            }
        } else {
            for (int e = 0; e < cnt; ++e) {
                const float4 a = W.a[e];
                const float4 bb = W.b[e];
                const float cb = W.c[e];
                const int q = W.pos[e] + 1, hm = W.half[e];
                if ((hm & 1) && !p0.done) fwd_step<false>(p0, a, bb, cb, fx0, fy, q);
                if ((hm & 2) && !p1.done) fwd_step<false>(p1, a, bb, cb, fx1, fy, q);
            }
        }
        __syncwarp();
    }
    if (COUNT) {
        const int n_items = (int)(it.s1 - it.s0);
        unsigned long long nev = 0, ncomp = 0;
        if (exact) {
            if (act0) { nev += p0.stop ? p0.stop : n_items; ncomp += p0.ncomp; }
            if (act1) { nev += p1.stop ? p1.stop : n_items; ncomp += p1.ncomp; }
        }
        count_add(n_eval, nev, ncomp, !multi);
    }
#pragma unroll
    for (int half = 0; half < 2; ++half) {
        const PixFwd &ps = half ? p1 : p0;
        const int pix = lp.pid0 + 8 * half;
        const int px = lp.px0 + 8 * half, py = lp.py;
        if (!multi) {
            if (half ? lp.in1 : lp.in0)
                write_image(vt, tc.v, px, py, ps.C0, ps.C1, ps.C2, ps.T, ps.last, bg0, bg1, bg2, image, T_final,
                            last);
            continue;
        }
        if (FIX) {
            if (!(half ? act1 : act0)) continue;
            float *c0 = state_plane(plan.state, item, 2), *c1 = state_plane(plan.state, item, 3);
            float *c2 = state_plane(plan.state, item, 4);
            const float f0 = c0[pix] + ps.C0, f1 = c1[pix] + ps.C1, f2 = c2[pix] + ps.C2;   // prefix incl. this chunk
            state_plane(plan.state, item, 1)[pix] = ps.T;
            c0[pix] = f0;
            c1[pix] = f1;
            c2[pix] = f2;
            reinterpret_cast<int *>(state_plane(plan.state, item, 5))[pix] = ps.last;
            write_image(vt, tc.v, px, py, f0, f1, f2, ps.T, ps.last > 0 ? it.k * plan.L + ps.last : -1, bg0, bg1,
                        bg2, image, T_final, last);
            continue;
        }
        // per-chunk state; a stop in chunk 0 is marked by Tprod = 0
        state_plane(plan.state, item, 0)[pix] = (it.k == 0 && ps.stop) ? 0.f : ps.T;
        state_plane(plan.state, item, 1)[pix] = ps.T;
        state_plane(plan.state, item, 2)[pix] = ps.C0;
        state_plane(plan.state, item, 3)[pix] = ps.C1;
        state_plane(plan.state, item, 4)[pix] = ps.C2;
        reinterpret_cast<int *>(state_plane(plan.state, item, 5))[pix] = ps.last;
        if (COUNT) reinterpret_cast<int *>(state_plane(plan.state, item, 6))[pix] = ps.ncomp;
    }
}

// Persistent compositing: each warp takes work units u = 4 i + w from the
// counter and composites block w of item i (the fix-up pass: of the i-th
// marked item).
template <bool COUNT, bool FIX>
__global__ void __launch_bounds__(kRThreads) chunk_kernel(const float4 *__restrict__ rec,
                                                          const uint32_t *__restrict__ vals,
                                                          const uint32_t *__restrict__ ranges, ViewTable vt,
                                                          RenderPlan plan, float bg0, float bg1, float bg2,
                                                          float *__restrict__ image, float *__restrict__ T_final,
                                                          int32_t *__restrict__ last,
                                                          unsigned long long *__restrict__ n_eval,
                                                          long long cap_cand, const gs_status *st)
{
    if (has_error(st)) return;
    __shared__ WarpStage WS[kRThreads / 32];
    WarpStage &W = WS[threadIdx.x >> 5];
    const int n_units =
        4 * (FIX ? *(volatile const int32_t *)(plan.counters + 3) : __ldg(plan.item_base + vt.total_tiles));
    int32_t *counter = plan.counters + (FIX ? 1 : 0);
    for (int u = next_unit(counter); u < n_units; u = next_unit(counter)) {
        const int b = FIX ? plan.fix_list[u >> 2] : (u >> 2);
        chunk_unit<COUNT, FIX>(rec, vals, ranges, vt, plan, bg0, bg1, bg2, image, T_final, last, n_eval, cap_cand, st,
                               b, u & 3, W);
    }
}

// Multi-chunk tiles, per pixel: chunk 0 is exact; every later chunk k is
// scaled by the transmittance T0 in front of it (its state becomes the
// chunk's true contribution) while T0 * Tprod_k >= 1e-4 -- no splat of the
// chunk can then meet the stop rule; the first chunk where that fails holds
// the pixel's stop and is marked for the fix-up, with T0 and the colour in
// front of it in its Tend / colour planes and last = -1.
constexpr int kCombineAhead = 16;   // chunk states loaded per group by the combine walk

template <bool COUNT>
__device__ __forceinline__ void combine_tile(int t, const uint32_t *__restrict__ ranges, const ViewTable &vt,
                                             const RenderPlan &plan, float bg0, float bg1, float bg2,
                                             float *__restrict__ image, float *__restrict__ T_final,
                                             int32_t *__restrict__ last, unsigned long long *__restrict__ n_eval)
{
    const int base = plan.item_base[t], nk = plan.item_base[t + 1] - base;
    if (nk <= 1) return;
    // one pixel per thread: tile thread (threadIdx & 127), pixel row half (threadIdx >> 7)
    const TileCoord tc = tile_coord(vt, t, threadIdx.x & (kRThreads - 1));
    const uint32_t s_start = ranges[2 * t], s_end = ranges[2 * t + 1];
    unsigned long long nev = 0, ncomp = 0;
    {
        const int half = threadIdx.x >> 7;
        const int pix = tc.pid0 + half * kTile;
        const int py = tc.py + half;
        const bool inside = half ? tc.in1 : tc.in0;
        float C0 = state_plane(plan.state, base, 2)[pix];
        float C1 = state_plane(plan.state, base, 3)[pix];
        float C2 = state_plane(plan.state, base, 4)[pix];
        const int l0 = reinterpret_cast<const int *>(state_plane(plan.state, base, 5))[pix];
        int lastg = l0 > 0 ? l0 : 0;
        float *t00 = state_plane(plan.state, base, 0);
        float T0 = t00[pix];   // chunk 0's own product (0: it stopped the pixel)
        t00[pix] = 1.f;        // chunk 0 is always active
        int k = 1;
        bool marked = false;
        if (T0 == 0.f) {       // chunk 0 stopped the pixel
            T0 = state_plane(plan.state, base, 1)[pix];
        } else {
            // the chunks' states are read kCombineAhead at a time before any of
            // them is written (different items: no overlap), so the walk waits
            // for one load latency per group instead of one per chunk
            bool go = true;
            while (go && k < nk) {
                const int k0 = k;
                float gTp[kCombineAhead], ga0[kCombineAhead], ga1[kCombineAhead], ga2[kCombineAhead];
                int gl[kCombineAhead], gc[kCombineAhead];
#pragma unroll
                for (int g = 0; g < kCombineAhead; ++g) {
                    gTp[g] = ga0[g] = ga1[g] = ga2[g] = 0.f;
                    gl[g] = gc[g] = 0;
                    if (k0 + g < nk) {
                        const int it2 = base + k0 + g;
                        gTp[g] = state_plane(plan.state, it2, 0)[pix];
                        ga0[g] = state_plane(plan.state, it2, 2)[pix];
                        ga1[g] = state_plane(plan.state, it2, 3)[pix];
                        ga2[g] = state_plane(plan.state, it2, 4)[pix];
                        gl[g] = reinterpret_cast<const int *>(state_plane(plan.state, it2, 5))[pix];
                        if (COUNT) gc[g] = reinterpret_cast<const int *>(state_plane(plan.state, it2, 6))[pix];
                    }
                }
#pragma unroll
                for (int g = 0; g < kCombineAhead; ++g) {
                    const int kk = k0 + g;
                    if (!go || kk >= nk) continue;
                    if (!(T0 >= kTMin)) { k = kk; go = false; continue; }
                    const int item = base + kk;
                    float *tp = state_plane(plan.state, item, 0);
                    float *te = state_plane(plan.state, item, 1);
                    float *c0 = state_plane(plan.state, item, 2), *c1 = state_plane(plan.state, item, 3);
                    float *c2 = state_plane(plan.state, item, 4);
                    int *lp = reinterpret_cast<int *>(state_plane(plan.state, item, 5));
                    tp[pix] = T0;
                    const float T1 = __fmul_rn(T0, gTp[g]);
                    if (T1 >= kTMin) {   // no stop inside: the chunk's true contribution
                        C0 += T0 * ga0[g];
                        C1 += T0 * ga1[g];
                        C2 += T0 * ga2[g];
                        c0[pix] = C0;
                        c1[pix] = C1;
                        c2[pix] = C2;
                        te[pix] = T1;
                        if (gl[g] > 0) lastg = kk * plan.L + gl[g];
                        if (COUNT && inside) {
                            nev += min((uint32_t)plan.L, s_end - (s_start + (uint32_t)kk * (uint32_t)plan.L));
                            ncomp += gc[g];
                        }
                        T0 = T1;
                        k = kk + 1;
                    } else {             // the pixel's stop lies in chunk kk
                        te[pix] = T0;
                        c0[pix] = C0;
                        c1[pix] = C1;
                        c2[pix] = C2;
                        lp[pix] = -1;
                        if (inside) {
                            if (atomicExch(plan.fix + item, 1) == 0)
                                plan.fix_list[atomicAdd(plan.counters + 3, 1)] = item;
                            if (last) last[vt.pix_base[tc.v] + (long long)py * vt.W[tc.v] + tc.px] = lastg;
                        }
                        marked = true;
                        k = kk + 1;
                        go = false;
                    }
                }
            }
        }
        for (; k < nk; ++k) state_plane(plan.state, base + k, 0)[pix] = 0.f;   // behind the stop: inactive
        if (!marked) {
            if (inside) write_image(vt, tc.v, tc.px, py, C0, C1, C2, T0, lastg, bg0, bg1, bg2, image, T_final, last);
        }
    }
    if (COUNT) count_add(n_eval, nev, ncomp);
}

// A long multi-chunk tile (more than kLongTile chunks), one group of 32 of
// its pixels per CTA: the chunk walk of combine_tile split over the CTA's 8
// warps as a scan.  Chunk 0 is the exact start; chunks 1 .. nk-1 are cut into
// 8 consecutive segments, warp w owning segment w for the group's pixels
// (lane = pixel, so every plane access is one coalesced 128-byte row).
//   1. each warp reduces its segment: P = the product of the chunks' own
//      transmittances (running partial products Pk, in chunk order), Cs = sum
//      of P(k-1) times the chunk's colour, and the last composited position;
//   2. the entering state of segment w follows from chunk 0 and segments
//      0 .. w-1: T_w+1 = T_w P_w, C_w+1 = C_w + T_w Cs_w;
//   3. each warp walks its segment again: chunk k is entered with T_w P(k-1)
//      and left with T_w P(k) -- one rounding each, the product that step 2
//      forms at the segment's end -- so the stop (the first chunk left below
//      1e-4) is found by exactly one warp, and the segments behind it are
//      those entered below 1e-4.
// The states written are those of combine_tile (entering and leaving
// transmittance, colour prefix, last position; -1 and a fix-up mark where the
// stop falls).
constexpr int kLongSplit = 8;    // pixel groups (CTAs) per long tile
constexpr int kLongAhead = 8;    // chunk states loaded per group by a segment walk

template <bool COUNT>
__device__ __forceinline__ void combine_long(int t, int grp, const uint32_t *__restrict__ ranges, const ViewTable &vt,
                                             const RenderPlan &plan, float bg0, float bg1, float bg2,
                                             float *__restrict__ image, float *__restrict__ T_final,
                                             int32_t *__restrict__ last, unsigned long long *__restrict__ n_eval)
{
    __shared__ float s_P[kLongSplit][32], s_C[3][kLongSplit][32];
    __shared__ int s_L[kLongSplit][32];
    const int base = plan.item_base[t], nk = plan.item_base[t + 1] - base;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const TileCoord tc = tile_coord(vt, t, 0);
    const int pix = grp * 32 + lane;
    const int px = tc.x0 + (pix & (kTile - 1)), py = tc.y0 + pix / kTile;
    const bool inside = px < vt.W[tc.v] && py < vt.H[tc.v];
    const uint32_t s_start = ranges[2 * t], s_end = ranges[2 * t + 1];
    const int m = nk - 1;
    const int k0 = 1 + (w * m) / kLongSplit, k1 = 1 + ((w + 1) * m) / kLongSplit;
    // ---- 1. segment reduction
    {
        float P = 1.f, C0 = 0.f, C1 = 0.f, C2 = 0.f;
        int L = 0;
        for (int kb = k0; kb < k1; kb += kLongAhead) {
            float gT[kLongAhead], g0[kLongAhead], g1[kLongAhead], g2[kLongAhead];
            int gl[kLongAhead];
#pragma unroll
            for (int g = 0; g < kLongAhead; ++g) {
                gT[g] = 1.f; g0[g] = g1[g] = g2[g] = 0.f; gl[g] = 0;
                if (kb + g < k1) {
                    const int it = base + kb + g;
                    gT[g] = state_plane(plan.state, it, 0)[pix];
                    g0[g] = state_plane(plan.state, it, 2)[pix];
                    g1[g] = state_plane(plan.state, it, 3)[pix];
                    g2[g] = state_plane(plan.state, it, 4)[pix];
                    gl[g] = reinterpret_cast<const int *>(state_plane(plan.state, it, 5))[pix];
                }
            }
#pragma unroll
            for (int g = 0; g < kLongAhead; ++g) {
                if (kb + g >= k1) continue;
                C0 = fmaf(P, g0[g], C0);
                C1 = fmaf(P, g1[g], C1);
                C2 = fmaf(P, g2[g], C2);
                P = __fmul_rn(P, gT[g]);
                if (gl[g] > 0) L = (kb + g) * plan.L + gl[g];
            }
        }
        s_P[w][lane] = P;
        s_C[0][w][lane] = C0;
        s_C[1][w][lane] = C1;
        s_C[2][w][lane] = C2;
        s_L[w][lane] = L;
    }
    __syncthreads();
    // ---- 2. entering state of the segment
    float *t00 = state_plane(plan.state, base, 0);
    const float Tp0 = t00[pix];   // chunk 0's own product (0: it stopped the pixel)
    const bool stop0 = Tp0 == 0.f;
    float C0 = state_plane(plan.state, base, 2)[pix];
    float C1 = state_plane(plan.state, base, 3)[pix];
    float C2 = state_plane(plan.state, base, 4)[pix];
    const int l0 = reinterpret_cast<const int *>(state_plane(plan.state, base, 5))[pix];
    int lastg = l0 > 0 ? l0 : 0;
    float Tw = stop0 ? state_plane(plan.state, base, 1)[pix] : Tp0;
    for (int u = 0; u < w; ++u) {
        C0 = fmaf(Tw, s_C[0][u][lane], C0);
        C1 = fmaf(Tw, s_C[1][u][lane], C1);
        C2 = fmaf(Tw, s_C[2][u][lane], C2);
        Tw = __fmul_rn(Tw, s_P[u][lane]);
        if (s_L[u][lane] > 0) lastg = s_L[u][lane];
    }
    __syncthreads();   // chunk 0's planes are read by every warp before warp 0 marks it active
    if (w == 0) t00[pix] = 1.f;   // chunk 0 is always active
    // ---- 3. the segment's states
    unsigned long long nev = 0, ncomp = 0;
    bool marked = false;
    int k = k0;
    if (!stop0 && Tw >= kTMin) {
        float P = 1.f;
        bool go = true;
        for (int kb = k0; go && kb < k1; kb += kLongAhead) {
            float gT[kLongAhead], g0[kLongAhead], g1[kLongAhead], g2[kLongAhead];
            int gl[kLongAhead], gc[kLongAhead];
#pragma unroll
            for (int g = 0; g < kLongAhead; ++g) {
                gT[g] = 1.f; g0[g] = g1[g] = g2[g] = 0.f; gl[g] = gc[g] = 0;
                if (kb + g < k1) {
                    const int it = base + kb + g;
                    gT[g] = state_plane(plan.state, it, 0)[pix];
                    g0[g] = state_plane(plan.state, it, 2)[pix];
                    g1[g] = state_plane(plan.state, it, 3)[pix];
                    g2[g] = state_plane(plan.state, it, 4)[pix];
                    gl[g] = reinterpret_cast<const int *>(state_plane(plan.state, it, 5))[pix];
                    if (COUNT) gc[g] = reinterpret_cast<const int *>(state_plane(plan.state, it, 6))[pix];
                }
            }
#pragma unroll
            for (int g = 0; g < kLongAhead; ++g) {
                const int kk = kb + g;
                if (!go || kk >= k1) continue;
                const int item = base + kk;
                const float Tin = __fmul_rn(Tw, P);
                const float Pn = __fmul_rn(P, gT[g]);
                const float T1 = __fmul_rn(Tw, Pn);
                state_plane(plan.state, item, 0)[pix] = Tin;
                float *c0 = state_plane(plan.state, item, 2), *c1 = state_plane(plan.state, item, 3);
                float *c2 = state_plane(plan.state, item, 4);
                if (T1 >= kTMin) {   // no stop inside: the chunk's true contribution
                    C0 = fmaf(Tin, g0[g], C0);
                    C1 = fmaf(Tin, g1[g], C1);
                    C2 = fmaf(Tin, g2[g], C2);
                    c0[pix] = C0;
                    c1[pix] = C1;
                    c2[pix] = C2;
                    state_plane(plan.state, item, 1)[pix] = T1;
                    if (gl[g] > 0) lastg = kk * plan.L + gl[g];
                    if (COUNT && inside) {
                        nev += min((uint32_t)plan.L, s_end - (s_start + (uint32_t)kk * (uint32_t)plan.L));
                        ncomp += gc[g];
                    }
                    P = Pn;
                    k = kk + 1;
                } else {             // the pixel's stop lies in chunk kk
                    state_plane(plan.state, item, 1)[pix] = Tin;
                    c0[pix] = C0;
                    c1[pix] = C1;
                    c2[pix] = C2;
                    reinterpret_cast<int *>(state_plane(plan.state, item, 5))[pix] = -1;
                    if (inside) {
                        if (atomicExch(plan.fix + item, 1) == 0)
                            plan.fix_list[atomicAdd(plan.counters + 3, 1)] = item;
                        if (last) last[vt.pix_base[tc.v] + (long long)py * vt.W[tc.v] + px] = lastg;
                    }
                    marked = true;
                    k = kk + 1;
                    go = false;
                }
            }
        }
        // the pixel never stopped: the last segment holds its final colour
        if (!marked && w == kLongSplit - 1 && inside)
            write_image(vt, tc.v, px, py, C0, C1, C2, __fmul_rn(Tw, P), lastg, bg0, bg1, bg2, image, T_final, last);
    } else if (stop0 && w == 0 && inside) {   // chunk 0 stopped the pixel: its state is final
        write_image(vt, tc.v, px, py, C0, C1, C2, Tw, lastg, bg0, bg1, bg2, image, T_final, last);
    }
    for (; k < k1; ++k) state_plane(plan.state, base + k, 0)[pix] = 0.f;   // behind the stop: inactive
    if (COUNT) count_add(n_eval, nev, ncomp);
}

// One CTA per tile cut into several chunks (per pixel group of a long one),
// taken from the plan's list of such tiles through a counter: the long tiles'
// units first, then the others (CTAs that finish a unit take the next).
template <bool COUNT>
__global__ void __launch_bounds__(2 * kRThreads) combine_kernel(const uint32_t *__restrict__ ranges, ViewTable vt,
                                                            RenderPlan plan, float bg0, float bg1, float bg2,
                                                            float *__restrict__ image, float *__restrict__ T_final,
                                                            int32_t *__restrict__ last,
                                                            unsigned long long *__restrict__ n_eval,
                                                            const gs_status *st)
{
    if (has_error(st)) return;
    __shared__ int s_j;
    const int n_long = *(volatile const int32_t *)(plan.counters + 5);
    const int n_split = kLongSplit * n_long;   // units of the long tiles, taken first
    const int n_units = n_split + *(volatile const int32_t *)(plan.counters + 7);
    for (;;) {
        __syncthreads();   // the previous unit's readers of s_j and of the shared segment states are done
        if (threadIdx.x == 0) s_j = atomicAdd(plan.counters + 6, 1);
        __syncthreads();
        const int j = s_j;
        if (j >= n_units) break;
        if (j < n_split) {
            combine_long<COUNT>(__ldg(plan.multi_list + j / kLongSplit), j % kLongSplit, ranges, vt, plan, bg0, bg1,
                                bg2, image, T_final, last, n_eval);
        } else {
            const int t = __ldg(plan.multi_list + vt.total_tiles - 1 - (j - n_split));
            combine_tile<COUNT>(t, ranges, vt, plan, bg0, bg1, bg2, image, T_final, last, n_eval);
        }
    }
}

int persistent_grid(const void *kernel, int cap_per_sm)
{
    static int dev_smem = 0, dev_reserve = 0;
    if (dev_smem == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&dev_smem, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
        cudaDeviceGetAttribute(&dev_reserve, cudaDevAttrReservedSharedMemoryPerBlock, dev);
    }
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, kernel) != cudaSuccess) return sm_count();
    int occ = 64 / (kRThreads / 32);                                             // warps per SM
    occ = std::min(occ, 65536 / std::max(1, fa.numRegs * kRThreads));           // registers
    occ = std::min(occ, dev_smem / std::max(1, (int)fa.sharedSizeBytes + dev_reserve));
    if (cap_per_sm > 0) occ = std::min(occ, cap_per_sm);
    return sm_count() * std::max(1, occ);
}

// ------------------------------------------------------------------- L1
__global__ void __launch_bounds__(256) l1_kernel(const float *__restrict__ image, const float *__restrict__ target,
                                                 ViewTable vt, float *__restrict__ loss, float *__restrict__ d_image)
{
    const long long n = 3 * vt.total_pixels;
    float acc = 0.f;
    // a thread's elements increase, so its view (and the view's 1 / (3 pixels)) is carried along
    int v = 0;
    float inv = 1.f / (float)(3 * vt.pix_base[1]);
    auto view_at = [&](long long i) {
        if (v + 1 < vt.V && 3 * vt.pix_base[v + 1] <= i) {
            while (v + 1 < vt.V && 3 * vt.pix_base[v + 1] <= i) ++v;
            inv = 1.f / (float)(3 * vt.pix_base[v + 1] - 3 * vt.pix_base[v]);
        }
    };
    const long long stride = (long long)gridDim.x * blockDim.x, t0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    long long head = 0;   // elements handled four at a time (16-byte loads and stores)
    if (((reinterpret_cast<uintptr_t>(image) | reinterpret_cast<uintptr_t>(target) |
          reinterpret_cast<uintptr_t>(d_image)) & 15) == 0) {
        head = n & ~3ll;
        for (long long q = t0; 4 * q < head; q += stride) {
            const float4 x = reinterpret_cast<const float4 *>(image)[q];
            const float4 y = reinterpret_cast<const float4 *>(target)[q];
            const float d[4] = {x.x - y.x, x.y - y.y, x.z - y.z, x.w - y.w};
            float g[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                view_at(4 * q + e);
                acc += fabsf(d[e]) * inv;
                g[e] = d[e] > 0.f ? inv : (d[e] < 0.f ? -inv : 0.f);
            }
            reinterpret_cast<float4 *>(d_image)[q] = make_float4(g[0], g[1], g[2], g[3]);
        }
        v = 0;
        inv = 1.f / (float)(3 * vt.pix_base[1]);
    }
    for (long long i = head + t0; i < n; i += stride) {
        view_at(i);
        const float d = image[i] - target[i];
        acc += fabsf(d) * inv;
        d_image[i] = d > 0.f ? inv : (d < 0.f ? -inv : 0.f);
    }
    // block sum, then one atomic per block (one per warp contended on a single address)
    __shared__ float s_w[8];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        acc = threadIdx.x < (blockDim.x >> 5) ? s_w[threadIdx.x] : 0.f;
        for (int o = 4; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
        if (threadIdx.x == 0) atomicAdd(loss, acc);
    }
}

// ------------------------------------------------------------ launchers
int render_max_items(const ViewTable &vt, long long cap_pairs, int L)
{
    return (int)std::min<long long>((long long)vt.total_tiles + (cap_pairs + L - 1) / L, 1ll << 30);
}

size_t render_workspace_bytes(const ViewTable &vt, long long cap_pairs, int L)
{
    const long long items = render_max_items(vt, cap_pairs, L);
    return align_up(sizeof(int32_t) * ((size_t)vt.total_tiles + 1), 256) + 256 +
           2 * align_up(sizeof(int32_t) * (size_t)items, 256) +
           align_up(sizeof(float) * (size_t)items * kStateWords * kRT, 256) +
           align_up(sizeof(int32_t) * 4 * (size_t)items, 256) + align_up(sizeof(int32_t) * (size_t)items, 256) +
           align_up(sizeof(int32_t) * (size_t)vt.total_tiles, 256) +
           align_up(sizeof(uint32_t) * 4 * (size_t)std::max<long long>(cap_pairs, 1), 256);
}

// Workspace: item_base [T + 1] | counters [8] | fix flags [max_items] | fix list [max_items] |
// state [max_items][kStateWords][256] | block-list counts [max_items][4] | item tiles [max_items] |
// multi-chunk tile list [T] | block lists [4 cap_pairs]
RenderPlan render_plan(const ViewTable &vt, long long cap_pairs, int L, void *ws)
{
    RenderPlan p;
    p.L = L;
    p.max_items = render_max_items(vt, cap_pairs, L);
    char *w = reinterpret_cast<char *>(ws);
    const size_t o0 = align_up(sizeof(int32_t) * ((size_t)vt.total_tiles + 1), 256);
    const size_t o1 = o0 + 256;
    const size_t o2 = o1 + 2 * align_up(sizeof(int32_t) * (size_t)p.max_items, 256);
    const size_t o3 = o2 + align_up(sizeof(float) * (size_t)p.max_items * kStateWords * kRT, 256);
    const size_t o35 = o3 + align_up(sizeof(int32_t) * 4 * (size_t)p.max_items, 256);
    const size_t o36 = o35 + align_up(sizeof(int32_t) * (size_t)p.max_items, 256);
    const size_t o4 = o36 + align_up(sizeof(int32_t) * (size_t)vt.total_tiles, 256);
    p.item_base = reinterpret_cast<int32_t *>(w);
    p.counters = reinterpret_cast<int32_t *>(w + o0);
    p.fix = reinterpret_cast<int32_t *>(w + o1);
    p.fix_list = reinterpret_cast<int32_t *>(w + o1 + align_up(sizeof(int32_t) * (size_t)p.max_items, 256));
    p.state = reinterpret_cast<float *>(w + o2);
    p.bcnt = reinterpret_cast<int32_t *>(w + o3);
    p.item_tile = reinterpret_cast<int32_t *>(w + o35);
    p.multi_list = reinterpret_cast<int32_t *>(w + o36);
    p.blist = reinterpret_cast<uint32_t *>(w + o4);
    return p;
}

template <bool COUNT>
static void launch_items(const float4 *rec, const gs_bins *bins, const ViewTable &vt, const RenderPlan &plan,
                         const float bg[3], float *image, float *T_final, int32_t *last, unsigned long long *n_eval,
                         long long cap, gs_status *st, cudaStream_t s)
{
    chunk_kernel<COUNT, false><<<persistent_grid((const void *)chunk_kernel<COUNT, false>, tuning().fwd_ctas_per_sm), kRThreads, 0, s>>>(rec, bins->vals, bins->ranges, vt, plan, bg[0],
                                                                   bg[1], bg[2], image, T_final, last, n_eval, cap,
                                                                   st);
    combine_kernel<COUNT><<<(int)std::min<long long>(vt.total_tiles, (long long)sm_count() * 8), 2 * kRThreads, 0, s>>>(
        bins->ranges, vt, plan, bg[0], bg[1], bg[2], image, T_final, last, n_eval, st);
    chunk_kernel<COUNT, true><<<persistent_grid((const void *)chunk_kernel<COUNT, true>, tuning().fwd_ctas_per_sm), kRThreads, 0, s>>>(rec, bins->vals, bins->ranges, vt, plan, bg[0],
                                                                  bg[1], bg[2], image, T_final, last, n_eval, cap,
                                                                  st);
}

int launch_render_fwd(const gs_splats *sp, const gs_bins *bins, const ViewTable &vt, const float bg[3], int L,
                      void *ws, float *image, float *T_final, int32_t *last, long long *n_eval, gs_status *st,
                      cudaStream_t s)
{
    if (vt.total_tiles == 0) return GS_OK;
    const float4 *rec = reinterpret_cast<const float4 *>(sp->rec);
    const RenderPlan plan = render_plan(vt, bins->cap_pairs, L, ws);
    plan_kernel<<<1, 1024, 0, s>>>(bins->ranges, vt.total_tiles, L, plan.max_items,
                                   const_cast<int32_t *>(plan.item_base), plan.fix, plan.counters, st);
    item_tiles_kernel<<<(int)std::max<long long>(1, std::min<long long>((vt.total_tiles + 255) / 256, (long long)sm_count() * 4)),
                        256, 0, s>>>(plan.item_base, vt.total_tiles, plan.max_items, plan.item_tile, plan.multi_list,
                                     plan.counters);
    block_lists_kernel<<<persistent_grid((const void *)block_lists_kernel), kRThreads, 0, s>>>(
        rec, bins->vals, bins->ranges, vt, plan, sp->cap, st);
    if (n_eval) {
        cudaMemsetAsync(n_eval, 0, 4 * sizeof(long long), s);
        launch_items<true>(rec, bins, vt, plan, bg, image, T_final, last,
                           reinterpret_cast<unsigned long long *>(n_eval), sp->cap, st, s);
    } else {
        launch_items<false>(rec, bins, vt, plan, bg, image, T_final, last, nullptr, sp->cap, st, s);
    }
    count_launches(6);
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

}  // namespace gs
