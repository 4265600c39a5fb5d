// render_fwd.cu -- front-to-back tile compositing (Eq. 1) over chunked work
// items, and the L1 term of Eq. 3.
//
// Kernels (all views in every launch, tiles numbered view-major; 128 threads
// per work item, each owning pixels (x, y) and (x, y + 1) of the 16x16 tile, so
// every splat read from shared memory serves two evaluations; each warp walks
// only the splats whose alpha >= 1/255 box meets its 16x4 block):
//   plan_kernel     per-tile chunk counts -> item_base (one CTA scan)
//   prod_kernel     Tprod of every chunk of a multi-chunk tile
//   chunk_kernel    compositing of every item; single-chunk tiles write the
//                   image directly, multi-chunk tiles write per-chunk state
//   combine_kernel  image (and optional T_final / last) of multi-chunk tiles
// The power / alpha arithmetic is pinned (explicit fmaf / __fmul_rn) so every
// pass that re-evaluates a pair takes bit-identical skip / stop decisions.
#include "render_common.cuh"

namespace gs {

__global__ void __launch_bounds__(1024) plan_kernel(const uint32_t *__restrict__ ranges, int T, int L,
                                                    int max_items, int32_t *__restrict__ item_base,
                                                    const gs_status *st)
{
    __shared__ int s_warp[32];
    __shared__ long long s_carry;
    if (threadIdx.x == 0) s_carry = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const bool err = has_error(st);
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

// Front-to-back state of one pixel.
struct PixFwd {
    float T, C0, C1, C2;
    int last;      // position of the last composited splat (1-based, in the chunk)
    int stop;      // position of the splat that stopped the pixel (0: not stopped)
    bool done;
};

// Eq. 1 step of one pixel over a staged splat at chunk position pos (1-based).
__device__ __forceinline__ void fwd_step(PixFwd &ps, const float4 a, const float4 bb, float cb, float px, float py,
                                         int pos)
{
    float dx, dy;
    const float q = splat_q(a, bb.x, px, py, &dx, &dy);
    if (q > 0.f) return;
    const float alpha = fminf(kAlphaMax, splat_alpha(q, bb.y));
    if (alpha < kAlphaMin) return;
    const float Tn = __fmul_rn(ps.T, 1.f - alpha);
    if (Tn < kTMin) { ps.done = true; ps.stop = pos; return; }
    const float w = __fmul_rn(alpha, ps.T);
    ps.C0 = fmaf(bb.z, w, ps.C0);
    ps.C1 = fmaf(bb.w, w, ps.C1);
    ps.C2 = fmaf(cb, w, ps.C2);
    ps.T = Tn;
    ps.last = pos;
}

// Transmittance product of one chunk (no stop rule; early exit below 1e-4).
// The last chunk of a tile needs none.
__global__ void __launch_bounds__(kRThreads) prod_kernel(const float4 *__restrict__ rec,
                                                         const uint32_t *__restrict__ vals,
                                                         const uint32_t *__restrict__ ranges, ViewTable vt,
                                                         RenderPlan plan, long long cap_cand, const gs_status *st)
{
    if (has_error(st)) return;
    Item it;
    if (!item_of(blockIdx.x, plan.item_base, vt.total_tiles, ranges, plan.L, &it) || it.nk == 1 ||
        it.k == it.nk - 1)
        return;
    __shared__ Staged S;
    const TileCoord tc = tile_coord(vt, it.t);
    const float fpx = (float)tc.px, fy0 = (float)tc.py, fy1 = (float)(tc.py + 1);
    float T0 = 1.f, T1 = 1.f;
    bool d0 = !tc.in0, d1 = !tc.in1;
    const int tid = threadIdx.x, warp = tid >> 5;
    for (uint32_t b0 = it.s0; b0 < it.s1; b0 += kRT) {
        if (__syncthreads_count(d0 && d1) == kRThreads) break;
        stage(S, tid, rec, vals, b0 + tid, b0 + tid < it.s1, cap_cand, st, 43, false);
        stage(S, tid + kRThreads, rec, vals, b0 + tid + kRThreads, b0 + tid + kRThreads < it.s1, cap_cand, st, 43,
              false);
        __syncthreads();
        const int n = (int)min((uint32_t)kRT, it.s1 - b0);
        const int cnt = warp_list(S, n, tc.x0, tc.y0);
        for (int li = 0; li < cnt; ++li) {
            const int j = S.wl[warp][li];
            const float4 a = S.a[j];
            const float4 bb = S.b[j];
            float dx, dy;
            if (!d0) {
                const float q = splat_q(a, bb.x, fpx, fy0, &dx, &dy);
                if (q <= 0.f) {
                    const float alpha = fminf(kAlphaMax, splat_alpha(q, bb.y));
                    if (alpha >= kAlphaMin) {
                        T0 = __fmul_rn(T0, 1.f - alpha);
                        d0 = T0 < kTMin;
                    }
                }
            }
            if (!d1) {
                const float q = splat_q(a, bb.x, fpx, fy1, &dx, &dy);
                if (q <= 0.f) {
                    const float alpha = fminf(kAlphaMax, splat_alpha(q, bb.y));
                    if (alpha >= kAlphaMin) {
                        T1 = __fmul_rn(T1, 1.f - alpha);
                        d1 = T1 < kTMin;
                    }
                }
            }
        }
    }
    float *pl = state_plane(plan.state, it.base + it.k, 0);
    pl[tc.pid0] = T0;
    pl[tc.pid0 + kTile] = T1;
}

__device__ __forceinline__ void write_pixel_or_state(const PixFwd &ps, bool inside, bool multi, int item, int pix,
                                                     const RenderPlan &plan, const ViewTable &vt, int v, int px,
                                                     int py, float bg0, float bg1, float bg2, float *image,
                                                     float *T_final, int32_t *last)
{
    if (multi) {
        state_plane(plan.state, item, 1)[pix] = ps.T;
        state_plane(plan.state, item, 2)[pix] = ps.C0;
        state_plane(plan.state, item, 3)[pix] = ps.C1;
        state_plane(plan.state, item, 4)[pix] = ps.C2;
        reinterpret_cast<int *>(state_plane(plan.state, item, 5))[pix] = ps.last;
        return;
    }
    if (!inside) return;
    const long long W = vt.W[v], H = vt.H[v];
    const long long p = (long long)py * W + px;
    float *img = image + 3 * vt.pix_base[v];
    img[p] = fmaf(ps.T, bg0, ps.C0);
    img[W * H + p] = fmaf(ps.T, bg1, ps.C1);
    img[2 * W * H + p] = fmaf(ps.T, bg2, ps.C2);
    if (T_final) T_final[vt.pix_base[v] + p] = ps.T;
    if (last) last[vt.pix_base[v] + p] = ps.last;
}

// Compositing of one work item.  Each warp walks only the staged splats whose
// alpha box meets its pixel block.  With COUNT, the pairs the method examines
// (every list position up to the stop) and the pairs composited are counted.
template <bool COUNT>
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
    Item it;
    if (!item_of(blockIdx.x, plan.item_base, vt.total_tiles, ranges, plan.L, &it)) return;
    __shared__ Staged S;
    const int tid = threadIdx.x, warp = tid >> 5;
    const TileCoord tc = tile_coord(vt, it.t);
    const float fpx = (float)tc.px, fy0 = (float)tc.py, fy1 = (float)(tc.py + 1);
    const bool multi = it.nk > 1;
    PixFwd p0, p1;
    p0.T = multi ? chunk_T0(plan.state, it, tc.pid0) : 1.f;
    p1.T = multi ? chunk_T0(plan.state, it, tc.pid0 + kTile) : 1.f;
    p0.C0 = p0.C1 = p0.C2 = p1.C0 = p1.C1 = p1.C2 = 0.f;
    p0.last = p1.last = p0.stop = p1.stop = 0;
    p0.done = !tc.in0 || p0.T < kTMin;
    p1.done = !tc.in1 || p1.T < kTMin;
    const bool act0 = !p0.done, act1 = !p1.done;
    for (uint32_t b0 = it.s0; b0 < it.s1; b0 += kRT) {
        if (__syncthreads_count(p0.done && p1.done) == kRThreads) break;
        stage(S, tid, rec, vals, b0 + tid, b0 + tid < it.s1, cap_cand, st, 42, true);
        stage(S, tid + kRThreads, rec, vals, b0 + tid + kRThreads, b0 + tid + kRThreads < it.s1, cap_cand, st, 42,
              true);
        __syncthreads();
        const int n = (int)min((uint32_t)kRT, it.s1 - b0);
        const int base = (int)(b0 - it.s0);
        const int cnt = warp_list(S, n, tc.x0, tc.y0);
        for (int li = 0; li < cnt; ++li) {
            const int j = S.wl[warp][li];
            const float4 a = S.a[j];
            const float4 bb = S.b[j];
            const float cb = S.c[j];
            if (!p0.done) fwd_step(p0, a, bb, cb, fpx, fy0, base + j + 1);
            if (!p1.done) fwd_step(p1, a, bb, cb, fpx, fy1, base + j + 1);
        }
    }
    if (COUNT) {
        const int n_items = (int)(it.s1 - it.s0);
        unsigned long long nev = 0, ncomp = 0;
        if (act0) nev += p0.stop ? p0.stop : n_items;
        if (act1) nev += p1.stop ? p1.stop : n_items;
        // composited pairs: recount over the list (cheap next to the composite itself)
        for (int pass = 0; pass < 2; ++pass) {
            const PixFwd &ps = pass ? p1 : p0;
            if (!(pass ? act1 : act0)) continue;
            float T = multi ? chunk_T0(plan.state, it, tc.pid0 + pass * kTile) : 1.f;
            const float fy = pass ? fy1 : fy0;
            for (int pos = 0; pos < ps.last; ++pos) {
                uint32_t id = vals[it.s0 + pos];
                if (!idx_ok(st, (long long)id, cap_cand, 44)) break;
                const float4 a = __ldg(&rec[3 * (size_t)id]);
                const float4 bb = __ldg(&rec[3 * (size_t)id + 1]);
                float dx, dy;
                const float q = splat_q(a, bb.x, fpx, fy, &dx, &dy);
                if (q > 0.f) continue;
                const float alpha = fminf(kAlphaMax, splat_alpha(q, bb.y));
                if (alpha < kAlphaMin) continue;
                T = __fmul_rn(T, 1.f - alpha);
                ++ncomp;
            }
        }
        for (int o = 16; o > 0; o >>= 1) {
            nev += __shfl_down_sync(0xffffffffu, nev, o);
            ncomp += __shfl_down_sync(0xffffffffu, ncomp, o);
        }
        if ((tid & 31) == 0 && nev) atomicAdd(n_eval, nev);
        if ((tid & 31) == 0 && ncomp) atomicAdd(n_eval + 1, ncomp);
    }
    const int item = it.base + it.k;
    write_pixel_or_state(p0, tc.in0, multi, item, tc.pid0, plan, vt, tc.v, tc.px, tc.py, bg0, bg1, bg2, image,
                         T_final, last);
    write_pixel_or_state(p1, tc.in1, multi, item, tc.pid0 + kTile, plan, vt, tc.v, tc.px, tc.py + 1, bg0, bg1, bg2,
                         image, T_final, last);
}

// Image of a multi-chunk tile: sum of the active chunks' colour plus the final
// transmittance (that of the last active chunk) times the background.
__global__ void __launch_bounds__(kRThreads) combine_kernel(const uint32_t *__restrict__ ranges, ViewTable vt,
                                                            RenderPlan plan, float bg0, float bg1, float bg2,
                                                            float *__restrict__ image, float *__restrict__ T_final,
                                                            int32_t *__restrict__ last, const gs_status *st)
{
    if (has_error(st)) return;
    const int t = blockIdx.x;
    const int base = plan.item_base[t], nk = plan.item_base[t + 1] - base;
    if (nk <= 1) return;
    const TileCoord tc = tile_coord(vt, t);
    for (int half = 0; half < 2; ++half) {
        const bool inside = half ? tc.in1 : tc.in0;
        if (!inside) continue;
        const int pix = tc.pid0 + half * kTile;
        float T0 = 1.f, Tf = 1.f, C0 = 0.f, C1 = 0.f, C2 = 0.f;
        int lastc = 0;
        for (int j = 0; j < nk; ++j) {
            if (!(T0 >= kTMin)) break;
            const int item = base + j;
            C0 += state_plane(plan.state, item, 2)[pix];
            C1 += state_plane(plan.state, item, 3)[pix];
            C2 += state_plane(plan.state, item, 4)[pix];
            Tf = state_plane(plan.state, item, 1)[pix];
            const int lj = reinterpret_cast<const int *>(state_plane(plan.state, item, 5))[pix];
            if (lj > 0) lastc = j * plan.L + lj;
            if (j < nk - 1) T0 = __fmul_rn(T0, state_plane(plan.state, item, 0)[pix]);
        }
        const int v = tc.v;
        const long long W = vt.W[v], H = vt.H[v];
        const long long p = (long long)(tc.py + half) * W + tc.px;
        float *img = image + 3 * vt.pix_base[v];
        img[p] = fmaf(Tf, bg0, C0);
        img[W * H + p] = fmaf(Tf, bg1, C1);
        img[2 * W * H + p] = fmaf(Tf, bg2, C2);
        if (T_final) T_final[vt.pix_base[v] + p] = Tf;
        if (last) last[vt.pix_base[v] + p] = lastc;
    }
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

// ------------------------------------------------------------ launchers
int render_max_items(const ViewTable &vt, long long cap_pairs, int L)
{
    return (int)std::min<long long>((long long)vt.total_tiles + (cap_pairs + L - 1) / L, 1ll << 30);
}

size_t render_workspace_bytes(const ViewTable &vt, long long cap_pairs, int L)
{
    const long long items = render_max_items(vt, cap_pairs, L);
    return align_up(sizeof(int32_t) * ((size_t)vt.total_tiles + 1), 256) +
           align_up(sizeof(float) * (size_t)items * kStateWords * kRT, 256);
}

RenderPlan render_plan(const ViewTable &vt, long long cap_pairs, int L, void *ws)
{
    RenderPlan p;
    p.L = L;
    p.max_items = render_max_items(vt, cap_pairs, L);
    char *w = reinterpret_cast<char *>(ws);
    p.item_base = reinterpret_cast<int32_t *>(w);
    p.state = reinterpret_cast<float *>(w + align_up(sizeof(int32_t) * ((size_t)vt.total_tiles + 1), 256));
    return p;
}

int launch_render_fwd(const gs_splats *sp, const gs_bins *bins, const ViewTable &vt, const float bg[3], int L,
                      void *ws, float *image, float *T_final, int32_t *last, long long *n_eval, gs_status *st,
                      cudaStream_t s)
{
    if (vt.total_tiles == 0) return GS_OK;
    const float4 *rec = reinterpret_cast<const float4 *>(sp->rec);
    const RenderPlan plan = render_plan(vt, bins->cap_pairs, L, ws);
    plan_kernel<<<1, 1024, 0, s>>>(bins->ranges, vt.total_tiles, L, plan.max_items,
                                   const_cast<int32_t *>(plan.item_base), st);
    prod_kernel<<<plan.max_items, kRThreads, 0, s>>>(rec, bins->vals, bins->ranges, vt, plan, sp->cap, st);
    if (n_eval) {
        cudaMemsetAsync(n_eval, 0, 2 * sizeof(long long), s);
        chunk_kernel<true><<<plan.max_items, kRThreads, 0, s>>>(rec, bins->vals, bins->ranges, vt, plan, bg[0], bg[1],
                                                          bg[2], image, T_final, last,
                                                          reinterpret_cast<unsigned long long *>(n_eval), sp->cap, st);
    } else {
        chunk_kernel<false><<<plan.max_items, kRThreads, 0, s>>>(rec, bins->vals, bins->ranges, vt, plan, bg[0], bg[1],
                                                           bg[2], image, T_final, last, nullptr, sp->cap, st);
    }
    combine_kernel<<<vt.total_tiles, kRThreads, 0, s>>>(bins->ranges, vt, plan, bg[0], bg[1], bg[2], image, T_final,
                                                   last, st);
    count_launches(4);
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
