// gs_api.cu -- extern "C" entry points of libgs: argument checks, view
// tables and dispatch to the kernels.  Nothing here allocates or syncs.
#include <atomic>
#include <cstring>
#include <mutex>

#include "gs_internal.cuh"

namespace gs {

bool make_view_table(const gs_view *views, int V, ViewTable *vt)
{
    if (V < 1 || V > GS_MAX_VIEWS || !views) return false;
    std::memset(vt, 0, sizeof(*vt));
    vt->V = V;
    long long tb = 0, pb = 0;
    for (int v = 0; v < V; ++v) {
        const int W = views[v].width, H = views[v].height;
        if (W <= 0 || H <= 0 || W > 65535 * kTile || H > 65535 * kTile) return false;
        vt->W[v] = W; vt->H[v] = H;
        vt->TX[v] = (W + kTile - 1) / kTile;
        vt->TY[v] = (H + kTile - 1) / kTile;
        vt->tile_base[v] = (int)tb;
        vt->pix_base[v] = pb;
        tb += (long long)vt->TX[v] * vt->TY[v];
        pb += (long long)W * H;
        if (tb > (1ll << 30)) return false;
    }
    vt->tile_base[V] = (int)tb;
    vt->pix_base[V] = pb;
    vt->total_tiles = (int)tb;
    vt->total_pixels = pb;
    return true;
}

static std::atomic<unsigned long long> g_launches{0};
void count_launches(int n) { g_launches.fetch_add((unsigned long long)n, std::memory_order_relaxed); }

static std::atomic<unsigned long long> g_wait_ns{kDefaultWaitNs};
unsigned long long wait_limit_ns() { return g_wait_ns.load(std::memory_order_relaxed); }

static std::mutex g_tuning_mu;
static gs_tuning g_tuning{0, 0, 0, 0};
gs_tuning tuning()
{
    std::lock_guard<std::mutex> lock(g_tuning_mu);
    return g_tuning;
}

int sm_count()
{
    static int cache[64] = {0};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) dev = 0;
    if (!cache[dev]) {
        int n = 0;
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        cache[dev] = n > 0 ? n : 1;
    }
    return cache[dev];
}

}  // namespace gs

using namespace gs;

static bool check_anchors(const gs_anchors *A)
{
    if (!A || A->N < 0 || A->F < 1 || A->F > 64 || A->k < 1 || A->k > 16 || A->hidden < 1 || A->hidden > 64 ||
        A->M < 1)
        return false;
    if (A->N > 0 && (!A->xyz || !A->feat || !A->log_scaling || !A->offsets || !A->part || !A->mlp)) return false;
    return true;
}

static bool check_gauss(const gs_gauss3d *g)
{
    return g && g->k >= 1 && g->cap_rows >= 0 && g->view_start && g->mu && g->scale && g->quat && g->opacity &&
           g->colour && g->cap_rows * (long long)g->k < (1ll << 31);
}

extern "C" {

uint64_t gs_kernel_launches(void) { return (uint64_t)g_launches.load(std::memory_order_relaxed); }

int gs_set_tuning(const gs_tuning *t)
{
    if (t && (t->fwd_ctas_per_sm < 0 || t->bwd_ctas_per_sm < 0 || t->sort_ctas_per_sm < 0 || t->emit_ctas_per_sm < 0))
        return GS_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lock(g_tuning_mu);
    g_tuning = t ? *t : gs_tuning{0, 0, 0, 0};
    return GS_OK;
}

int gs_get_tuning(gs_tuning *t)
{
    if (!t) return GS_ERR_INVALID_ARG;
    *t = tuning();
    return GS_OK;
}

int gs_set_wait_limit(int64_t ns)
{
    g_wait_ns.store(ns < 0 ? kDefaultWaitNs : (unsigned long long)ns, std::memory_order_relaxed);
    return GS_OK;
}

int64_t gs_mlp_floats(int32_t F, int32_t k, int32_t hidden)
{
    const int64_t din = F + 4;
    const int64_t douts[3] = {k, 3 * (int64_t)k, 7 * (int64_t)k};
    int64_t s = 0;
    for (int i = 0; i < 3; ++i) s += hidden * din + hidden + douts[i] * hidden + douts[i];
    return s;
}

int64_t gs_total_tiles(const gs_view *views, int32_t V)
{
    ViewTable vt;
    return make_view_table(views, V, &vt) ? vt.total_tiles : -1;
}

int64_t gs_total_pixels(const gs_view *views, int32_t V)
{
    ViewTable vt;
    return make_view_table(views, V, &vt) ? vt.total_pixels : -1;
}

size_t gs_decode_workspace(int32_t N, int32_t V, int32_t M, int64_t cap_rows)
{
    (void)M; (void)cap_rows;
    return decode_workspace_bytes(N, V);
}

size_t gs_bin_sort_workspace(const gs_view *views, int32_t V, int64_t cap_cand, int64_t cap_pairs)
{
    ViewTable vt;
    if (!make_view_table(views, V, &vt)) return 0;
    return bin_sort_workspace_bytes(vt, cap_cand, cap_pairs);
}

size_t gs_decode_bwd_workspace(int32_t N, int32_t V, int32_t M, int64_t cap_rows)
{
    return decode_bwd_workspace_bytes(N, V, M, cap_rows);
}

const char *gs_status_string(int32_t code)
{
    switch (code) {
    case GS_OK: return "ok";
    case GS_ERR_INVALID_ARG: return "invalid argument";
    case GS_ERR_CAPACITY: return "capacity exceeded";
    case GS_ERR_CUDA: return "CUDA error";
    case GS_ERR_TIMEOUT: return "bounded wait timed out";
    case GS_ERR_UNSUPPORTED: return "unsupported configuration";
    default: return "unknown status";
    }
}

int gs_decode(const gs_anchors *A, const gs_camera *cams, const gs_view *views, int32_t V, int32_t precision,
              gs_gauss3d *out, void *ws, size_t ws_bytes, gs_status *status, void *stream)
{
    ViewTable vt;
    if (!check_anchors(A) || !cams || !status || !check_gauss(out) || !out->row_anchor ||
        !make_view_table(views, V, &vt) || out->k != A->k)
        return GS_ERR_INVALID_ARG;
    if (precision != GS_PREC_FP32 && precision != GS_PREC_BF16) return GS_ERR_INVALID_ARG;
    if (ws_bytes < decode_workspace_bytes(A->N, V) || (!ws && ws_bytes > 0)) return GS_ERR_INVALID_ARG;
    return launch_decode(A, cams, vt, precision, out, ws, status, (cudaStream_t)stream);
}

int gs_decode_project(const gs_anchors *A, const gs_camera *cams, const gs_view *views, int32_t V,
                      int32_t precision, gs_gauss3d *g, gs_splats *sp, void *ws, size_t ws_bytes, gs_status *status,
                      void *stream)
{
    ViewTable vt;
    if (!check_anchors(A) || !cams || !status || !check_gauss(g) || !g->row_anchor ||
        !make_view_table(views, V, &vt) || g->k != A->k || !sp || !sp->rec || !sp->tiles)
        return GS_ERR_INVALID_ARG;
    if (precision != GS_PREC_FP32 && precision != GS_PREC_BF16) return GS_ERR_INVALID_ARG;
    if ((reinterpret_cast<uintptr_t>(sp->rec) & 15) != 0 || sp->cap < g->cap_rows * (long long)g->k)
        return GS_ERR_INVALID_ARG;
    if (ws_bytes < decode_workspace_bytes(A->N, V) || (!ws && ws_bytes > 0)) return GS_ERR_INVALID_ARG;
    return launch_decode(A, cams, vt, precision, g, ws, status, (cudaStream_t)stream, sp);
}

int gs_project(const gs_gauss3d *g, const gs_camera *cams, const gs_view *views, int32_t V, gs_splats *out,
               gs_status *status, void *stream)
{
    ViewTable vt;
    if (!check_gauss(g) || !cams || !out || !out->rec || !out->tiles || !status || !make_view_table(views, V, &vt))
        return GS_ERR_INVALID_ARG;
    if ((reinterpret_cast<uintptr_t>(out->rec) & 15) != 0 || out->cap < g->cap_rows * (long long)g->k)
        return GS_ERR_INVALID_ARG;
    return launch_project(g, cams, vt, out, status, (cudaStream_t)stream);
}

int gs_bin_sort(const gs_splats *sp, int32_t k, const int32_t *view_start, int64_t cap_rows, const gs_view *views,
                int32_t V, gs_bins *bins, void *ws, size_t ws_bytes, gs_status *status, void *stream)
{
    ViewTable vt;
    if (!sp || !sp->rec || !sp->tiles || k < 1 || !view_start || cap_rows < 0 || !bins || !bins->vals ||
        !bins->ranges || !bins->n_pairs || bins->cap_pairs < 0 || bins->cap_pairs > 0xffffffffll || !status ||
        !make_view_table(views, V, &vt) || cap_rows * (long long)k >= (1ll << 31))
        return GS_ERR_INVALID_ARG;
    if (!ws || sp->cap < cap_rows * (long long)k || (reinterpret_cast<uintptr_t>(sp->rec) & 15) != 0)
        return GS_ERR_INVALID_ARG;
    return launch_bin_sort(sp, k, view_start, cap_rows, vt, bins, ws, ws_bytes, status, (cudaStream_t)stream);
}

static int chunk_len(int32_t chunk) { return chunk == 0 ? 384 : chunk; }

size_t gs_render_workspace(const gs_view *views, int32_t V, int64_t cap_pairs, int32_t chunk)
{
    ViewTable vt;
    if (!make_view_table(views, V, &vt) || cap_pairs < 0 || (chunk != 0 && (chunk < 256 || chunk > (1 << 24))))
        return 0;
    return render_workspace_bytes(vt, cap_pairs, chunk_len(chunk));
}

int gs_render_fwd(const gs_splats *sp, const gs_bins *bins, const gs_view *views, int32_t V, const float *bg,
                  int32_t chunk, void *ws, size_t ws_bytes, float *image, float *T_final, int32_t *last,
                  int64_t *n_eval, gs_status *status, void *stream)
{
    ViewTable vt;
    if (!sp || !sp->rec || !bins || !bins->vals || !bins->ranges || !bins->n_pairs || !bg || !image || !status ||
        !make_view_table(views, V, &vt) || (T_final == nullptr) != (last == nullptr))
        return GS_ERR_INVALID_ARG;
    if ((chunk != 0 && (chunk < 256 || chunk > (1 << 24))) || !ws ||
        (reinterpret_cast<uintptr_t>(ws) & 255) != 0 ||
        ws_bytes < render_workspace_bytes(vt, bins->cap_pairs, chunk_len(chunk)))
        return GS_ERR_INVALID_ARG;
    return launch_render_fwd(sp, bins, vt, bg, chunk_len(chunk), ws, image, T_final, last,
                             reinterpret_cast<long long *>(n_eval), status, (cudaStream_t)stream);
}

int gs_l1_loss(const float *image, const float *target, const gs_view *views, int32_t V, float *loss,
               float *d_image, void *stream)
{
    ViewTable vt;
    if (!image || !target || !loss || !d_image || !make_view_table(views, V, &vt)) return GS_ERR_INVALID_ARG;
    return launch_l1(image, target, vt, loss, d_image, (cudaStream_t)stream);
}

size_t gs_photometric_workspace(const gs_view *views, int32_t V)
{
    ViewTable vt;
    return make_view_table(views, V, &vt) ? photometric_workspace_bytes(vt) : 0;
}

int gs_photometric_loss(const float *image, const float *target, const gs_view *views, int32_t V, float lambda,
                        void *ws, size_t ws_bytes, float *loss, float *d_image, void *stream)
{
    ViewTable vt;
    if (!image || !target || !loss || !d_image || !make_view_table(views, V, &vt)) return GS_ERR_INVALID_ARG;
    if (!(lambda >= 0.f && lambda <= 1.f) || !ws || (reinterpret_cast<uintptr_t>(ws) & 255) != 0 ||
        ws_bytes < photometric_workspace_bytes(vt))
        return GS_ERR_INVALID_ARG;
    return launch_photometric(image, target, vt, lambda, ws, loss, d_image, (cudaStream_t)stream);
}

int gs_adam_step(const gs_adam_group *groups, int32_t n_groups, int64_t step, double beta1, double beta2, double eps,
                 void *stream)
{
    if (!groups || n_groups < 1 || n_groups > GS_ADAM_MAX_GROUPS || step < 1) return GS_ERR_INVALID_ARG;
    if (!(beta1 >= 0.0 && beta1 < 1.0) || !(beta2 >= 0.0 && beta2 < 1.0) || !(eps >= 0.0)) return GS_ERR_INVALID_ARG;
    for (int i = 0; i < n_groups; ++i) {
        const gs_adam_group &g = groups[i];
        if (g.n < 0 || (g.n > 0 && (!g.param || !g.grad || !g.m || !g.v))) return GS_ERR_INVALID_ARG;
    }
    return launch_adam(groups, n_groups, step, beta1, beta2, eps, (cudaStream_t)stream);
}

int gs_densify_stats(const gs_gauss3d *g, int32_t V, const int32_t *tiles, const float *sgrad, int32_t N,
                     float *grad_accum, int32_t *offset_denom, float *opacity_accum, int32_t *anchor_denom,
                     gs_status *status, void *stream)
{
    if (!g || !g->row_anchor || !g->view_start || !g->opacity || g->k < 1 || g->cap_rows < 0 || V < 1 ||
        V > GS_MAX_VIEWS || !tiles || !sgrad || N < 0 || !grad_accum || !offset_denom || !opacity_accum ||
        !anchor_denom || !status)
        return GS_ERR_INVALID_ARG;
    return launch_densify_stats(g, V, tiles, sgrad, N, grad_accum, offset_denom, opacity_accum, anchor_denom, status,
                                (cudaStream_t)stream);
}

int gs_densify_masks(int64_t N, int32_t k, const float *grad_accum, const int32_t *offset_denom,
                     const float *opacity_accum, const int32_t *anchor_denom, float grad_thr, float opacity_thr,
                     int32_t min_count, uint8_t *grow, uint8_t *prune, void *stream)
{
    if (N < 0 || k < 1 || !grad_accum || !offset_denom || !opacity_accum || !anchor_denom || !grow || !prune)
        return GS_ERR_INVALID_ARG;
    if (N == 0) return GS_OK;
    return launch_densify_masks(N, k, grad_accum, offset_denom, opacity_accum, anchor_denom, grad_thr, opacity_thr,
                                min_count, grow, prune, (cudaStream_t)stream);
}

size_t gs_voxelize_workspace(int64_t P) { return P < 0 ? 0 : voxelize_workspace_bytes(P); }

int gs_voxelize(const float *points, int64_t P, float eps, const uint64_t *existing, int64_t n_existing,
                uint64_t *keys_out, float *centers_out, int64_t cap_out, uint32_t *n_out, void *ws, size_t ws_bytes,
                gs_status *status, void *stream)
{
    if (P < 0 || P >= (1ll << 31) || (P > 0 && !points) || !(eps > 0.f) || n_existing < 0 ||
        (n_existing > 0 && !existing) || cap_out < 0 || !keys_out || !centers_out || !n_out || !status || !ws ||
        (reinterpret_cast<uintptr_t>(ws) & 255) != 0 || ws_bytes < voxelize_workspace_bytes(P))
        return GS_ERR_INVALID_ARG;
    return launch_voxelize(points, P, eps, reinterpret_cast<const unsigned long long *>(existing), n_existing,
                           reinterpret_cast<unsigned long long *>(keys_out), centers_out, cap_out, n_out, ws, status,
                           (cudaStream_t)stream);
}

int gs_loop_closure(float *xyz, int32_t N, const gs_camera *old_cams, const gs_camera *new_cams, const int32_t *wh,
                    int32_t K, float z_far, int32_t *assigned, void *stream)
{
    if (N < 0 || (N > 0 && !xyz) || K < 1 || !old_cams || !new_cams || !wh || !(z_far > 0.f))
        return GS_ERR_INVALID_ARG;
    return launch_loop_closure(xyz, N, old_cams, new_cams, wh, K, z_far, assigned, (cudaStream_t)stream);
}

size_t gs_flow_workspace(int32_t N) { return N < 0 ? 0 : flow_workspace_bytes(N); }

int gs_flow_triangulate(const gs_camera *cam1, const gs_camera *cam2, int32_t width, int32_t height, const float *flow,
                        const int32_t *samples, int32_t N, double tau, float *residual, int32_t *kept, float *points,
                        int64_t cap, uint32_t *n_kept, void *ws, size_t ws_bytes, gs_status *status, void *stream)
{
    if (!cam1 || !cam2 || width < 1 || height < 1 || (long long)width * height >= (1ll << 31) || !flow || N < 0 ||
        (N > 0 && !samples) || !(tau >= 0.0) || cap < 0 || !kept || !points || !n_kept || !status || !ws ||
        (reinterpret_cast<uintptr_t>(ws) & 255) != 0 || ws_bytes < flow_workspace_bytes(N))
        return GS_ERR_INVALID_ARG;
    return launch_flow_triangulate(cam1, cam2, width, height, flow, samples, N, tau, residual, kept, points, cap,
                                   n_kept, ws, status, (cudaStream_t)stream);
}

int gs_render_bwd(const gs_gauss3d *g, const gs_camera *cams, const gs_splats *sp, const gs_bins *bins,
                  const gs_view *views, int32_t V, int32_t chunk, void *ws, size_t ws_bytes, const float *image,
                  const float *d_image, const int32_t *last, gs_splat_grad *sgrad, gs_gauss3d_grad *out,
                  gs_status *status, void *stream)
{
    ViewTable vt;
    if (!check_gauss(g) || !cams || !sp || !sp->rec || !sp->tiles || !bins || !bins->vals || !bins->ranges ||
        !bins->n_pairs || !image || !d_image || !sgrad || !sgrad->g ||
        (sgrad->layout != GS_SGRAD_CANDIDATE && sgrad->layout != GS_SGRAD_ROW_TILES) ||
        (out && (sgrad->layout != GS_SGRAD_CANDIDATE || !out->dmu || !out->dscale || !out->dquat || !out->dopacity ||
                 !out->dcolour)) ||
        !status || !make_view_table(views, V, &vt) || sp->cap < g->cap_rows * (long long)g->k)
        return GS_ERR_INVALID_ARG;
    if ((chunk != 0 && (chunk < 256 || chunk > (1 << 24))) || !ws ||
        (reinterpret_cast<uintptr_t>(ws) & 255) != 0 ||
        ws_bytes < render_workspace_bytes(vt, bins->cap_pairs, chunk_len(chunk)))
        return GS_ERR_INVALID_ARG;
    return launch_render_bwd(g, cams, sp, bins, vt, chunk_len(chunk), ws, image, d_image, last, sgrad, out, status,
                             (cudaStream_t)stream);
}

int gs_project_bwd(const gs_gauss3d *g, const gs_camera *cams, const gs_splats *sp, const gs_view *views,
                   int32_t V, const gs_splat_grad *sgrad, gs_gauss3d_grad *out, gs_status *status, void *stream)
{
    ViewTable vt;
    if (!check_gauss(g) || !cams || !sp || !sp->tiles || !sgrad || !sgrad->g ||
        sgrad->layout != GS_SGRAD_CANDIDATE || !out || !out->dmu || !out->dscale || !out->dquat || !out->dopacity ||
        !out->dcolour || !status || !make_view_table(views, V, &vt) || sp->cap < g->cap_rows * (long long)g->k)
        return GS_ERR_INVALID_ARG;
    return launch_project_bwd(g, cams, sp, vt, sgrad, out, status, (cudaStream_t)stream);
}

size_t gs_decode_project_bwd_workspace(int32_t k, int64_t cap_rows, int32_t precision)
{
    return decode_project_bwd_workspace_bytes(k, cap_rows, precision);
}

int gs_decode_project_bwd(const gs_anchors *A, const gs_camera *cams, const gs_view *views, int32_t V,
                          int32_t precision, const gs_gauss3d *g, const gs_splats *sp, const gs_splat_grad *sgrad,
                          gs_anchor_grad *out, void *ws, size_t ws_bytes, gs_status *status, void *stream)
{
    ViewTable vt;
    if (!check_anchors(A) || !cams || !check_gauss(g) || !g->row_anchor || !sp || !sp->tiles || !sgrad ||
        !sgrad->g || !out || !out->dxyz || !out->dfeat || !out->dlog_scaling || !out->doffsets || !out->dmlp ||
        !status || !make_view_table(views, V, &vt) || g->k != A->k || sp->cap < g->cap_rows * (long long)g->k)
        return GS_ERR_INVALID_ARG;
    if (precision != GS_PREC_FP32 && precision != GS_PREC_BF16) return GS_ERR_INVALID_ARG;
    if (sgrad->layout != GS_SGRAD_CANDIDATE &&
        (sgrad->layout != GS_SGRAD_ROW_TILES || precision != GS_PREC_BF16))
        return GS_ERR_INVALID_ARG;
    const bool needs_ws = sgrad->layout == GS_SGRAD_CANDIDATE;   // the row-tiled gradients are read in place
    if ((needs_ws && ws_bytes < decode_project_bwd_workspace_bytes(g->k, g->cap_rows, precision)) ||
        (needs_ws && ws_bytes > 0 && (!ws || (reinterpret_cast<uintptr_t>(ws) & 255) != 0)))
        return GS_ERR_INVALID_ARG;
    return launch_decode_project_bwd(A, cams, vt, precision, g, sp, sgrad, out, ws, status, (cudaStream_t)stream);
}

int gs_decode_bwd(const gs_anchors *A, const gs_camera *cams, const gs_view *views, int32_t V, int32_t precision,
                  const gs_gauss3d *g, const gs_gauss3d_grad *dg, gs_anchor_grad *out, void *ws, size_t ws_bytes,
                  gs_status *status, void *stream)
{
    ViewTable vt;
    if (!check_anchors(A) || !cams || !check_gauss(g) || !g->row_anchor || !dg || !dg->dmu || !dg->dscale ||
        !dg->dquat || !dg->dopacity || !dg->dcolour || !out || !out->dxyz || !out->dfeat || !out->dlog_scaling ||
        !out->doffsets || !out->dmlp || !status || !make_view_table(views, V, &vt) || g->k != A->k)
        return GS_ERR_INVALID_ARG;
    if (precision != GS_PREC_FP32 && precision != GS_PREC_BF16) return GS_ERR_INVALID_ARG;
    if (ws_bytes < decode_bwd_workspace_bytes(A->N, V, A->M, g->cap_rows)) return GS_ERR_INVALID_ARG;
    return launch_decode_bwd(A, cams, vt, precision, g, dg, out, ws, status, (cudaStream_t)stream);
}

}  // extern "C"
