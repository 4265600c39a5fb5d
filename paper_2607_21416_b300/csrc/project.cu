// project.cu -- EWA projection of candidate Gaussians to 2D splat records.
//
// One thread per candidate (grid-stride over the device-side candidate count).
// Each writes a 48-byte record (mean, conic, opacity, colour, depth, tile
// rectangle) and its tile count; culled candidates get an empty rectangle.
// Near-degenerate splats (det < 1e-3 a c from the FP32 covariance) have
// their covariance formed again in compensated single precision
// (cov2d_f2.cuh) and its determinant and conic taken in FP64; everything
// else is FP32.
#include "proj_fwd.cuh"

namespace gs {

struct ProjectArgs {
    const float *mu, *scale, *quat, *opacity, *colour;
    const int32_t *view_start;
    const gs_camera *cams;
    int k, V;
    long long cap_cand;
    float4 *rec;
    int32_t *tiles;
    const gs_status *st;
};


__global__ void __launch_bounds__(256) project_kernel(ProjectArgs a, ViewTable vt)
{
    if (has_error(a.st)) return;
    const long long rows = __ldg(a.view_start + a.V);
    const long long C = std::min<long long>(rows * a.k, a.cap_cand);
    for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < C;
         c += (long long)gridDim.x * blockDim.x) {
        float4 r0 = make_float4(0.f, 0.f, 0.f, 0.f), r1 = r0, r2 = r0;
        int ntiles = 0;
        const float op = __ldg(a.opacity + c);
        const int v = view_of_row(a.view_start, a.V, (int)(c / a.k));
        const Cam cm = load_cam(a.cams, v);
        const float mx_ = __ldg(a.mu + 3 * c), my_ = __ldg(a.mu + 3 * c + 1), mz_ = __ldg(a.mu + 3 * c + 2);
        const float sc[3] = {__ldg(a.scale + 3 * c), __ldg(a.scale + 3 * c + 1), __ldg(a.scale + 3 * c + 2)};
        const float q[4] = {__ldg(a.quat + 4 * c), __ldg(a.quat + 4 * c + 1), __ldg(a.quat + 4 * c + 2),
                            __ldg(a.quat + 4 * c + 3)};
        const float col[3] = {__ldg(a.colour + 3 * c), __ldg(a.colour + 3 * c + 1), __ldg(a.colour + 3 * c + 2)};
        project_one(cm, (float)vt.W[v], (float)vt.H[v], vt.TX[v], vt.TY[v], mx_, my_, mz_, sc, q, op, col, r0, r1, r2,
                    ntiles);
        a.rec[3 * c] = r0;
        a.rec[3 * c + 1] = r1;
        a.rec[3 * c + 2] = r2;
        a.tiles[c] = ntiles;
    }
}

int launch_project(const gs_gauss3d *g, const gs_camera *cams, const ViewTable &vt, gs_splats *out,
                   gs_status *st, cudaStream_t s)
{
    ProjectArgs a;
    a.mu = g->mu; a.scale = g->scale; a.quat = g->quat; a.opacity = g->opacity; a.colour = g->colour;
    a.view_start = g->view_start; a.cams = cams; a.k = g->k; a.V = vt.V;
    a.cap_cand = g->cap_rows * (long long)g->k;
    a.rec = reinterpret_cast<float4 *>(out->rec); a.tiles = out->tiles; a.st = st;
    const long long need = (a.cap_cand + 255) / 256;
    const int grid = (int)std::max<long long>(1, std::min<long long>(need, (long long)sm_count() * 16));
    project_kernel<<<grid, 256, 0, s>>>(a, vt);
    count_launches(1);
    return cudaPeekAtLastError() == cudaSuccess ? GS_OK : GS_ERR_CUDA;
}

}  // namespace gs
