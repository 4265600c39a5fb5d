// gs_internal.cuh -- argument blocks and launchers shared by the .cu files.
#pragma once

#include <algorithm>

#include "gs_common.cuh"

namespace gs {

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

struct DecodeArgs {
    const float *xyz, *feat, *log_scaling, *offsets, *mlp;
    const int32_t *part;
    long long mlp_floats;
    int N, F, k, H, M, V;
    const gs_camera *cams;
    const int32_t *view_start, *row_anchor;
    float *mu, *scale, *quat, *opacity, *colour;
    gs_status *st;
    long long cap_rows;
    unsigned long long wait_ns;   // limit of the tensor-core kernels' MMA completion waits
};

struct DecodeBwdArgsB {
    DecodeArgs f;   // forward inputs (the candidate outputs are not read)
    const float *dmu, *dscale, *dquat, *dopacity, *dcolour;
    float *dxyz, *dfeat, *dls, *doff, *dmlp;
    // fused with the projection's reverse (tcgen05 path): the splat gradients
    // in row tiles, [tile of 128 rows][i < k][9][128 rows] (zero for a
    // candidate that covers no tile), replace the five gradients above (NULL:
    // not fused)
    const float *sgT;
    int W[GS_MAX_VIEWS], H[GS_MAX_VIEWS];
};
int launch_decode_bwd_bf16(const DecodeBwdArgsB &a, cudaStream_t s);

// Splat records written by the decoder itself (decode fused with the
// projection): the output and the views' sizes in pixels and tiles.
struct ProjOut {
    float4 *rec;
    int32_t *tiles;
    long long cap;
    int W[GS_MAX_VIEWS], H[GS_MAX_VIEWS], TX[GS_MAX_VIEWS], TY[GS_MAX_VIEWS];
};

size_t decode_workspace_bytes(int N, int V);
int launch_decode(const gs_anchors *A, const gs_camera *cams, const ViewTable &vt, int precision,
                  gs_gauss3d *out, void *ws, gs_status *st, cudaStream_t s, const gs_splats *proj = nullptr);
int launch_decode_bf16(const DecodeArgs &a, cudaStream_t s, const ProjOut *po = nullptr);

int launch_project(const gs_gauss3d *g, const gs_camera *cams, const ViewTable &vt, gs_splats *out,
                   gs_status *st, cudaStream_t s);

size_t bin_sort_workspace_bytes(const ViewTable &vt, long long cap_cand, long long cap_pairs);
int launch_bin_sort(const gs_splats *sp, int k, const int32_t *view_start, long long cap_rows,
                    const ViewTable &vt, gs_bins *bins, void *ws, size_t ws_bytes, gs_status *st,
                    cudaStream_t s);

struct RenderPlan;
int render_max_items(const ViewTable &vt, long long cap_pairs, int L);
size_t render_workspace_bytes(const ViewTable &vt, long long cap_pairs, int L);
int launch_render_fwd(const gs_splats *sp, const gs_bins *bins, const ViewTable &vt, const float bg[3], int L,
                      void *ws, float *image, float *T_final, int32_t *last, long long *n_eval, gs_status *st,
                      cudaStream_t s);
int launch_l1(const float *image, const float *target, const ViewTable &vt, float *loss, float *d_image,
              cudaStream_t s);
size_t photometric_workspace_bytes(const ViewTable &vt);
size_t voxelize_workspace_bytes(long long P);
size_t flow_workspace_bytes(int N);
int launch_flow_triangulate(const gs_camera *c1, const gs_camera *c2, int W, int H, const float *flow,
                            const int32_t *samples, int N, double tau, float *residual, int32_t *kept, float *points,
                            long long cap, uint32_t *n_kept, void *ws, gs_status *st, cudaStream_t s);
int launch_voxelize(const float *pts, long long P, float eps, const unsigned long long *existing, long long n_ex,
                    unsigned long long *keys_out, float *centers_out, long long cap, uint32_t *n_out, void *ws,
                    gs_status *st, cudaStream_t s);
int launch_loop_closure(float *xyz, int N, const gs_camera *old_cams, const gs_camera *new_cams, const int32_t *wh,
                        int K, float z_far, int32_t *assigned, cudaStream_t s);
int launch_adam(const gs_adam_group *groups, int ng, long long step, double b1, double b2, double eps, cudaStream_t s);
int launch_densify_stats(const gs_gauss3d *g, int V, const int32_t *tiles, const float *sgrad, int N,
                         float *grad_accum, int32_t *offset_denom, float *opacity_accum, int32_t *anchor_denom,
                         gs_status *st, cudaStream_t s);
int launch_densify_masks(long long N, int k, const float *grad_accum, const int32_t *offset_denom,
                         const float *opacity_accum, const int32_t *anchor_denom, float grad_thr, float opacity_thr,
                         int min_count, uint8_t *grow, uint8_t *prune, cudaStream_t s);
int launch_photometric(const float *image, const float *target, const ViewTable &vt, float lam, void *ws,
                       float *loss, float *d_image, cudaStream_t s);
int launch_render_bwd(const gs_gauss3d *g, const gs_camera *cams, const gs_splats *sp, const gs_bins *bins,
                      const ViewTable &vt, int L, void *ws, const float *image, const float *d_image,
                      const int32_t *last, gs_splat_grad *sgrad, gs_gauss3d_grad *out, gs_status *st,
                      cudaStream_t s);
int launch_project_bwd(const gs_gauss3d *g, const gs_camera *cams, const gs_splats *sp, const ViewTable &vt,
                       const gs_splat_grad *sgrad, gs_gauss3d_grad *out, gs_status *st, cudaStream_t s);

size_t decode_bwd_workspace_bytes(int N, int V, int M, long long cap_rows);
size_t decode_project_bwd_workspace_bytes(int k, long long cap_rows, int precision);
int launch_decode_project_bwd(const gs_anchors *A, const gs_camera *cams, const ViewTable &vt, int precision,
                              const gs_gauss3d *g, const gs_splats *sp, const gs_splat_grad *sgrad,
                              gs_anchor_grad *out, void *ws, gs_status *st, cudaStream_t s);
int launch_decode_bwd(const gs_anchors *A, const gs_camera *cams, const ViewTable &vt, int precision,
                      const gs_gauss3d *g, const gs_gauss3d_grad *dg, gs_anchor_grad *out, void *ws,
                      gs_status *st, cudaStream_t s);

}  // namespace gs
