// maintenance.cu -- loop-closure deformation of the anchor grid (Eq. 7).
//
// For each corrected keyframe i, Delta T_i = T_new,i^-1 T_old,i maps an
// anchor x to R_new^T (R_old x + t_old - t_new).  It applies to the anchors
// inside keyframe i's local view frustum -- the decoder's visibility rule
// under the old pose (in front of the near plane, inside the image grown by
// 15 % per side) cut at depth z_far -- and an anchor inside several frusta
// takes the nearest keyframe (distance to the old camera centre, lowest index
// on ties).  One thread per anchor; the keyframes are staged through shared
// memory 128 at a time.
#include "gs_internal.cuh"

namespace gs {

constexpr int kLcThreads = 256;
constexpr int kLcStage = 128;   // keyframes per shared-memory round

__global__ void __launch_bounds__(kLcThreads) loop_closure_kernel(float *__restrict__ xyz, int N,
                                                                  const gs_camera *__restrict__ old_cams,
                                                                  const gs_camera *__restrict__ new_cams,
                                                                  const int32_t *__restrict__ wh, int K, float z_far,
                                                                  int32_t *__restrict__ assigned)
{
    __shared__ float s_cam[kLcStage][16];
    __shared__ float s_lim[kLcStage][4];   // u and v limits of the grown image
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    const bool live = a < N;
    float x = 0.f, y = 0.f, z = 0.f;
    if (live) { x = xyz[3 * (size_t)a]; y = xyz[3 * (size_t)a + 1]; z = xyz[3 * (size_t)a + 2]; }
    int best = -1;
    float bd = 0.f;
    for (int k0 = 0; k0 < K; k0 += kLcStage) {
        const int nk = min(kLcStage, K - k0);
        __syncthreads();
        for (int i = threadIdx.x; i < nk * 16; i += blockDim.x)
            s_cam[i >> 4][i & 15] = __ldg(reinterpret_cast<const float *>(old_cams + k0 + (i >> 4)) + (i & 15));
        for (int i = threadIdx.x; i < nk; i += blockDim.x) {
            const float W = (float)__ldg(wh + 2 * (k0 + i)), H = (float)__ldg(wh + 2 * (k0 + i) + 1);
            s_lim[i][0] = -kMargin * W;
            s_lim[i][1] = (1.0f + kMargin) * W;
            s_lim[i][2] = -kMargin * H;
            s_lim[i][3] = (1.0f + kMargin) * H;
        }
        __syncthreads();
        if (!live) continue;
        for (int i = 0; i < nk; ++i) {
            const float *c = s_cam[i];
            const float pz = fmaf(c[12], z, fmaf(c[11], y, fmaf(c[10], x, c[15])));
            if (!(pz > kNear && pz <= z_far)) continue;
            const float px = fmaf(c[6], z, fmaf(c[5], y, fmaf(c[4], x, c[13])));
            const float py = fmaf(c[9], z, fmaf(c[8], y, fmaf(c[7], x, c[14])));
            const float u = fmaf(c[0], __fdiv_rn(px, pz), c[2]);
            const float v = fmaf(c[1], __fdiv_rn(py, pz), c[3]);
            if (!(u >= s_lim[i][0] && u < s_lim[i][1] && v >= s_lim[i][2] && v < s_lim[i][3])) continue;
            const float d = fmaf(px, px, fmaf(py, py, pz * pz));
            if (best < 0 || d < bd) {
                best = k0 + i;
                bd = d;
            }
        }
    }
    if (!live) return;
    if (best >= 0) {
        const Cam o = load_cam(old_cams, best), n = load_cam(new_cams, best);
        const float q0 = fmaf(o.R[2], z, fmaf(o.R[1], y, fmaf(o.R[0], x, o.t[0]))) - n.t[0];
        const float q1 = fmaf(o.R[5], z, fmaf(o.R[4], y, fmaf(o.R[3], x, o.t[1]))) - n.t[1];
        const float q2 = fmaf(o.R[8], z, fmaf(o.R[7], y, fmaf(o.R[6], x, o.t[2]))) - n.t[2];
        xyz[3 * (size_t)a] = fmaf(n.R[6], q2, fmaf(n.R[3], q1, n.R[0] * q0));
        xyz[3 * (size_t)a + 1] = fmaf(n.R[7], q2, fmaf(n.R[4], q1, n.R[1] * q0));
        xyz[3 * (size_t)a + 2] = fmaf(n.R[8], q2, fmaf(n.R[5], q1, n.R[2] * q0));
    }
    if (assigned) assigned[a] = best;
}

int launch_loop_closure(float *xyz, int N, const gs_camera *old_cams, const gs_camera *new_cams, const int32_t *wh,
                        int K, float z_far, int32_t *assigned, cudaStream_t s)
{
    if (N == 0) return GS_OK;
    loop_closure_kernel<<<(N + kLcThreads - 1) / kLcThreads, kLcThreads, 0, s>>>(xyz, N, old_cams, new_cams, wh, K,
                                                                                z_far, assigned);
    count_launches(1);
    return cudaPeekAtLastError() == cudaSuccess ? GS_OK : GS_ERR_CUDA;
}

}  // namespace gs
