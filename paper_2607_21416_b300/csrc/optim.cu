// optim.cu -- the optimizer step and the densification statistics that follow
// the reverse pass in a mapping iteration (Sec. III, "System Overview": the
// Gaussian optimisation refines, densifies and prunes the anchor map to
// minimise Eq. 3; the growth / pruning rules are those of the incremental
// Scaffold-GS the paper adopts).
//
//   adam_kernel           one launch over up to GS_ADAM_MAX_GROUPS parameter
//                         tensors, each with its own learning rate; a CTA owns
//                         4096 consecutive elements of one tensor (16-byte
//                         vectors when the tensor's four arrays are aligned)
//   densify_stats_kernel  one thread per decoded row: per-offset rendered
//                         counts and gradient norms of the projected mean,
//                         per-anchor visible counts and opacity sums
//   densify_masks_kernel  growth / pruning candidates from the statistics
#include <cmath>

#include "gs_internal.cuh"

namespace gs {

constexpr int kAdamThreads = 256;
constexpr int kAdamChunk = kAdamThreads * 4 * 4;   // elements per CTA

struct AdamTable {
    float *p[GS_ADAM_MAX_GROUPS];
    const float *g[GS_ADAM_MAX_GROUPS];
    float *m[GS_ADAM_MAX_GROUPS];
    float *v[GS_ADAM_MAX_GROUPS];
    long long n[GS_ADAM_MAX_GROUPS];
    float step_size[GS_ADAM_MAX_GROUPS];   // lr / (1 - b1^t)
    int vec[GS_ADAM_MAX_GROUPS];           // all four arrays 16-byte aligned
    int block_base[GS_ADAM_MAX_GROUPS + 1];
    int ng;
};

// Scalars of one step: betas and their complements (formed in double on the
// host), eps, 1 / sqrt(1 - b2^t).
struct AdamScalars {
    float b1, omb1, b2, omb2, eps, inv_sqrt_bc2;
};

__device__ __forceinline__ void adam_one(float &p, float g, float &m, float &v, const AdamScalars &a, float step_size)
{
    m = fmaf(a.b1, m, a.omb1 * g);
    v = fmaf(a.b2, v, a.omb2 * g * g);
    p -= step_size * m / fmaf(sqrtf(v), a.inv_sqrt_bc2, a.eps);
}

__global__ void __launch_bounds__(kAdamThreads) adam_kernel(AdamTable t, AdamScalars sc)
{
    int gi = 0;
    while (gi + 1 < t.ng && t.block_base[gi + 1] <= (int)blockIdx.x) ++gi;
    const long long n = t.n[gi];
    const long long e0 = (long long)(blockIdx.x - t.block_base[gi]) * kAdamChunk;
    const long long e1 = min(n, e0 + kAdamChunk);
    float *P = t.p[gi], *M = t.m[gi], *Vv = t.v[gi];
    const float *G = t.g[gi];
    const float ss = t.step_size[gi];
    long long done = e0;
    if (t.vec[gi]) {
        const long long q1 = e0 + (e1 - e0) / 4 * 4;
        for (long long e = e0 + 4 * (long long)threadIdx.x; e < q1; e += 4 * kAdamThreads) {
            float4 p = *reinterpret_cast<float4 *>(P + e), m = *reinterpret_cast<float4 *>(M + e);
            float4 v = *reinterpret_cast<float4 *>(Vv + e);
            const float4 g = __ldg(reinterpret_cast<const float4 *>(G + e));
            adam_one(p.x, g.x, m.x, v.x, sc, ss);
            adam_one(p.y, g.y, m.y, v.y, sc, ss);
            adam_one(p.z, g.z, m.z, v.z, sc, ss);
            adam_one(p.w, g.w, m.w, v.w, sc, ss);
            *reinterpret_cast<float4 *>(P + e) = p;
            *reinterpret_cast<float4 *>(M + e) = m;
            *reinterpret_cast<float4 *>(Vv + e) = v;
        }
        done = q1;
    }
    for (long long e = done + threadIdx.x; e < e1; e += kAdamThreads) {
        float p = P[e], m = M[e], v = Vv[e];
        adam_one(p, __ldg(G + e), m, v, sc, ss);
        P[e] = p;
        M[e] = m;
        Vv[e] = v;
    }
}

__global__ void __launch_bounds__(256) densify_stats_kernel(const int32_t *__restrict__ row_anchor,
                                                            const int32_t *__restrict__ view_start, int V,
                                                            long long cap_rows, int k,
                                                            const int32_t *__restrict__ tiles,
                                                            const float *__restrict__ opacity,
                                                            const float *__restrict__ sgrad, int N,
                                                            float *__restrict__ grad_accum,
                                                            int32_t *__restrict__ offset_denom,
                                                            float *__restrict__ opacity_accum,
                                                            int32_t *__restrict__ anchor_denom, gs_status *st)
{
    if (has_error(st)) return;
    const long long rows = min((long long)__ldg(view_start + V), cap_rows);
    for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < rows;
         r += (long long)gridDim.x * blockDim.x) {
        const int a = __ldg(row_anchor + r);
        if (!idx_ok(st, a, N, 70)) continue;
        float so = 0.f;
        for (int i = 0; i < k; ++i) {
            const long long c = r * k + i;
            so += fmaxf(__ldg(opacity + c), 0.f);
            if (__ldg(tiles + c) > 0) {
                const float gx = __ldg(sgrad + 9 * c), gy = __ldg(sgrad + 9 * c + 1);
                atomicAdd(grad_accum + (long long)a * k + i, sqrtf(fmaf(gx, gx, gy * gy)));
                atomicAdd(offset_denom + (long long)a * k + i, 1);
            }
        }
        atomicAdd(opacity_accum + a, so);
        atomicAdd(anchor_denom + a, 1);
    }
}

__global__ void __launch_bounds__(256) densify_masks_kernel(long long N, int k, const float *__restrict__ grad_accum,
                                                            const int32_t *__restrict__ offset_denom,
                                                            const float *__restrict__ opacity_accum,
                                                            const int32_t *__restrict__ anchor_denom,
                                                            float grad_thr, float opacity_thr, int min_count,
                                                            uint8_t *__restrict__ grow, uint8_t *__restrict__ prune)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < N * k; j += stride) {
        const int d = offset_denom[j];
        grow[j] = (uint8_t)(d >= min_count && d > 0 && __fdiv_rn(grad_accum[j], (float)d) >= grad_thr);
    }
    for (long long a = (long long)blockIdx.x * blockDim.x + threadIdx.x; a < N; a += stride) {
        const int d = anchor_denom[a];
        prune[a] = (uint8_t)(d >= min_count && d > 0 && __fdiv_rn(opacity_accum[a], (float)d) < opacity_thr);
    }
}

int launch_adam(const gs_adam_group *groups, int ng, long long step, double b1, double b2, double eps, cudaStream_t s)
{
    AdamTable t;
    t.ng = ng;
    const double bc1 = 1.0 - std::pow(b1, (double)step), bc2 = 1.0 - std::pow(b2, (double)step);
    AdamScalars sc;
    sc.b1 = (float)b1;
    sc.omb1 = (float)(1.0 - b1);
    sc.b2 = (float)b2;
    sc.omb2 = (float)(1.0 - b2);
    sc.eps = (float)eps;
    sc.inv_sqrt_bc2 = (float)(1.0 / std::sqrt(bc2));
    long long blocks = 0;
    for (int i = 0; i < ng; ++i) {
        const gs_adam_group &g = groups[i];
        t.p[i] = g.param; t.g[i] = g.grad; t.m[i] = g.m; t.v[i] = g.v; t.n[i] = g.n;
        t.step_size[i] = (float)((double)g.lr / bc1);
        t.vec[i] = ((reinterpret_cast<uintptr_t>(g.param) | reinterpret_cast<uintptr_t>(g.grad) |
                     reinterpret_cast<uintptr_t>(g.m) | reinterpret_cast<uintptr_t>(g.v)) & 15) == 0;
        t.block_base[i] = (int)blocks;
        blocks += (g.n + kAdamChunk - 1) / kAdamChunk;
        if (blocks > (1ll << 30)) return GS_ERR_INVALID_ARG;
    }
    t.block_base[ng] = (int)blocks;
    if (blocks > 0) {
        adam_kernel<<<(unsigned)blocks, kAdamThreads, 0, s>>>(t, sc);
        count_launches(1);
    }
    return cudaPeekAtLastError() == cudaSuccess ? GS_OK : GS_ERR_CUDA;
}

int launch_densify_stats(const gs_gauss3d *g, int V, const int32_t *tiles, const float *sgrad, int N,
                         float *grad_accum, int32_t *offset_denom, float *opacity_accum, int32_t *anchor_denom,
                         gs_status *st, cudaStream_t s)
{
    const int grid = (int)std::max<long long>(1, std::min<long long>((g->cap_rows + 255) / 256,
                                                                      (long long)sm_count() * 8));
    densify_stats_kernel<<<grid, 256, 0, s>>>(g->row_anchor, g->view_start, V, g->cap_rows, g->k, tiles,
                                              g->opacity, sgrad, N, grad_accum, offset_denom, opacity_accum,
                                              anchor_denom, st);
    count_launches(1);
    return cudaPeekAtLastError() == cudaSuccess ? GS_OK : GS_ERR_CUDA;
}

int launch_densify_masks(long long N, int k, const float *grad_accum, const int32_t *offset_denom,
                         const float *opacity_accum, const int32_t *anchor_denom, float grad_thr, float opacity_thr,
                         int min_count, uint8_t *grow, uint8_t *prune, cudaStream_t s)
{
    const int grid = (int)std::max<long long>(1, std::min<long long>((N * k + 255) / 256, (long long)sm_count() * 8));
    densify_masks_kernel<<<grid, 256, 0, s>>>(N, k, grad_accum, offset_denom, opacity_accum, anchor_denom, grad_thr,
                                              opacity_thr, min_count, grow, prune);
    count_launches(1);
    return cudaPeekAtLastError() == cudaSuccess ? GS_OK : GS_ERR_CUDA;
}

}  // namespace gs
