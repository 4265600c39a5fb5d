// decode.cu -- anchor visibility (row building) and FP32 anchor decoding.
//
// Visibility: one row per (view, anchor) whose centre is in front of the near
// plane and projects inside the image grown by 15 % per side, view-major and
// in anchor order (a deterministic three-kernel count / scan / write
// compaction, so row ids do not depend on scheduling).
//
// Decoding (Sec. III-A with Eq. 2; partition selection of Eq. 6): one thread
// per row runs the row's partition MLP set (three two-layer heads) on
// u = [f_a, d_ac, delta_ac] and writes the k candidate Gaussians.
#include "gs_common.cuh"
#include "gs_internal.cuh"

namespace gs {

constexpr int kVisThreads = 256;
constexpr int kVisItems = 8;
constexpr int kVisChunk = kVisThreads * kVisItems;

// Explicit fmaf / __fmul_rn / __fdiv_rn so the counting and the writing
// kernels take bit-identical decisions.
__device__ __forceinline__ float dot3_rn(const float *r, float x, float y, float z, float t)
{
    return fmaf(r[2], z, fmaf(r[1], y, fmaf(r[0], x, t)));
}
__device__ __forceinline__ bool anchor_visible(const Cam &c, int W, int H, float x, float y, float z)
{
    const float pz = dot3_rn(c.R + 6, x, y, z, c.t[2]);
    if (!(pz > kNear)) return false;
    const float px = dot3_rn(c.R, x, y, z, c.t[0]);
    const float py = dot3_rn(c.R + 3, x, y, z, c.t[1]);
    const float u = fmaf(c.fx, __fdiv_rn(px, pz), c.cx);
    const float v = fmaf(c.fy, __fdiv_rn(py, pz), c.cy);
    return u >= -kMargin * W && u < (1.0f + kMargin) * W && v >= -kMargin * H &&
           v < (1.0f + kMargin) * H;
}

// Block-wide exclusive scan of one int per thread (blockDim = kVisThreads).
__device__ __forceinline__ int block_excl_scan(int x, int *s_warp, int *total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int v = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += y;
    }
    if (lane == 31) s_warp[warp] = v;
    __syncthreads();
    if (warp == 0) {
        int w = lane < (kVisThreads / 32) ? s_warp[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < (kVisThreads / 32)) s_warp[lane] = w;
    }
    __syncthreads();
    int excl = v - x + (warp > 0 ? s_warp[warp - 1] : 0);
    *total = s_warp[kVisThreads / 32 - 1];
    __syncthreads();
    return excl;
}

__global__ void __launch_bounds__(kVisThreads) vis_count_kernel(
    const float *__restrict__ xyz, int N, const gs_camera *__restrict__ cams, ViewTable vt,
    int *__restrict__ counts, int nchunks, const gs_status *st)
{
    if (__syncthreads_or(has_error(st))) return;   // block-uniform exit
    const int v = blockIdx.y, b = blockIdx.x;
    const Cam c = load_cam(cams, v);
    int n = 0;
#pragma unroll
    for (int j = 0; j < kVisItems; ++j) {
        int a = b * kVisChunk + j * kVisThreads + threadIdx.x;
        if (a < N)
            n += anchor_visible(c, vt.W[v], vt.H[v], __ldg(xyz + 3 * a), __ldg(xyz + 3 * a + 1),
                                __ldg(xyz + 3 * a + 2));
    }
    __shared__ int s_warp[32];
    int total;
    block_excl_scan(n, s_warp, &total);
    if (threadIdx.x == 0) counts[v * nchunks + b] = total;
}

// Single-block exclusive scan over V*nchunks counts; writes view_start.
__global__ void __launch_bounds__(1024) vis_scan_kernel(int *__restrict__ counts, int n, int nchunks,
                                                        int V, int32_t *__restrict__ view_start,
                                                        long long cap_rows, gs_status *st)
{
    if (__syncthreads_or(has_error(st))) return;   // block-uniform exit
    __shared__ int s_warp[32];
    __shared__ long long s_carry;
    if (threadIdx.x == 0) s_carry = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int base = 0; base < n; base += 1024) {
        int i = base + threadIdx.x;
        int x = i < n ? counts[i] : 0;
        int v = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, v, o);
            if (lane >= o) v += y;
        }
        if (lane == 31) s_warp[warp] = v;
        __syncthreads();
        if (warp == 0) {
            int w = s_warp[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                int y = __shfl_up_sync(0xffffffffu, w, o);
                if (lane >= o) w += y;
            }
            s_warp[lane] = w;
        }
        __syncthreads();
        long long excl = s_carry + v - x + (warp > 0 ? s_warp[warp - 1] : 0);
        if (i < n) {
            counts[i] = (int)excl;
            if (i % nchunks == 0) view_start[i / nchunks] = (int32_t)excl;
        }
        __syncthreads();
        if (threadIdx.x == 0) s_carry += s_warp[31];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        long long total = s_carry;
        view_start[V] = (int32_t)(total < cap_rows ? total : cap_rows);
        if (total > cap_rows) {
            set_error(st, GS_ERR_CAPACITY, 1);
            set_needed(st, total);
        }
    }
}

__global__ void __launch_bounds__(kVisThreads) vis_write_kernel(
    const float *__restrict__ xyz, int N, const gs_camera *__restrict__ cams, ViewTable vt,
    const int *__restrict__ offsets, int nchunks, int32_t *__restrict__ row_anchor,
    long long cap_rows, const gs_status *st)
{
    if (__syncthreads_or(has_error(st))) return;   // block-uniform exit
    const int v = blockIdx.y, b = blockIdx.x;
    const Cam c = load_cam(cams, v);
    __shared__ int s_warp[32];
    long long base = offsets[v * nchunks + b];
    for (int j = 0; j < kVisItems; ++j) {
        int a = b * kVisChunk + j * kVisThreads + threadIdx.x;
        int vis = 0;
        if (a < N)
            vis = anchor_visible(c, vt.W[v], vt.H[v], __ldg(xyz + 3 * a), __ldg(xyz + 3 * a + 1),
                                 __ldg(xyz + 3 * a + 2));
        int total;
        int off = block_excl_scan(vis, s_warp, &total);
        if (vis && base + off < cap_rows) row_anchor[base + off] = a;
        base += total;
    }
}

// ---------------------------------------------------------------------------
// FP32 decode: one thread per row.  Per-thread vectors (u, hid) live in shared
// memory laid out [element][thread] (conflict-free).

struct HeadPtr {
    const float *W1, *b1, *W2, *b2;
};

__device__ __forceinline__ void head_ptrs(const float *m, int F, int k, int H, HeadPtr h[3])
{
    const int din = F + 4;
    const int douts[3] = {k, 3 * k, 7 * k};
    const float *p = m;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        h[i].W1 = p; p += H * din;
        h[i].b1 = p; p += H;
        h[i].W2 = p; p += douts[i] * H;
        h[i].b2 = p; p += douts[i];
    }
}

// Builds u = [f, dir, delta] in s_u (stride nt); returns delta and dir.
__device__ __forceinline__ void build_input(const float *__restrict__ feat, const float *__restrict__ xyz,
                                            int a, int F, const float xc[3], float *s_u, int nt,
                                            float d[3], float *delta)
{
    for (int i = 0; i < F; ++i) s_u[i * nt] = __ldg(feat + (size_t)a * F + i);
    float dx = __ldg(xyz + 3 * a) - xc[0], dy = __ldg(xyz + 3 * a + 1) - xc[1],
          dz = __ldg(xyz + 3 * a + 2) - xc[2];
    float n = sqrtf(dx * dx + dy * dy + dz * dz);
    d[0] = dx; d[1] = dy; d[2] = dz;
    *delta = n;
    s_u[F * nt] = dx / n;
    s_u[(F + 1) * nt] = dy / n;
    s_u[(F + 2) * nt] = dz / n;
    s_u[(F + 3) * nt] = n;
}

__device__ __forceinline__ void cam_centre(const Cam &c, float xc[3])
{
#pragma unroll
    for (int i = 0; i < 3; ++i) xc[i] = -(c.R[i] * c.t[0] + c.R[3 + i] * c.t[1] + c.R[6 + i] * c.t[2]);
}

// Hidden layer of one head into s_h (stride nt); pre-activation into s_pre if given.
__device__ __forceinline__ void hidden_layer(const HeadPtr &h, int din, int H, const float *s_u,
                                             float *s_h, float *s_pre, int nt)
{
    for (int j = 0; j < H; ++j) {
        const float *w = h.W1 + j * din;
        float s = __ldg(h.b1 + j);
        for (int i = 0; i < din; ++i) s = fmaf(__ldg(w + i), s_u[i * nt], s);
        if (s_pre) s_pre[j * nt] = s;
        s_h[j * nt] = fmaxf(s, 0.0f);
    }
}

__device__ __forceinline__ float out_unit(const HeadPtr &h, int H, int o, const float *s_h, int nt)
{
    const float *w = h.W2 + o * H;
    float s = __ldg(h.b2 + o);
    for (int j = 0; j < H; ++j) s = fmaf(__ldg(w + j), s_h[j * nt], s);
    return s;
}

__global__ void __launch_bounds__(128) decode_fp32_kernel(DecodeArgs a)
{
    if (__syncthreads_or(has_error(a.st))) return;   // block-uniform exit
    extern __shared__ float smem[];
    const int nt = blockDim.x;
    const int din = a.F + 4;
    float *s_u = smem + threadIdx.x;
    float *s_h = s_u + din * nt;
    const int rows = __ldg(a.view_start + a.V);
    const long long msz = a.mlp_floats;
    for (int r = blockIdx.x * nt + threadIdx.x; r < rows; r += gridDim.x * nt) {
        const int v = view_of_row(a.view_start, a.V, r);
        const Cam c = load_cam(a.cams, v);
        float xc[3];
        cam_centre(c, xc);
        const int an = __ldg(a.row_anchor + r);
        if (!idx_ok(a.st, an, a.N, 11)) continue;
        const int pm = __ldg(a.part + an);
        if (!idx_ok(a.st, pm, a.M, 12)) continue;
        HeadPtr hp[3];
        head_ptrs(a.mlp + (size_t)pm * msz, a.F, a.k, a.H, hp);
        float d[3], delta;
        build_input(a.feat, a.xyz, an, a.F, xc, s_u, nt, d, &delta);
        const size_t c0 = (size_t)r * a.k;
        // opacity head
        hidden_layer(hp[0], din, a.H, s_u, s_h, nullptr, nt);
        for (int i = 0; i < a.k; ++i) a.opacity[c0 + i] = tanhf(out_unit(hp[0], a.H, i, s_h, nt));
        // colour head
        hidden_layer(hp[1], din, a.H, s_u, s_h, nullptr, nt);
        for (int o = 0; o < 3 * a.k; ++o) a.colour[c0 * 3 + o] = sigmoidf_(out_unit(hp[1], a.H, o, s_h, nt));
        // covariance head
        hidden_layer(hp[2], din, a.H, s_u, s_h, nullptr, nt);
        const float *ls = a.log_scaling + 6 * an;
        const float e0 = expf(__ldg(ls)), e1 = expf(__ldg(ls + 1)), e2 = expf(__ldg(ls + 2));
        const float s0 = expf(__ldg(ls + 3)), s1 = expf(__ldg(ls + 4)), s2 = expf(__ldg(ls + 5));
        const float x0 = __ldg(a.xyz + 3 * an), x1 = __ldg(a.xyz + 3 * an + 1), x2 = __ldg(a.xyz + 3 * an + 2);
        for (int i = 0; i < a.k; ++i) {
            float z[7];
#pragma unroll
            for (int j = 0; j < 7; ++j) z[j] = out_unit(hp[2], a.H, 7 * i + j, s_h, nt);
            const size_t c = c0 + i;
            a.scale[3 * c] = s0 * sigmoidf_(z[0]);
            a.scale[3 * c + 1] = s1 * sigmoidf_(z[1]);
            a.scale[3 * c + 2] = s2 * sigmoidf_(z[2]);
            float qn = sqrtf(z[3] * z[3] + z[4] * z[4] + z[5] * z[5] + z[6] * z[6]);
            float inv = 1.0f / qn;
            a.quat[4 * c] = z[3] * inv;
            a.quat[4 * c + 1] = z[4] * inv;
            a.quat[4 * c + 2] = z[5] * inv;
            a.quat[4 * c + 3] = z[6] * inv;
            const float *off = a.offsets + ((size_t)an * a.k + i) * 3;
            a.mu[3 * c] = x0 + __ldg(off) * e0;
            a.mu[3 * c + 1] = x1 + __ldg(off + 1) * e1;
            a.mu[3 * c + 2] = x2 + __ldg(off + 2) * e2;
        }
    }
}

// ---------------------------------------------------------------------------
size_t decode_workspace_bytes(int N, int V)
{
    const int nchunks = div_up(N, kVisChunk);
    return align_up((size_t)nchunks * V * sizeof(int), 256);
}

int launch_decode(const gs_anchors *A, const gs_camera *cams, const ViewTable &vt, int precision,
                  gs_gauss3d *out, void *ws, gs_status *st, cudaStream_t s, const gs_splats *proj)
{
    const int N = A->N, V = vt.V;
    const int nchunks = N > 0 ? div_up(N, kVisChunk) : 1;
    int *counts = reinterpret_cast<int *>(ws);
    if (N > 0) {
        vis_count_kernel<<<dim3(nchunks, V), kVisThreads, 0, s>>>(A->xyz, N, cams, vt, counts, nchunks, st);
        vis_scan_kernel<<<1, 1024, 0, s>>>(counts, nchunks * V, nchunks, V, out->view_start, out->cap_rows, st);
        vis_write_kernel<<<dim3(nchunks, V), kVisThreads, 0, s>>>(A->xyz, N, cams, vt, counts, nchunks,
                                                                 out->row_anchor, out->cap_rows, st);
        count_launches(3);
    } else {
        cudaMemsetAsync(out->view_start, 0, sizeof(int32_t) * (V + 1), s);
    }
    DecodeArgs a;
    a.xyz = A->xyz; a.feat = A->feat; a.log_scaling = A->log_scaling; a.offsets = A->offsets;
    a.part = A->part; a.mlp = A->mlp; a.mlp_floats = gs_mlp_floats(A->F, A->k, A->hidden);
    a.N = N; a.F = A->F; a.k = A->k; a.H = A->hidden; a.M = A->M; a.V = V;
    a.cams = cams; a.view_start = out->view_start; a.row_anchor = out->row_anchor;
    a.mu = out->mu; a.scale = out->scale; a.quat = out->quat; a.opacity = out->opacity;
    a.colour = out->colour; a.st = st; a.cap_rows = out->cap_rows; a.wait_ns = wait_limit_ns();
    if (precision == GS_PREC_BF16 && proj) {   // decoded and projected in one kernel
        ProjOut po;
        po.rec = reinterpret_cast<float4 *>(proj->rec);
        po.tiles = proj->tiles;
        po.cap = std::min<long long>(proj->cap, out->cap_rows * (long long)out->k);
        for (int v = 0; v < GS_MAX_VIEWS; ++v) {
            po.W[v] = v < V ? vt.W[v] : 0;
            po.H[v] = v < V ? vt.H[v] : 0;
            po.TX[v] = v < V ? vt.TX[v] : 0;
            po.TY[v] = v < V ? vt.TY[v] : 0;
        }
        return launch_decode_bf16(a, s, &po);
    }
    if (precision == GS_PREC_BF16) {
        const int rc = launch_decode_bf16(a, s);
        if (rc != GS_OK || !proj) return rc;
    }
    const int nt = 128;
    const size_t smem = (size_t)(A->F + 4 + A->hidden) * nt * sizeof(float);
    const long long grid_max = (out->cap_rows + nt - 1) / nt;
    int grid = (int)std::min<long long>(grid_max > 0 ? grid_max : 1, (long long)sm_count() * 8);
    if (smem > 48 * 1024 &&
        cudaFuncSetAttribute(decode_fp32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return GS_ERR_UNSUPPORTED;
    decode_fp32_kernel<<<grid, nt, smem, s>>>(a);
    count_launches(1);
    if (cudaPeekAtLastError() != cudaSuccess) return GS_ERR_CUDA;
    if (proj) return launch_project(out, cams, vt, const_cast<gs_splats *>(proj), st, s);
    return GS_OK;
}

}  // namespace gs
