// decode_bwd.cu -- reverse of the partitioned anchor decoder (Eq. 6, Eq. 2),
// FP32 SIMT.
//
// Persistent CTAs of 128 threads walk tiles of 128 consecutive rows.  Per
// tile and per head, every thread recomputes its row's hidden layer (nothing
// of the forward pass is stored), forms the output gradient dz through the
// activation, back-propagates to dpre and du, and leaves u, hid, dz, dpre in
// shared memory ([element][row], row stride 129 so that both the per-row and
// the per-weight phases are bank-conflict free).  The CTA then accumulates the
// head's weight gradients over the tile's rows into a shared-memory
// accumulator of the current partition, flushed to global memory (atomicAdd)
// only when the partition changes and at the end.  Per-anchor gradients are
// summed over views with atomics.
#include "gs_internal.cuh"

namespace gs {

constexpr int kDbRows = 128;
constexpr int kDbStride = kDbRows + 1;


__device__ __forceinline__ void head_layout(int F, int k, int H, int h, int *off, int *din, int *dout)
{
    const int d = F + 4;
    const int douts[3] = {k, 3 * k, 7 * k};
    int o = 0;
    for (int i = 0; i < h; ++i) o += H * d + H + douts[i] * H + douts[i];
    *off = o; *din = d; *dout = douts[h];
}

__global__ void __launch_bounds__(kDbRows) decode_bwd_fp32_kernel(DecodeBwdArgsB a)
{
    if (__syncthreads_or(has_error(a.f.st))) return;   // block-uniform exit
    extern __shared__ float sm[];
    const int F = a.f.F, k = a.f.k, H = a.f.H, din = F + 4;
    const long long P = a.f.mlp_floats;
    float *s_u = sm;                         // [din][stride]
    float *s_hid = s_u + din * kDbStride;    // [H][stride]
    float *s_dz = s_hid + H * kDbStride;     // [7k][stride]
    float *s_dpre = s_dz + 7 * k * kDbStride; // [H][stride]
    float *s_du = s_dpre + H * kDbStride;    // [din][stride]
    float *s_acc = s_du + din * kDbStride;   // [P]
    __shared__ int s_part[kDbRows];
    __shared__ int s_accpart[3];
    const int tid = threadIdx.x;
    const int rows = __ldg(a.f.view_start + a.f.V);
    const int ntiles = (rows + kDbRows - 1) / kDbRows;
    if (tid < 3) s_accpart[tid] = -1;
    for (long long i = tid; i < P; i += kDbRows) s_acc[i] = 0.f;
    __syncthreads();
    // contiguous tile ranges per CTA: few partition changes, so few flushes of the accumulators
    const int per_cta = (ntiles + (int)gridDim.x - 1) / (int)gridDim.x;
    const int tile_end = min(ntiles, ((int)blockIdx.x + 1) * per_cta);
    for (int tile = (int)blockIdx.x * per_cta; tile < tile_end; ++tile) {
        const int r = tile * kDbRows + tid;
        const bool live = r < rows;
        int an = 0, v = 0, m = -1;
        float xc[3] = {0.f, 0.f, 0.f}, d[3] = {0.f, 0.f, 0.f}, delta = 1.f;
        if (live) {
            v = view_of_row(a.f.view_start, a.f.V, r);
            const Cam c = load_cam(a.f.cams, v);
#pragma unroll
            for (int i = 0; i < 3; ++i) xc[i] = -(c.R[i] * c.t[0] + c.R[3 + i] * c.t[1] + c.R[6 + i] * c.t[2]);
            an = __ldg(a.f.row_anchor + r);
            if (!idx_ok(a.f.st, an, a.f.N, 61)) an = 0;
            m = __ldg(a.f.part + an);
            if (!idx_ok(a.f.st, m, a.f.M, 62)) m = 0;
            for (int i = 0; i < F; ++i) s_u[i * kDbStride + tid] = __ldg(a.f.feat + (size_t)an * F + i);
            d[0] = __ldg(a.f.xyz + 3 * an) - xc[0];
            d[1] = __ldg(a.f.xyz + 3 * an + 1) - xc[1];
            d[2] = __ldg(a.f.xyz + 3 * an + 2) - xc[2];
            delta = sqrtf(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
            s_u[F * kDbStride + tid] = d[0] / delta;
            s_u[(F + 1) * kDbStride + tid] = d[1] / delta;
            s_u[(F + 2) * kDbStride + tid] = d[2] / delta;
            s_u[(F + 3) * kDbStride + tid] = delta;
        }
        s_part[tid] = m;
        for (int i = 0; i < din; ++i) s_du[i * kDbStride + tid] = 0.f;
        const float *mlp_m = live ? a.f.mlp + (size_t)m * P : a.f.mlp;
        unsigned gate = 0;   // bit i: candidate i survived decoding (opacity > 0)
        const size_t c0 = (size_t)r * k;
        float dls[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        for (int h = 0; h < 3; ++h) {
            int hoff, hdin, dout;
            head_layout(F, k, H, h, &hoff, &hdin, &dout);
            const float *W1 = mlp_m + hoff, *b1 = W1 + H * din, *W2 = b1 + H, *b2 = W2 + dout * H;
            if (live) {
                for (int j = 0; j < H; ++j) {
                    float s = __ldg(b1 + j);
                    for (int i = 0; i < din; ++i) s = fmaf(__ldg(W1 + j * din + i), s_u[i * kDbStride + tid], s);
                    s_hid[j * kDbStride + tid] = fmaxf(s, 0.f);
                }
                if (h == 0) {
                    for (int i = 0; i < k; ++i) {
                        float z = __ldg(b2 + i);
                        for (int j = 0; j < H; ++j) z = fmaf(__ldg(W2 + i * H + j), s_hid[j * kDbStride + tid], z);
                        const float op = tanhf(z);
                        float g = 0.f;
                        if (op > 0.f) {
                            gate |= 1u << i;
                            g = __ldg(a.dopacity + c0 + i) * (1.f - op * op);
                        }
                        s_dz[i * kDbStride + tid] = g;
                    }
                } else if (h == 1) {
                    for (int o = 0; o < 3 * k; ++o) {
                        float z = __ldg(b2 + o);
                        for (int j = 0; j < H; ++j) z = fmaf(__ldg(W2 + o * H + j), s_hid[j * kDbStride + tid], z);
                        float g = 0.f;
                        if (gate >> (o / 3) & 1u) {
                            const float sg = sigmoidf_(z);
                            g = __ldg(a.dcolour + c0 * 3 + o) * sg * (1.f - sg);
                        }
                        s_dz[o * kDbStride + tid] = g;
                    }
                } else {
                    const float *ls = a.f.log_scaling + 6 * an;
                    for (int i = 0; i < k; ++i) {
                        float z[7];
#pragma unroll
                        for (int q = 0; q < 7; ++q) {
                            float s = __ldg(b2 + 7 * i + q);
                            for (int j = 0; j < H; ++j) s = fmaf(__ldg(W2 + (7 * i + q) * H + j), s_hid[j * kDbStride + tid], s);
                            z[q] = s;
                        }
                        const bool g = gate >> i & 1u;
                        const size_t c = c0 + i;
#pragma unroll
                        for (int q = 0; q < 3; ++q) {
                            const float sg = sigmoidf_(z[q]);
                            const float e = expf(__ldg(ls + 3 + q));
                            const float dsq = g ? __ldg(a.dscale + 3 * c + q) : 0.f;
                            s_dz[(7 * i + q) * kDbStride + tid] = dsq * e * sg * (1.f - sg);
                            dls[3 + q] += dsq * e * sg;
                        }
                        const float qn = sqrtf(z[3] * z[3] + z[4] * z[4] + z[5] * z[5] + z[6] * z[6]);
                        const float inv = 1.f / qn;
                        float dq[4], qd = 0.f;
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            dq[q] = g ? __ldg(a.dquat + 4 * c + q) : 0.f;
                            qd += z[3 + q] * inv * dq[q];
                        }
#pragma unroll
                        for (int q = 0; q < 4; ++q)
                            s_dz[(7 * i + 3 + q) * kDbStride + tid] = (dq[q] - z[3 + q] * inv * qd) * inv;
                    }
                }
                // dpre = (W2^T dz) masked by pre > 0 ; du += W1^T dpre
                for (int j = 0; j < H; ++j) {
                    float s = 0.f;
                    if (s_hid[j * kDbStride + tid] > 0.f)
                        for (int o = 0; o < dout; ++o) s = fmaf(__ldg(W2 + o * H + j), s_dz[o * kDbStride + tid], s);
                    s_dpre[j * kDbStride + tid] = s;
                }
                for (int i = 0; i < din; ++i) {
                    float s = s_du[i * kDbStride + tid];
                    for (int j = 0; j < H; ++j) s = fmaf(__ldg(W1 + j * din + i), s_dpre[j * kDbStride + tid], s);
                    s_du[i * kDbStride + tid] = s;
                }
            } else {
                for (int j = 0; j < H; ++j) { s_hid[j * kDbStride + tid] = 0.f; s_dpre[j * kDbStride + tid] = 0.f; }
                for (int o = 0; o < dout; ++o) s_dz[o * kDbStride + tid] = 0.f;
            }
            __syncthreads();
            // weight gradients of head h over the tile, segment by partition
            const int nent = H * din + H + dout * H + dout;
            int s0 = 0;
            while (s0 < kDbRows) {
                const int pm = s_part[s0];
                int s1 = s0 + 1;
                while (s1 < kDbRows && s_part[s1] == pm) ++s1;
                if (pm >= 0) {
                    if (s_accpart[h] != pm) {
                        const int old = s_accpart[h];
                        __syncthreads();
                        if (old >= 0)
                            for (int e = tid; e < nent; e += kDbRows) {
                                atomicAdd(a.dmlp + (size_t)old * P + hoff + e, s_acc[hoff + e]);
                                s_acc[hoff + e] = 0.f;
                            }
                        __syncthreads();
                        if (tid == 0) s_accpart[h] = pm;
                        __syncthreads();
                    }
                    for (int e = tid; e < nent; e += kDbRows) {
                        float acc = 0.f;
                        if (e < H * din) {
                            const int j = e / din, i = e % din;
                            for (int rr = s0; rr < s1; ++rr) acc = fmaf(s_dpre[j * kDbStride + rr], s_u[i * kDbStride + rr], acc);
                        } else if (e < H * din + H) {
                            const int j = e - H * din;
                            for (int rr = s0; rr < s1; ++rr) acc += s_dpre[j * kDbStride + rr];
                        } else if (e < H * din + H + dout * H) {
                            const int q = e - H * din - H, o = q / H, j = q % H;
                            for (int rr = s0; rr < s1; ++rr) acc = fmaf(s_dz[o * kDbStride + rr], s_hid[j * kDbStride + rr], acc);
                        } else {
                            const int o = e - H * din - H - dout * H;
                            for (int rr = s0; rr < s1; ++rr) acc += s_dz[o * kDbStride + rr];
                        }
                        s_acc[hoff + e] += acc;
                    }
                }
                s0 = s1;
            }
            __syncthreads();
        }
        if (live) {
            // features
            for (int i = 0; i < F; ++i) atomicAdd(a.dfeat + (size_t)an * F + i, s_du[i * kDbStride + tid]);
            // direction and distance inputs -> anchor position
            const float inv = 1.f / delta;
            const float dir[3] = {d[0] * inv, d[1] * inv, d[2] * inv};
            const float g0 = s_du[F * kDbStride + tid], g1 = s_du[(F + 1) * kDbStride + tid],
                        g2 = s_du[(F + 2) * kDbStride + tid], gd = s_du[(F + 3) * kDbStride + tid];
            const float dd = g0 * dir[0] + g1 * dir[1] + g2 * dir[2];
            float dx[3];
            dx[0] = (g0 - dir[0] * dd) * inv + gd * dir[0];
            dx[1] = (g1 - dir[1] * dd) * inv + gd * dir[1];
            dx[2] = (g2 - dir[2] * dd) * inv + gd * dir[2];
            // positions mu = x_a + off * exp(l[0:3])
            const float *ls = a.f.log_scaling + 6 * an;
            const float e[3] = {expf(__ldg(ls)), expf(__ldg(ls + 1)), expf(__ldg(ls + 2))};
            for (int i = 0; i < k; ++i) {
                if (!(gate >> i & 1u)) continue;
                const size_t c = c0 + i;
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    const float g = __ldg(a.dmu + 3 * c + q);
                    dx[q] += g;
                    const float off = __ldg(a.f.offsets + ((size_t)an * k + i) * 3 + q);
                    atomicAdd(a.doff + ((size_t)an * k + i) * 3 + q, g * e[q]);
                    dls[q] += g * off * e[q];
                }
            }
#pragma unroll
            for (int q = 0; q < 3; ++q) atomicAdd(a.dxyz + 3 * an + q, dx[q]);
#pragma unroll
            for (int q = 0; q < 6; ++q) atomicAdd(a.dls + 6 * an + q, dls[q]);
        }
        __syncthreads();
    }
    // final flush
    for (int h = 0; h < 3; ++h) {
        int hoff, hdin, dout;
        head_layout(F, k, H, h, &hoff, &hdin, &dout);
        const int nent = H * din + H + dout * H + dout;
        const int pm = s_accpart[h];
        if (pm >= 0)
            for (int e = tid; e < nent; e += kDbRows) atomicAdd(a.dmlp + (size_t)pm * P + hoff + e, s_acc[hoff + e]);
    }
}

size_t decode_bwd_workspace_bytes(int N, int V, int M, long long cap_rows)
{
    (void)N; (void)V; (void)M; (void)cap_rows;
    return 0;
}

static size_t fp32_smem(int F, int k, int H, long long P)
{
    const int din = F + 4;
    return sizeof(float) * ((size_t)(din + H + 7 * k + H + din) * kDbStride + (size_t)P);
}

// Reverse of the decoders from the 3D-Gaussian gradients dg, or (dg NULL, BF16)
// from the splat gradients with the projection's chain rule fused in.
static int launch_decode_bwd_impl(const gs_anchors *A, const gs_camera *cams, const ViewTable &vt, int precision,
                                  const gs_gauss3d *g, const gs_gauss3d_grad *dg, const gs_splats *sp,
                                  const float *sgrad, gs_anchor_grad *out, gs_status *st, cudaStream_t s)
{
    const long long P = gs_mlp_floats(A->F, A->k, A->hidden);
    cudaMemsetAsync(out->dxyz, 0, sizeof(float) * 3 * (size_t)A->N, s);
    cudaMemsetAsync(out->dfeat, 0, sizeof(float) * (size_t)A->F * A->N, s);
    cudaMemsetAsync(out->dlog_scaling, 0, sizeof(float) * 6 * (size_t)A->N, s);
    cudaMemsetAsync(out->doffsets, 0, sizeof(float) * 3 * (size_t)A->k * A->N, s);
    cudaMemsetAsync(out->dmlp, 0, sizeof(float) * (size_t)P * A->M, s);
    DecodeBwdArgsB a;
    DecodeArgs &f = a.f;
    f.xyz = A->xyz; f.feat = A->feat; f.log_scaling = A->log_scaling; f.offsets = A->offsets;
    f.part = A->part; f.mlp = A->mlp; f.mlp_floats = P; f.N = A->N; f.F = A->F; f.k = A->k; f.H = A->hidden;
    f.M = A->M; f.V = vt.V; f.cams = cams; f.view_start = g->view_start; f.row_anchor = g->row_anchor;
    f.mu = g->mu; f.scale = g->scale; f.quat = g->quat; f.opacity = g->opacity; f.colour = g->colour;
    f.st = st; f.cap_rows = g->cap_rows; f.wait_ns = wait_limit_ns();
    a.dmu = a.dscale = a.dquat = a.dopacity = a.dcolour = nullptr;
    if (dg) {
        a.dmu = dg->dmu; a.dscale = dg->dscale; a.dquat = dg->dquat; a.dopacity = dg->dopacity; a.dcolour = dg->dcolour;
    }
    a.dxyz = out->dxyz; a.dfeat = out->dfeat; a.dls = out->dlog_scaling; a.doff = out->doffsets; a.dmlp = out->dmlp;
    a.sgT = dg ? nullptr : sgrad;
    for (int v = 0; v < GS_MAX_VIEWS; ++v) {
        a.W[v] = v < vt.V ? vt.W[v] : 0;
        a.H[v] = v < vt.V ? vt.H[v] : 0;
    }
    if (precision == GS_PREC_BF16) return launch_decode_bwd_bf16(a, s);
    if (!dg) return GS_ERR_UNSUPPORTED;   // the FP32 decoder takes the 3D gradients (see below)
    const size_t smem = fp32_smem(A->F, A->k, A->hidden, P);
    static int configured_smem = 0;
    if ((int)smem > configured_smem) {
        if (cudaFuncSetAttribute(decode_bwd_fp32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
            cudaSuccess)
            return GS_ERR_UNSUPPORTED;
        configured_smem = (int)smem;
    }
    const int tiles = (int)std::max<long long>(1, (g->cap_rows + kDbRows - 1) / kDbRows);
    const int grid = std::min(tiles, sm_count());
    decode_bwd_fp32_kernel<<<grid, kDbRows, smem, s>>>(a);
    count_launches(1);
    return cudaPeekAtLastError() == cudaSuccess ? GS_OK : GS_ERR_CUDA;
}

int launch_decode_bwd(const gs_anchors *A, const gs_camera *cams, const ViewTable &vt, int precision,
                      const gs_gauss3d *g, const gs_gauss3d_grad *dg, gs_anchor_grad *out, void *ws,
                      gs_status *st, cudaStream_t s)
{
    (void)ws;
    return launch_decode_bwd_impl(A, cams, vt, precision, g, dg, nullptr, nullptr, out, st, s);
}

// Workspace of the fused reverse: none for the tensor-core path; the FP32 path
// keeps the candidates' 3D gradients (14 floats each) between its two steps.
// Rows per tile of the tensor-core reverse decoder (its kBRows).
constexpr int kRowTile = 128;

// The splat gradients [C][9] of the candidates rearranged in row tiles,
// out[((t k + i) 9 + v) 128 + r] = sgrad[9 ((128 t + r) k + i) + v] for the
// candidates that cover a tile and zero for the others: in that layout the
// reverse decoder, one thread per row, reads each value with one coalesced
// load per warp.  One thread per row here too: it reads its row's 9 k
// contiguous values (8-byte loads where aligned) and writes each to its
// plane, where the warp's 32 consecutive rows make one coalesced store.
__global__ void __launch_bounds__(256) sgrad_row_tiles(const float *__restrict__ sgrad,
                                                       const int32_t *__restrict__ tiles,
                                                       const int32_t *__restrict__ view_start, int V, int k,
                                                       long long cap_rows, float *__restrict__ out,
                                                       const gs_status *st)
{
    if (has_error(st)) return;
    const long long rows = std::min<long long>(__ldg(view_start + V), cap_rows);
    const bool pairs = ((9 * k) & 1) == 0 && (reinterpret_cast<uintptr_t>(sgrad) & 7) == 0;
    for (long long row = (long long)blockIdx.x * blockDim.x + threadIdx.x; row < rows;
         row += (long long)gridDim.x * blockDim.x) {
        const long long t = row / kRowTile;
        const int r = (int)(row - t * kRowTile);
        const float *src = sgrad + 9 * (size_t)k * row;
        float *dst = out + (size_t)t * k * 9 * kRowTile + r;
        for (int i = 0; i < k; ++i) {
            const bool drawn = __ldg(tiles + (size_t)k * row + i) > 0;
            float v[10];
            if (pairs) {   // 9 values from 8-byte pieces: candidate i starts at an even or odd float
                const int f0 = 9 * i, e0 = f0 & ~1;
                const float2 *p2 = reinterpret_cast<const float2 *>(src + e0);
#pragma unroll
                for (int j = 0; j < 5; ++j) {
                    const float2 q = __ldg(p2 + j);
                    v[2 * j] = q.x;
                    v[2 * j + 1] = q.y;
                }
                if (f0 & 1) {
#pragma unroll
                    for (int j = 0; j < 9; ++j) v[j] = v[j + 1];
                }
            } else {
#pragma unroll
                for (int j = 0; j < 9; ++j) v[j] = __ldg(src + 9 * i + j);
            }
#pragma unroll
            for (int j = 0; j < 9; ++j) dst[((size_t)i * 9 + j) * kRowTile] = drawn ? v[j] : 0.f;
        }
    }
}

size_t decode_project_bwd_workspace_bytes(int k, long long cap_rows, int precision)
{
    if (precision == GS_PREC_BF16) {
        const size_t tiles = (size_t)std::max<long long>((cap_rows + kRowTile - 1) / kRowTile, 1);
        return align_up(sizeof(float) * 9 * (size_t)k * kRowTile * tiles, 256);
    }
    const size_t C = (size_t)std::max<long long>(cap_rows * k, 1);
    return align_up(sizeof(float) * 3 * C, 256) * 3 + align_up(sizeof(float) * 4 * C, 256) +
           align_up(sizeof(float) * C, 256);
}

int launch_decode_project_bwd(const gs_anchors *A, const gs_camera *cams, const ViewTable &vt, int precision,
                              const gs_gauss3d *g, const gs_splats *sp, const gs_splat_grad *sgrad,
                              gs_anchor_grad *out, void *ws, gs_status *st, cudaStream_t s)
{
    if (precision == GS_PREC_BF16) {
        if (sgrad->layout == GS_SGRAD_ROW_TILES)   // already in row tiles: read in place
            return launch_decode_bwd_impl(A, cams, vt, precision, g, nullptr, sp, sgrad->g, out, st, s);
        // the splat gradients in row tiles (workspace), then the fused reverse
        float *sgT = reinterpret_cast<float *>(ws);
        const int grid = (int)std::max<long long>(
            1, std::min<long long>((g->cap_rows + 255) / 256, (long long)sm_count() * 8));
        sgrad_row_tiles<<<grid, 256, 0, s>>>(sgrad->g, sp->tiles, g->view_start, vt.V, g->k, g->cap_rows, sgT, st);
        count_launches(1);
        return launch_decode_bwd_impl(A, cams, vt, precision, g, nullptr, sp, sgT, out, st, s);
    }
    // FP32: the projection's chain rule into the workspace, then the decoders' reverse
    const size_t C = (size_t)std::max<long long>(g->cap_rows * g->k, 1);
    char *w = reinterpret_cast<char *>(ws);
    gs_gauss3d_grad dg;
    size_t o = 0;
    dg.dmu = reinterpret_cast<float *>(w + o); o += align_up(sizeof(float) * 3 * C, 256);
    dg.dscale = reinterpret_cast<float *>(w + o); o += align_up(sizeof(float) * 3 * C, 256);
    dg.dcolour = reinterpret_cast<float *>(w + o); o += align_up(sizeof(float) * 3 * C, 256);
    dg.dquat = reinterpret_cast<float *>(w + o); o += align_up(sizeof(float) * 4 * C, 256);
    dg.dopacity = reinterpret_cast<float *>(w + o);
    const int rc = launch_project_bwd(g, cams, sp, vt, sgrad, &dg, st, s);
    if (rc != GS_OK) return rc;
    return launch_decode_bwd_impl(A, cams, vt, precision, g, &dg, nullptr, nullptr, out, st, s);
}

}  // namespace gs
