// flow.cu -- geometry of the flow densification (Sec. III, Flow
// Densification; Eq. 5): correspondence filtering by the epipolar residual of
// the known poses and linear triangulation of the kept pairs.
//
// F = [e2]x P2 P1^+ with P_i = K_i [R_i | t_i], e2 = P2 C1 and C1 the centre of
// keyframe 1; P1^+ = P1^T (P1 P1^T)^-1 (P1 has full row rank).  Every CTA
// forms F once in double precision; the residual |x'^T F x| of each sampled
// pair x <-> x' = x + flow(x) is evaluated in double, so the keep decision
// (residual < tau) does not depend on single-precision rounding.  Kept pairs
// are triangulated by linear least squares on the four DLT rows with the
// homogeneous coordinate fixed to 1 (3x3 normal equations, double), and
// written in sample order (two passes: per-CTA counts, scan, write).
#include "gs_internal.cuh"

namespace gs {

constexpr int kFlowThreads = 256;
constexpr int kFlowItems = 8;
constexpr int kFlowTile = kFlowThreads * kFlowItems;

struct FlowGeom {
    double F[9], P1[12], P2[12];
};

__device__ void proj_matrix(const gs_camera *c, double P[12])
{
    const float *p = reinterpret_cast<const float *>(c);
    const double fx = p[0], fy = p[1], cx = p[2], cy = p[3];
    double Rt[12];
    for (int r = 0; r < 3; ++r) {
        for (int j = 0; j < 3; ++j) Rt[4 * r + j] = p[4 + 3 * r + j];
        Rt[4 * r + 3] = p[13 + r];
    }
    for (int j = 0; j < 4; ++j) {
        P[j] = fx * Rt[j] + cx * Rt[8 + j];
        P[4 + j] = fy * Rt[4 + j] + cy * Rt[8 + j];
        P[8 + j] = Rt[8 + j];
    }
}

// 3x3 inverse by the adjugate (row-major); returns the determinant.
__device__ double inv3(const double a[9], double o[9])
{
    o[0] = a[4] * a[8] - a[5] * a[7];
    o[1] = a[2] * a[7] - a[1] * a[8];
    o[2] = a[1] * a[5] - a[2] * a[4];
    o[3] = a[5] * a[6] - a[3] * a[8];
    o[4] = a[0] * a[8] - a[2] * a[6];
    o[5] = a[2] * a[3] - a[0] * a[5];
    o[6] = a[3] * a[7] - a[4] * a[6];
    o[7] = a[1] * a[6] - a[0] * a[7];
    o[8] = a[0] * a[4] - a[1] * a[3];
    const double det = a[0] * o[0] + a[1] * o[3] + a[2] * o[6];
    const double id = 1.0 / det;
    for (int i = 0; i < 9; ++i) o[i] *= id;
    return det;
}

__device__ void flow_geometry(const gs_camera *c1, const gs_camera *c2, FlowGeom *g)
{
    proj_matrix(c1, g->P1);
    proj_matrix(c2, g->P2);
    const float *p1 = reinterpret_cast<const float *>(c1);
    double C1[4];   // -R1^T t1, 1
    for (int j = 0; j < 3; ++j)
        C1[j] = -((double)p1[4 + j] * p1[13] + (double)p1[7 + j] * p1[14] + (double)p1[10 + j] * p1[15]);
    C1[3] = 1.0;
    double e2[3];
    for (int r = 0; r < 3; ++r)
        e2[r] = g->P2[4 * r] * C1[0] + g->P2[4 * r + 1] * C1[1] + g->P2[4 * r + 2] * C1[2] + g->P2[4 * r + 3];
    double PPt[9], iPPt[9];
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) {
            double s = 0.0;
            for (int j = 0; j < 4; ++j) s += g->P1[4 * r + j] * g->P1[4 * c + j];
            PPt[3 * r + c] = s;
        }
    inv3(PPt, iPPt);
    double Pp[12];   // P1^+ (4x3) = P1^T (P1 P1^T)^-1
    for (int j = 0; j < 4; ++j)
        for (int c = 0; c < 3; ++c)
            Pp[3 * j + c] = g->P1[j] * iPPt[c] + g->P1[4 + j] * iPPt[3 + c] + g->P1[8 + j] * iPPt[6 + c];
    double M[9];     // P2 P1^+
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) {
            double s = 0.0;
            for (int j = 0; j < 4; ++j) s += g->P2[4 * r + j] * Pp[3 * j + c];
            M[3 * r + c] = s;
        }
    const double S[9] = {0.0, -e2[2], e2[1], e2[2], 0.0, -e2[0], -e2[1], e2[0], 0.0};
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) g->F[3 * r + c] = S[3 * r] * M[c] + S[3 * r + 1] * M[3 + c] + S[3 * r + 2] * M[6 + c];
}

// Residual and keep decision of sample s (pixel q = y W + x).
__device__ __forceinline__ bool flow_keep(const FlowGeom &g, const float *__restrict__ flow, int q, int W, double tau,
                                          double *x, double *y, double *xp, double *yp, double *res)
{
    *x = (double)(q % W);
    *y = (double)(q / W);
    *xp = *x + (double)__ldg(flow + 2 * (size_t)q);
    *yp = *y + (double)__ldg(flow + 2 * (size_t)q + 1);
    const double f0 = g.F[0] * *x + g.F[1] * *y + g.F[2];
    const double f1 = g.F[3] * *x + g.F[4] * *y + g.F[5];
    const double f2 = g.F[6] * *x + g.F[7] * *y + g.F[8];
    *res = fabs(*xp * f0 + *yp * f1 + f2);
    return *res < tau;
}

__global__ void __launch_bounds__(kFlowThreads) flow_count_kernel(const gs_camera *c1, const gs_camera *c2, int W,
                                                                  int HW, const float *__restrict__ flow,
                                                                  const int32_t *__restrict__ samples, int N,
                                                                  double tau, float *__restrict__ residual,
                                                                  uint32_t *__restrict__ block_counts, gs_status *st)
{
    __shared__ FlowGeom g;
    __shared__ uint32_t s_cnt;
    if (threadIdx.x == 0) { flow_geometry(c1, c2, &g); s_cnt = 0; }
    __syncthreads();
    uint32_t c = 0;
    const int i0 = blockIdx.x * kFlowTile;
    for (int i = i0 + threadIdx.x; i < min(N, i0 + kFlowTile); i += kFlowThreads) {
        const int q = samples[i];
        if (!idx_ok(st, q, HW, 90)) continue;
        double x, y, xp, yp, r;
        c += flow_keep(g, flow, q, W, tau, &x, &y, &xp, &yp, &r);
        if (residual) residual[i] = (float)r;
    }
    atomicAdd(&s_cnt, c);
    __syncthreads();
    if (threadIdx.x == 0) block_counts[blockIdx.x] = s_cnt;
}

// Exclusive scan of the per-CTA counts (one block, sequential chunks of 1024).
__global__ void __launch_bounds__(1024) flow_scan_kernel(uint32_t *__restrict__ counts, int nb,
                                                         uint32_t *__restrict__ n_kept, long long cap, gs_status *st)
{
    __shared__ uint32_t s_warp[32];
    __shared__ unsigned long long s_carry;
    if (threadIdx.x == 0) s_carry = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int base = 0; base < nb; base += 1024) {
        const int i = base + threadIdx.x;
        const uint32_t x = i < nb ? counts[i] : 0u;
        uint32_t v = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t yv = __shfl_up_sync(0xffffffffu, v, o);
            if (lane >= o) v += yv;
        }
        if (lane == 31) s_warp[warp] = v;
        __syncthreads();
        if (warp == 0) {
            uint32_t w = s_warp[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t yv = __shfl_up_sync(0xffffffffu, w, o);
                if (lane >= o) w += yv;
            }
            s_warp[lane] = w;
        }
        __syncthreads();
        const unsigned long long ex = s_carry + v - x + (warp > 0 ? s_warp[warp - 1] : 0u);
        if (i < nb) counts[i] = (uint32_t)ex;
        __syncthreads();
        if (threadIdx.x == 0) s_carry += s_warp[31];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        if ((long long)s_carry > cap) {
            set_error(st, GS_ERR_CAPACITY, 91);
            set_needed(st, (long long)s_carry);
            *n_kept = 0;
        } else {
            *n_kept = (uint32_t)s_carry;
        }
    }
}

__global__ void __launch_bounds__(kFlowThreads) flow_write_kernel(const gs_camera *c1, const gs_camera *c2, int W,
                                                                  int HW, const float *__restrict__ flow,
                                                                  const int32_t *__restrict__ samples, int N,
                                                                  double tau, const uint32_t *__restrict__ block_off,
                                                                  int32_t *__restrict__ kept,
                                                                  float *__restrict__ points, long long cap,
                                                                  gs_status *st)
{
    // block-uniform exit (the kernel has block barriers below)
    if (__syncthreads_or(has_error(st))) return;
    __shared__ FlowGeom g;
    __shared__ uint32_t s_warp[kFlowThreads / 32];
    if (threadIdx.x == 0) flow_geometry(c1, c2, &g);
    __syncthreads();
    // thread t owns samples i0 + 8 t .. i0 + 8 t + 7 (sample order is kept)
    const int i0 = blockIdx.x * kFlowTile + threadIdx.x * kFlowItems;
    bool kp[kFlowItems];
    uint32_t c = 0;
#pragma unroll
    for (int j = 0; j < kFlowItems; ++j) {
        kp[j] = false;
        const int i = i0 + j;
        if (i < N) {
            const int q = samples[i];
            if (q >= 0 && q < HW) {
                double x, y, xp, yp, r;
                kp[j] = flow_keep(g, flow, q, W, tau, &x, &y, &xp, &yp, &r);
            }
        }
        c += kp[j];
    }
    // block exclusive scan of c
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t v = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t yv = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += yv;
    }
    if (lane == 31) s_warp[warp] = v;
    __syncthreads();
    uint32_t wpre = 0;
    for (int w = 0; w < warp; ++w) wpre += s_warp[w];
    uint32_t off = block_off[blockIdx.x] + wpre + v - c;
#pragma unroll
    for (int j = 0; j < kFlowItems; ++j) {
        if (!kp[j]) continue;
        const int i = i0 + j;
        const int q = samples[i];
        double x, y, xp, yp, r;
        flow_keep(g, flow, q, W, tau, &x, &y, &xp, &yp, &r);
        // rows x P1[2] - P1[0], y P1[2] - P1[1], x' P2[2] - P2[0], y' P2[2] - P2[1]
        double A[4][4];
        for (int k = 0; k < 4; ++k) {
            A[0][k] = x * g.P1[8 + k] - g.P1[k];
            A[1][k] = y * g.P1[8 + k] - g.P1[4 + k];
            A[2][k] = xp * g.P2[8 + k] - g.P2[k];
            A[3][k] = yp * g.P2[8 + k] - g.P2[4 + k];
        }
        double Nm[9], b[3], iN[9];
        for (int r0 = 0; r0 < 3; ++r0) {
            double s = 0.0;
            for (int k = 0; k < 4; ++k) s -= A[k][r0] * A[k][3];
            b[r0] = s;
            for (int c0 = 0; c0 < 3; ++c0) {
                double t = 0.0;
                for (int k = 0; k < 4; ++k) t += A[k][r0] * A[k][c0];
                Nm[3 * r0 + c0] = t;
            }
        }
        inv3(Nm, iN);
        if (idx_ok(st, off, cap, 92)) {
            kept[off] = i;
            for (int r0 = 0; r0 < 3; ++r0)
                points[3 * (size_t)off + r0] = (float)(iN[3 * r0] * b[0] + iN[3 * r0 + 1] * b[1] + iN[3 * r0 + 2] * b[2]);
        }
        ++off;
    }
}

size_t flow_workspace_bytes(int N) { return align_up(sizeof(uint32_t) * (size_t)std::max(1, (N + kFlowTile - 1) / kFlowTile), 256); }

int launch_flow_triangulate(const gs_camera *c1, const gs_camera *c2, int W, int H, const float *flow,
                            const int32_t *samples, int N, double tau, float *residual, int32_t *kept, float *points,
                            long long cap, uint32_t *n_kept, void *ws, gs_status *st, cudaStream_t s)
{
    const int nb = std::max(1, (N + kFlowTile - 1) / kFlowTile);
    uint32_t *counts = reinterpret_cast<uint32_t *>(ws);
    flow_count_kernel<<<nb, kFlowThreads, 0, s>>>(c1, c2, W, W * H, flow, samples, N, tau, residual, counts, st);
    flow_scan_kernel<<<1, 1024, 0, s>>>(counts, nb, n_kept, cap, st);
    flow_write_kernel<<<nb, kFlowThreads, 0, s>>>(c1, c2, W, W * H, flow, samples, N, tau, counts, kept, points, cap,
                                                  st);
    count_launches(3);
    return cudaPeekAtLastError() == cudaSuccess ? GS_OK : GS_ERR_CUDA;
}

}  // namespace gs
