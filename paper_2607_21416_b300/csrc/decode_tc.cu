// decode_tc.cu -- BF16 anchor decoding on the 5th-generation tensor cores
// (tcgen05.mma, shared-memory operands, FP32 accumulators in tensor memory).
//
// Same arithmetic as the FP32 decoder (Sec. III-A, Eq. 2; the partition MLP
// sets of Eq. 6), with both MLP layers as M = 128 MMAs:
//   layer 1:  PRE[128 x 3H] = U[128 x KP] W1^T            (all three heads)
//   layer 2:  Z_oc [128 x Noc]  = HID[:, 0:2H] W2oc^T     (opacity + colour)
//             Z_cov[128 x Ncov] = HID[:, 2H:3H] W2cov^T   (scale + rotation)
// with HID = relu(PRE + b1) rounded to BF16.  The layer-2 weights are stored
// with their output rows permuted so that candidate i's values sit at aligned
// accumulator columns: [opacity, r, g, b] at 4i of Z_oc (W2oc is block
// diagonal over the opacity / colour hidden units) and [s0 s1 s2 q0 q1 q2 q3 -]
// at 8i of Z_cov.
//
// One CTA of 128 threads owns 128 rows at a time, one thread per row: the
// thread builds its row of U, reads its accumulator lane after each MMA and
// writes its row's k candidates.  The CTA is persistent over the row range;
// the partition's weights are converted to BF16 into shared memory only when
// the partition changes, and a tile with rows of several partitions runs the
// MMAs once per partition (rows of other partitions discard the result).
// Outputs go through a per-warp shared-memory stage so that every global
// store is a contiguous 16-byte piece of the SoA arrays.
#include <cuda_bf16.h>

#include "gs_internal.cuh"
#include "proj_fwd.cuh"
#include "tc05.cuh"

namespace gs {

constexpr int kTRows = 128;
constexpr int kTThreads = 128;

struct TcShape {
    int F, Din, KP, H, k, N1, Noc, Ncov, tcols;
    int dout[3], hoff[3];
    uint32_t o_U, o_R, o_W1, o_W2oc, o_W2cov, o_b1, o_b2;
    int stage_floats;   // per warp
    size_t smem;
};

static int up16(int x) { return (x + 15) / 16 * 16; }


static TcShape tc_shape(int F, int k, int H)
{
    TcShape s;
    s.F = F; s.Din = F + 4; s.KP = up16(s.Din); s.H = H; s.k = k;
    s.N1 = 3 * H;
    s.Noc = up16(4 * k);
    s.Ncov = up16(8 * k);
    int need = std::max(s.N1, s.Noc + s.Ncov), c = 32;
    while (c < need) c <<= 1;
    s.tcols = c;
    const int d[3] = {k, 3 * k, 7 * k};
    int h = 0;
    for (int i = 0; i < 3; ++i) {
        s.dout[i] = d[i];
        s.hoff[i] = h;
        h += H * s.Din + H + d[i] * H + d[i];
    }
    s.stage_floats = 32 * 4 * k;
    size_t b = 0;
    auto take = [&](size_t bytes) { uint32_t at = (uint32_t)b; b = align_up(b + bytes, 128); return at; };
    // the layer-1 operand U, the hidden operand R and the output stages share one region: U is dead
    // once the layer-1 MMA has completed, R once the layer-2 MMA has, and U is rebuilt for every
    // partition pass (more resident CTAs: the kernel waits on global loads)
    s.o_U = take(std::max<size_t>(std::max<size_t>(2ull * kTRows * s.KP, 2ull * kTRows * s.N1),
                                  4ull * 4 * s.stage_floats));
    s.o_R = s.o_U;
    s.o_W1 = take(2ull * s.N1 * s.KP);
    s.o_W2oc = take(2ull * s.Noc * 2 * H);
    s.o_W2cov = take(2ull * s.Ncov * H);
    s.o_b1 = take(4ull * s.N1);
    s.o_b2 = take(4ull * (s.Noc + s.Ncov));
    s.smem = b;
    return s;
}

// Converts partition p's FP32 weights into the BF16 core-matrix layouts.
__device__ void tc_stage_weights(const TcShape &s, char *sm, const float *__restrict__ w)
{
    const int tid = threadIdx.x, H = s.H, K2 = 2 * H;
    for (int idx = tid; idx < s.N1 * s.KP; idx += kTThreads) {
        const int j = idx / s.KP, i = idx % s.KP, h = j / H, jj = j % H;
        const int ho = h == 0 ? s.hoff[0] : (h == 1 ? s.hoff[1] : s.hoff[2]);   // no dynamic indexing of
        const float v = i < s.Din ? __ldg(w + ho + jj * s.Din + i) : 0.f;        // the parameter block
        *reinterpret_cast<__nv_bfloat16 *>(sm + s.o_W1 + tc::kmajor_offset(j, i, s.KP)) = __float2bfloat16_rn(v);
    }
    for (int idx = tid; idx < s.Noc * K2; idx += kTThreads) {
        const int o = idx / K2, kk = idx % K2, i = o >> 2, c = o & 3;
        float v = 0.f;
        if (i < s.k) {
            if (c == 0 && kk < H) v = __ldg(w + s.hoff[0] + H * s.Din + H + i * H + kk);
            else if (c > 0 && kk >= H) v = __ldg(w + s.hoff[1] + H * s.Din + H + (3 * i + c - 1) * H + (kk - H));
        }
        *reinterpret_cast<__nv_bfloat16 *>(sm + s.o_W2oc + tc::kmajor_offset(o, kk, K2)) = __float2bfloat16_rn(v);
    }
    for (int idx = tid; idx < s.Ncov * H; idx += kTThreads) {
        const int o = idx / H, kk = idx % H, i = o >> 3, j = o & 7;
        const float v = (i < s.k && j < 7) ? __ldg(w + s.hoff[2] + H * s.Din + H + (7 * i + j) * H + kk) : 0.f;
        *reinterpret_cast<__nv_bfloat16 *>(sm + s.o_W2cov + tc::kmajor_offset(o, kk, H)) = __float2bfloat16_rn(v);
    }
    float *b1 = reinterpret_cast<float *>(sm + s.o_b1);
    for (int j = tid; j < s.N1; j += kTThreads) {
        const int h = j / H, ho = h == 0 ? s.hoff[0] : (h == 1 ? s.hoff[1] : s.hoff[2]);
        b1[j] = __ldg(w + ho + H * s.Din + j % H);
    }
    float *b2 = reinterpret_cast<float *>(sm + s.o_b2);
    for (int o = tid; o < s.Noc + s.Ncov; o += kTThreads) {
        float v = 0.f;
        if (o < s.Noc) {
            const int i = o >> 2, c = o & 3;
            if (i < s.k)
                v = c == 0 ? __ldg(w + s.hoff[0] + H * s.Din + H + s.dout[0] * H + i)
                           : __ldg(w + s.hoff[1] + H * s.Din + H + s.dout[1] * H + 3 * i + c - 1);
        } else {
            const int oo = o - s.Noc, i = oo >> 3, j = oo & 7;
            if (i < s.k && j < 7) v = __ldg(w + s.hoff[2] + H * s.Din + H + s.dout[2] * H + 7 * i + j);
        }
        b2[o] = v;
    }
}

// Copies n floats of a warp's stage to global memory (16-byte pieces when
// both sides allow it).
__device__ __forceinline__ void stage_out(const float *stage, float *dst, int n, bool vec)
{
    const int lane = threadIdx.x & 31;
    if (vec) {
        const int n4 = n >> 2;
        for (int i = lane; i < n4; i += 32)
            reinterpret_cast<float4 *>(dst)[i] = reinterpret_cast<const float4 *>(stage)[i];
        for (int i = 4 * n4 + lane; i < n; i += 32) dst[i] = stage[i];
    } else {
        for (int i = lane; i < n; i += 32) dst[i] = stage[i];
    }
}

// vec: bit 0 = the five output arrays are 16-byte aligned, bit 1 = feature rows are.
// PROJ: instead of the decoded Gaussians, each candidate's splat record is
// written (the projection of gs_project applied in the epilogue).
template <bool PROJ>
__global__ void __launch_bounds__(kTThreads) decode_tc_kernel(DecodeArgs a, TcShape s, int vec, ProjOut po)
{
    if (__syncthreads_or(has_error(a.st))) return;   // block-uniform exit
    extern __shared__ __align__(1024) char sm[];
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t tslot;
    __shared__ int s_p, s_staged;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int k = s.k, H = s.H;
    if (warp == 0) {
        tc::tmem_alloc(&tslot, (uint32_t)s.tcols);
        tc::tmem_relinquish();
    }
    if (tid == 0) {
        tc::mbar_init(&bar, 1);
        s_staged = -1;
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = tslot;
    const uint32_t sU = tc::smem_u32(sm + s.o_U), sR = tc::smem_u32(sm + s.o_R);
    const uint32_t sW1 = tc::smem_u32(sm + s.o_W1), sW2oc = tc::smem_u32(sm + s.o_W2oc);
    const uint32_t sW2cov = tc::smem_u32(sm + s.o_W2cov);
    const float *b1 = reinterpret_cast<const float *>(sm + s.o_b1);
    const float *b2 = reinterpret_cast<const float *>(sm + s.o_b2);
    float *stage = reinterpret_cast<float *>(sm + s.o_R) + warp * s.stage_floats;
    const int rows = __ldg(a.view_start + a.V);
    const int ntiles = (rows + kTRows - 1) / kTRows;
    const long long P = a.mlp_floats;
    uint32_t phase = 0;
    bool failed = false;   // an MMA completion wait ran out; `phase` is then the parity it waited for

    // each CTA takes a contiguous range of tiles: rows are view-major and partition-sorted inside a
    // view, so a CTA meets few partitions (the weights are staged, and the weight gradients flushed,
    // only when the partition changes)
    const int per_cta = (ntiles + (int)gridDim.x - 1) / (int)gridDim.x;
    const int tile_end = min(ntiles, ((int)blockIdx.x + 1) * per_cta);
    for (int tile = (int)blockIdx.x * per_cta; tile < tile_end && !failed; ++tile) {
        // ---- this thread's row: anchor, partition, view inputs of Eq. 2, U row
        const int row = tile * kTRows + tid;
        int an = -1, pm = -1, vw = 0;
        float d0 = 0.f, d1 = 0.f, d2 = 0.f, dl = 1.f;
        Cam cam;
        if (row < rows) {
            an = __ldg(a.row_anchor + row);
            if (!idx_ok(a.st, an, a.N, 13)) an = -1;
        }
        if (an >= 0) {
            pm = __ldg(a.part + an);
            if (!idx_ok(a.st, pm, a.M, 14)) { pm = -1; an = -1; }
        }
        if (an >= 0) {
            vw = view_of_row(a.view_start, a.V, row);
            cam = load_cam(a.cams, vw);
            const Cam &c = cam;
            float xc[3];
#pragma unroll
            for (int i = 0; i < 3; ++i) xc[i] = -(c.R[i] * c.t[0] + c.R[3 + i] * c.t[1] + c.R[6 + i] * c.t[2]);
            d0 = __ldg(a.xyz + 3 * an) - xc[0];
            d1 = __ldg(a.xyz + 3 * an + 1) - xc[1];
            d2 = __ldg(a.xyz + 3 * an + 2) - xc[2];
            dl = sqrtf(d0 * d0 + d1 * d1 + d2 * d2);
        }
        // U row = [f_a, d / |d|, |d|, 0 ...] in BF16, 16-byte pieces of 8 columns (rebuilt for every
        // partition pass: its region is the hidden operand's)
        auto build_u = [&]() {
            const float inv = 1.f / dl;
            const float *f = a.feat + (size_t)(an >= 0 ? an : 0) * s.F;
            auto put8 = [&](int kc, const float u[8]) {
                uint4 pk;
                __nv_bfloat162 t0 = __floats2bfloat162_rn(u[0], u[1]), t1 = __floats2bfloat162_rn(u[2], u[3]);
                __nv_bfloat162 t2 = __floats2bfloat162_rn(u[4], u[5]), t3 = __floats2bfloat162_rn(u[6], u[7]);
                pk.x = *reinterpret_cast<uint32_t *>(&t0); pk.y = *reinterpret_cast<uint32_t *>(&t1);
                pk.z = *reinterpret_cast<uint32_t *>(&t2); pk.w = *reinterpret_cast<uint32_t *>(&t3);
                *reinterpret_cast<uint4 *>(sm + s.o_U + tc::kmajor_offset(tid, kc, s.KP)) = pk;
            };
            const int kfull = an >= 0 ? (s.F & ~7) : 0;   // columns filled by whole 8-feature pieces
            int kc = 0;
            if (vec & 2) {   // 16-byte aligned feature rows
                for (; kc < kfull; kc += 8) {
                    const float4 x0 = __ldg(reinterpret_cast<const float4 *>(f + kc));
                    const float4 x1 = __ldg(reinterpret_cast<const float4 *>(f + kc + 4));
                    const float u[8] = {x0.x, x0.y, x0.z, x0.w, x1.x, x1.y, x1.z, x1.w};
                    put8(kc, u);
                }
            } else {
                for (; kc < kfull; kc += 8) {
                    float u[8];
#pragma unroll
                    for (int j = 0; j < 8; ++j) u[j] = __ldg(f + kc + j);
                    put8(kc, u);
                }
            }
            for (; kc < s.KP; kc += 8) {
                float u[8];
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const int i = kc + j;
                    float x = 0.f;
                    if (an >= 0) {
                        if (i < s.F) x = __ldg(f + i);
                        else if (i == s.F) x = d0 * inv;
                        else if (i == s.F + 1) x = d1 * inv;
                        else if (i == s.F + 2) x = d2 * inv;
                        else if (i == s.F + 3) x = dl;
                    }
                    u[j] = x;
                }
                put8(kc, u);
            }
        };
        bool done = pm < 0;
        const int row0 = tile * kTRows + warp * 32;
        const int nval = max(0, min(32, rows - row0));

        for (;;) {
            // ---- next partition present among the rows not yet decoded
            if (tid == 0) s_p = 0x7fffffff;
            __syncthreads();
            if (!done) atomicMin(&s_p, pm);
            __syncthreads();
            const int p = s_p;
            if (p == 0x7fffffff) break;
            if (p != s_staged) {
                tc_stage_weights(s, sm, a.mlp + (size_t)p * P);
                if (tid == 0) s_staged = p;
            }
            build_u();   // every thread is past the previous pass's use of the region (two barriers above)
            // ---- layer 1
            tc::fence_async_smem();
            tc::fence_before_sync();
            __syncthreads();
            tc::fence_after_sync();
            if (tid == 0) {
                const uint32_t id = tc::idesc_bf16(kTRows, s.N1);
                for (int ks = 0; ks < s.KP / 16; ++ks)
                    tc::mma_bf16(tmem, tc::sdesc(sU + 256 * ks, 128, s.KP * 16), tc::sdesc(sW1 + 256 * ks, 128, s.KP * 16),
                                 id, ks > 0);
                tc::mma_commit(&bar);
            }
            bool ok = tc::mbar_wait(&bar, phase, a.wait_ns);
            if (__syncthreads_or(!ok)) { failed = true; break; }
            phase ^= 1u;
            tc::fence_after_sync();
            // ---- HID = relu(PRE + b1) -> BF16 operand of layer 2
            for (int c = 0; c < s.N1; c += 16) {
                float v[16];
                tc::tmem_ld16(tc::tmem_addr(tmem, warp, c), v);
                uint32_t pk[8];
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    __nv_bfloat162 t = __floats2bfloat162_rn(fmaxf(v[2 * j] + b1[c + 2 * j], 0.f),
                                                            fmaxf(v[2 * j + 1] + b1[c + 2 * j + 1], 0.f));
                    pk[j] = *reinterpret_cast<uint32_t *>(&t);
                }
                *reinterpret_cast<uint4 *>(sm + s.o_R + tc::kmajor_offset(tid, c, s.N1)) =
                    make_uint4(pk[0], pk[1], pk[2], pk[3]);
                *reinterpret_cast<uint4 *>(sm + s.o_R + tc::kmajor_offset(tid, c + 8, s.N1)) =
                    make_uint4(pk[4], pk[5], pk[6], pk[7]);
            }
            // ---- layer 2
            tc::fence_async_smem();
            tc::fence_before_sync();
            __syncthreads();
            tc::fence_after_sync();
            if (tid == 0) {
                const uint32_t sbo = s.N1 * 16;
                const uint32_t ioc = tc::idesc_bf16(kTRows, s.Noc), icov = tc::idesc_bf16(kTRows, s.Ncov);
                for (int ks = 0; ks < 2 * H / 16; ++ks)
                    tc::mma_bf16(tmem, tc::sdesc(sR + 256 * ks, 128, sbo), tc::sdesc(sW2oc + 256 * ks, 128, 2 * H * 16),
                                 ioc, ks > 0);
                const uint32_t hcov = sR + (2 * H / 8) * 128;
                for (int ks = 0; ks < H / 16; ++ks)
                    tc::mma_bf16(tmem + (uint32_t)s.Noc, tc::sdesc(hcov + 256 * ks, 128, sbo),
                                 tc::sdesc(sW2cov + 256 * ks, 128, H * 16), icov, ks > 0);
                tc::mma_commit(&bar);
            }
            ok = tc::mbar_wait(&bar, phase, a.wait_ns);
            if (__syncthreads_or(!ok)) { failed = true; break; }
            phase ^= 1u;
            tc::fence_after_sync();

            // ---- epilogue: this thread's row, if it belongs to partition p
            if (PROJ) {
                // each candidate decoded and projected straight to its splat record
                const bool mine = !done && pm == p;
                float el[6], xa[3];
#pragma unroll
                for (int e = 0; e < 6; ++e) el[e] = mine ? expf(__ldg(a.log_scaling + 6 * an + e)) : 0.f;
#pragma unroll
                for (int e = 0; e < 3; ++e) xa[e] = mine ? __ldg(a.xyz + 3 * an + e) : 0.f;
                const float *off = a.offsets + (size_t)(an >= 0 ? an : 0) * k * 3;
                const size_t c0 = (size_t)row * k;
                // the offsets of candidate i + 1 are loaded while candidate i is projected
                float on[3];
#pragma unroll
                for (int e = 0; e < 3; ++e) on[e] = mine ? __ldg(off + e) : 0.f;
                for (int i = 0; i < k; ++i) {
                    float vo[4], vc[8];
                    const float oc[3] = {on[0], on[1], on[2]};
#pragma unroll
                    for (int e = 0; e < 3; ++e) on[e] = (mine && i + 1 < k) ? __ldg(off + 3 * (i + 1) + e) : 0.f;
                    __syncwarp();
                    tc::tmem_ld4(tc::tmem_addr(tmem, warp, 4 * i), vo);            // all lanes: warp-collective
                    tc::tmem_ld8(tc::tmem_addr(tmem, warp, s.Noc + 8 * i), vc);
                    const size_t ci = c0 + i;
                    if (mine && idx_ok(a.st, (long long)ci, po.cap, 16)) {
                        const float op = tanh_fast(vo[0] + b2[4 * i]);
                        const float col[3] = {sigmoid_fast(vo[1] + b2[4 * i + 1]), sigmoid_fast(vo[2] + b2[4 * i + 2]),
                                              sigmoid_fast(vo[3] + b2[4 * i + 3])};
                        const float *bc = b2 + s.Noc + 8 * i;
                        const float sc[3] = {el[3] * sigmoid_fast(vc[0] + bc[0]), el[4] * sigmoid_fast(vc[1] + bc[1]),
                                             el[5] * sigmoid_fast(vc[2] + bc[2])};
                        float q[4] = {vc[3] + bc[3], vc[4] + bc[4], vc[5] + bc[5], vc[6] + bc[6]};
                        const float inv = rsqrtf(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
#pragma unroll
                        for (int e = 0; e < 4; ++e) q[e] *= inv;
                        const float m0 = xa[0] + oc[0] * el[0];
                        const float m1 = xa[1] + oc[1] * el[1];
                        const float m2 = xa[2] + oc[2] * el[2];
                        float4 r0 = make_float4(0.f, 0.f, 0.f, 0.f), r1 = r0, r2 = r0;
                        int nt = 0;
                        project_one(cam, (float)po.W[vw], (float)po.H[vw], po.TX[vw], po.TY[vw], m0, m1, m2, sc, q,
                                    op, col, r0, r1, r2, nt);
                        po.rec[3 * ci] = r0;
                        po.rec[3 * ci + 1] = r1;
                        po.rec[3 * ci + 2] = r2;
                        po.tiles[ci] = nt;
                    }
                }
                if (pm == p) done = true;
                tc::fence_before_sync();
                continue;
            }
            const bool mine = !done && pm == p;
            const bool mixed = !__all_sync(0xffffffffu, mine || pm < 0);   // rows of other partitions in the warp
            const size_t c0 = (size_t)row * k;
            // (a) opacity = tanh, colour = sigmoid
            for (int c = 0; c < s.Noc; c += 16) {
                float v[16];
                tc::tmem_ld16(tc::tmem_addr(tmem, warp, c), v);
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int i = c / 4 + j;
                    if (!mine || i >= k) continue;
                    const float op = tanh_fast(v[4 * j] + b2[c + 4 * j]);
                    const float r = sigmoid_fast(v[4 * j + 1] + b2[c + 4 * j + 1]);
                    const float g = sigmoid_fast(v[4 * j + 2] + b2[c + 4 * j + 2]);
                    const float bb = sigmoid_fast(v[4 * j + 3] + b2[c + 4 * j + 3]);
                    if (mixed) {
                        a.opacity[c0 + i] = op;
                        a.colour[3 * (c0 + i)] = r; a.colour[3 * (c0 + i) + 1] = g; a.colour[3 * (c0 + i) + 2] = bb;
                    } else {
                        stage[lane * k + i] = op;
                        float *sc = stage + 32 * k + lane * 3 * k + 3 * i;
                        sc[0] = r; sc[1] = g; sc[2] = bb;
                    }
                }
            }
            if (!mixed) {
                __syncwarp();
                stage_out(stage, a.opacity + (size_t)row0 * k, nval * k, vec & 1);
                stage_out(stage + 32 * k, a.colour + (size_t)row0 * 3 * k, nval * 3 * k, vec & 1);
                __syncwarp();
            }
            // (b) rotation = normalised quaternion
            for (int c = 0; c < s.Ncov; c += 16) {
                float v[16];
                tc::tmem_ld16(tc::tmem_addr(tmem, warp, s.Noc + c), v);
#pragma unroll
                for (int j = 0; j < 2; ++j) {
                    const int i = c / 8 + j;
                    if (!mine || i >= k) continue;
                    const float *bq = b2 + s.Noc + c + 8 * j + 3;
                    const float q0 = v[8 * j + 3] + bq[0], q1 = v[8 * j + 4] + bq[1];
                    const float q2 = v[8 * j + 5] + bq[2], q3 = v[8 * j + 6] + bq[3];
                    const float inv = rsqrtf(q0 * q0 + q1 * q1 + q2 * q2 + q3 * q3);
                    float *dst = mixed ? a.quat + 4 * (c0 + i) : stage + lane * 4 * k + 4 * i;
                    dst[0] = q0 * inv; dst[1] = q1 * inv; dst[2] = q2 * inv; dst[3] = q3 * inv;
                }
            }
            if (!mixed) {
                __syncwarp();
                stage_out(stage, a.quat + (size_t)row0 * 4 * k, nval * 4 * k, vec & 1);
                __syncwarp();
            }
            // (c) scale = exp(l[3:6]) * sigmoid
            float el[6];
#pragma unroll
            for (int j = 0; j < 6; ++j) el[j] = mine ? expf(__ldg(a.log_scaling + 6 * an + j)) : 0.f;
            for (int c = 0; c < s.Ncov; c += 16) {
                float v[16];
                tc::tmem_ld16(tc::tmem_addr(tmem, warp, s.Noc + c), v);
#pragma unroll
                for (int j = 0; j < 2; ++j) {
                    const int i = c / 8 + j;
                    if (!mine || i >= k) continue;
                    const float *bs = b2 + s.Noc + c + 8 * j;
                    float *dst = mixed ? a.scale + 3 * (c0 + i) : stage + lane * 3 * k + 3 * i;
#pragma unroll
                    for (int e = 0; e < 3; ++e) dst[e] = el[3 + e] * sigmoid_fast(v[8 * j + e] + bs[e]);
                }
            }
            if (!mixed) {
                __syncwarp();
                stage_out(stage, a.scale + (size_t)row0 * 3 * k, nval * 3 * k, vec & 1);
                __syncwarp();
            }
            // (d) positions mu = x_a + offset * exp(l[0:3])
            if (mine) {
                const float x0 = __ldg(a.xyz + 3 * an), x1 = __ldg(a.xyz + 3 * an + 1), x2 = __ldg(a.xyz + 3 * an + 2);
                const float *off = a.offsets + (size_t)an * k * 3;
                for (int i = 0; i < k; ++i) {
                    float *dst = mixed ? a.mu + 3 * (c0 + i) : stage + lane * 3 * k + 3 * i;
                    dst[0] = x0 + __ldg(off + 3 * i) * el[0];
                    dst[1] = x1 + __ldg(off + 3 * i + 1) * el[1];
                    dst[2] = x2 + __ldg(off + 3 * i + 2) * el[2];
                }
            }
            if (!mixed) {
                __syncwarp();
                stage_out(stage, a.mu + (size_t)row0 * 3 * k, nval * 3 * k, vec & 1);
            }
            if (pm == p) done = true;
            tc::fence_before_sync();
        }
    }
    if (failed) {
        if (tid == 0) set_error(a.st, GS_ERR_TIMEOUT, 15);
        tc::mbar_wait(&bar, phase);   // MMAs still in flight (bounded by the default limit)
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (warp == 0) tc::tmem_dealloc(tmem, (uint32_t)s.tcols);
}

// Shared memory, residency and grid of one decode_tc_kernel instantiation.
template <bool PROJ>
static int launch_decode_tc(const DecodeArgs &a, const ProjOut &po, cudaStream_t st)
{
    const TcShape s = tc_shape(a.F, a.k, a.H);
    if (a.H % 16 != 0 || s.N1 > 256 || s.Noc > 256 || s.Ncov > 256 || s.tcols > 256 || s.KP > 256 ||
        s.smem > 200 * 1024)
        return GS_ERR_UNSUPPORTED;
    // Device limits, read once: shared memory per SM and per-CTA reservation,
    // the kernel's static shared memory and registers.
    static int dev_smem = 0, dev_reserve = 0, static_smem = 0, regs = 0;
    if (dev_smem == 0) {
        int dev = 0;
        cudaFuncAttributes fa;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&dev_smem, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&dev_reserve, cudaDevAttrReservedSharedMemoryPerBlock, dev) != cudaSuccess ||
            cudaFuncGetAttributes(&fa, decode_tc_kernel<PROJ>) != cudaSuccess)
            return GS_ERR_CUDA;
        static_smem = (int)fa.sharedSizeBytes;
        regs = fa.numRegs;
    }
    // At most 512 / tcols CTAs may hold tensor memory on one SM: request enough
    // shared memory that no more than that many can be resident.
    const int max_res = 512 / s.tcols;
    const size_t per_cta = (size_t)static_smem + dev_reserve;
    size_t smem = s.smem;
    const size_t floor_bytes = (size_t)dev_smem / (max_res + 1) + 16 - std::min(per_cta, (size_t)dev_smem / (max_res + 1));
    if (smem < floor_bytes) smem = floor_bytes;
    if (smem + per_cta > (size_t)dev_smem) return GS_ERR_UNSUPPORTED;
    static size_t configured = 0;
    if (smem > configured) {
        // the whole unified L1 / shared array as shared memory, or the runtime
        // may size the carveout for fewer resident CTAs
        if (cudaFuncSetAttribute(decode_tc_kernel<PROJ>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
                cudaSuccess ||
            cudaFuncSetAttribute(decode_tc_kernel<PROJ>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 cudaSharedmemCarveoutMaxShared) != cudaSuccess)
            return GS_ERR_UNSUPPORTED;
        configured = smem;
    }
    int occ = (int)(dev_smem / (smem + per_cta));
    occ = std::min(occ, 65536 / std::max(1, regs * kTThreads));
    occ = std::min(occ, max_res);
    if (occ < 1) return GS_ERR_UNSUPPORTED;
    const bool vec_out = ((reinterpret_cast<uintptr_t>(a.opacity) | reinterpret_cast<uintptr_t>(a.colour) |
                           reinterpret_cast<uintptr_t>(a.quat) | reinterpret_cast<uintptr_t>(a.scale) |
                           reinterpret_cast<uintptr_t>(a.mu)) & 15) == 0;
    const bool vec_feat = (reinterpret_cast<uintptr_t>(a.feat) & 15) == 0 && a.F % 4 == 0;
    const long long tiles = (a.cap_rows + kTRows - 1) / kTRows;
    const int grid = (int)std::max<long long>(1, std::min<long long>(tiles, (long long)sm_count() * occ));
    decode_tc_kernel<PROJ><<<grid, kTThreads, smem, st>>>(a, s, (vec_out ? 1 : 0) | (vec_feat ? 2 : 0), po);
    count_launches(1);
    return cudaPeekAtLastError() == cudaSuccess ? GS_OK : GS_ERR_CUDA;
}

int launch_decode_bf16(const DecodeArgs &a, cudaStream_t st, const ProjOut *po)
{
    if (po) return launch_decode_tc<true>(a, *po, st);
    ProjOut none;
    none.rec = nullptr;
    none.tiles = nullptr;
    none.cap = 0;
    return launch_decode_tc<false>(a, none, st);
}

}  // namespace gs
