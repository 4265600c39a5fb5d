// decode_bwd_tc.cu -- reverse of the partitioned anchor decoder (Sec. III-A,
// Eq. 2; per-partition MLP sets of Eq. 6) on the 5th-generation tensor cores.
//
// Per tile of 128 rows (one thread per row, MMAs with M = 128, FP32
// accumulators in tensor memory), for each partition present in the tile:
//   1. PRE = U W1^T, recomputed in split BF16 (U = Uh + Ul, W1 = W1h + W1l,
//      three MMAs per k-step, about 2^-16 relative error): it decides the
//      relu masks, and a BF16-rounded recompute flips masks of
//      pre-activations near zero;
//   2. HID = relu(PRE + b1) in BF16; Z_oc = HID W2oc^T (opacity, colour) and
//      Z_cov = HID W2cov^T (scale, rotation) -- the same permuted output
//      layout as the forward decoder;
//   3. dZ through the activations (tanh, sigmoid, exp * sigmoid, quaternion
//      normalisation) from the candidates' gradients, with the per-anchor
//      terms of the scale and position parameters (atomics);
//   4. dHID = dZ W2 and dW2 += dZ^T [HID | 1];
//   5. dPRE = dHID * [PRE > 0]; dU = dPRE W1 and dW1 += dPRE^T [U | 1];
//   6. dU -> feature gradient, and through (d, |d|) of Eq. 2 -> position.
// Every operand is stored once in shared memory, K-major for the product
// that reads it first; the transposed products (dW1, dW2 and the products
// with W1 / W2 in steps 4-5) read the same bytes as MN-major operands.  The
// weight-gradient accumulators stay in tensor memory across the tiles of a
// partition and are added to global memory when the partition changes and at
// the end.  Constant-one columns (column 4 of U, column 3H of [HID | 1]) give
// the bias gradients from the same MMAs.
//
// Column order of U here: [d/|d| (3), |d|, 1, 0, 0, 0, f_a (F), 0 ...], so that
// the view inputs and the bias column sit at fixed positions of the first
// 16-column accumulator chunk; W1 is staged in the same column order.
#include <cuda_bf16.h>

#include "gs_internal.cuh"
#include "proj_bwd.cuh"
#include "tc05.cuh"

namespace gs {

constexpr int kBRows = 128;
constexpr int kBThreads = 128;

struct TbShape {
    int F, Din, KP, H, k, N1, Noc, Ncov, NZ, NH1, Wcols, tcols;
    int dout[3], hoff[3];
    uint32_t c_dW2, c_dW1;   // tensor-memory columns of the weight-gradient accumulators
    uint32_t o_Uh, o_A, o_HX, o_W1h, o_W1l, o_W2oc, o_W2cov, o_b1, o_b2;
    size_t smem;
};

static int up16b(int x) { return (x + 15) / 16 * 16; }

static TbShape tb_shape(int F, int k, int H)
{
    TbShape s;
    s.F = F; s.Din = F + 4; s.KP = up16b(8 + F); s.H = H; s.k = k;
    s.N1 = 3 * H;
    s.Noc = up16b(4 * k);
    s.Ncov = up16b(8 * k);
    s.NZ = s.Noc + s.Ncov;
    s.NH1 = s.N1 + 16;
    s.Wcols = std::max(std::max(s.N1, s.KP), std::max(s.Noc, s.Ncov));
    s.c_dW2 = (uint32_t)s.Wcols;
    s.c_dW1 = (uint32_t)(s.Wcols + s.NH1);
    const int need = s.Wcols + s.NH1 + s.KP;
    int c = 32;
    while (c < need) c <<= 1;
    s.tcols = c;
    const int d[3] = {k, 3 * k, 7 * k};
    int h = 0;
    for (int i = 0; i < 3; ++i) {
        s.dout[i] = d[i];
        s.hoff[i] = h;
        h += H * s.Din + H + d[i] * H + d[i];
    }
    size_t b = 0;
    auto take = [&](size_t bytes) { uint32_t at = (uint32_t)b; b = align_up(b + bytes, 128); return at; };
    s.o_Uh = take(2ull * kBRows * s.KP);
    // region A holds U lo, then dZ, then dPRE; 2 KB of slack after the largest:
    // the MN-major reads of dZ / dPRE with M = 128 run past their NZ / 3H
    // columns in the last 8-row group (those accumulator rows are never read)
    s.o_A = take(2ull * kBRows * std::max(std::max(s.KP, s.NZ), s.N1) + 2048);
    s.o_HX = take(2ull * kBRows * s.NH1);
    s.o_W1h = take(2ull * s.N1 * s.KP);
    s.o_W1l = take(2ull * s.N1 * s.KP);
    s.o_W2oc = take(2ull * s.Noc * 2 * H);
    s.o_W2cov = take(2ull * s.Ncov * H);
    s.o_b1 = take(4ull * s.N1);
    s.o_b2 = take(4ull * s.NZ);
    s.smem = b;
    return s;
}

__device__ __forceinline__ int head_off(const TbShape &s, int h)
{
    return h == 0 ? s.hoff[0] : (h == 1 ? s.hoff[1] : s.hoff[2]);
}

__device__ __forceinline__ void put_bf16(char *base, uint32_t off, float v)
{
    *reinterpret_cast<__nv_bfloat16 *>(base + off) = __float2bfloat16_rn(v);
}

// Eight columns (one 16-byte core-matrix row) of BF16 values.
__device__ __forceinline__ void put8_bf16(char *base, uint32_t off, const float u[8])
{
    uint4 pk;
    __nv_bfloat162 t0 = __floats2bfloat162_rn(u[0], u[1]), t1 = __floats2bfloat162_rn(u[2], u[3]);
    __nv_bfloat162 t2 = __floats2bfloat162_rn(u[4], u[5]), t3 = __floats2bfloat162_rn(u[6], u[7]);
    pk.x = *reinterpret_cast<uint32_t *>(&t0); pk.y = *reinterpret_cast<uint32_t *>(&t1);
    pk.z = *reinterpret_cast<uint32_t *>(&t2); pk.w = *reinterpret_cast<uint32_t *>(&t3);
    *reinterpret_cast<uint4 *>(base + off) = pk;
}

// Input index (into [f_a, d/|d|, |d|]) of U column c; Din for the bias
// column, -1 for padding.
__device__ __forceinline__ int u_input(const TbShape &s, int c)
{
    if (c < 4) return s.F + c;
    if (c == 4) return s.Din;
    if (c >= 8 && c < 8 + s.F) return c - 8;
    return -1;
}

// Partition p's weights: W1 as hi + lo BF16 parts (U column order), W2 in
// the permuted layer-2 layout of the forward decoder, FP32 biases.
__device__ void tb_stage_weights(const TbShape &s, char *sm, const float *__restrict__ w)
{
    const int tid = threadIdx.x, H = s.H, K2 = 2 * H;
    for (int idx = tid; idx < s.N1 * s.KP; idx += kBThreads) {
        const int j = idx / s.KP, c = idx % s.KP, h = j / H, jj = j % H, i = u_input(s, c);
        const float v = (i >= 0 && i < s.Din) ? __ldg(w + head_off(s, h) + jj * s.Din + i) : 0.f;
        const __nv_bfloat16 hi = __float2bfloat16_rn(v);
        const uint32_t off = tc::kmajor_offset(j, c, s.KP);
        *reinterpret_cast<__nv_bfloat16 *>(sm + s.o_W1h + off) = hi;
        put_bf16(sm + s.o_W1l, off, v - __bfloat162float(hi));
    }
    for (int idx = tid; idx < s.Noc * K2; idx += kBThreads) {
        const int o = idx / K2, kk = idx % K2, i = o >> 2, c = o & 3;
        float v = 0.f;
        if (i < s.k) {
            if (c == 0 && kk < H) v = __ldg(w + s.hoff[0] + H * s.Din + H + i * H + kk);
            else if (c > 0 && kk >= H) v = __ldg(w + s.hoff[1] + H * s.Din + H + (3 * i + c - 1) * H + (kk - H));
        }
        put_bf16(sm + s.o_W2oc, tc::kmajor_offset(o, kk, K2), v);
    }
    for (int idx = tid; idx < s.Ncov * H; idx += kBThreads) {
        const int o = idx / H, kk = idx % H, i = o >> 3, j = o & 7;
        const float v = (i < s.k && j < 7) ? __ldg(w + s.hoff[2] + H * s.Din + H + (7 * i + j) * H + kk) : 0.f;
        put_bf16(sm + s.o_W2cov, tc::kmajor_offset(o, kk, H), v);
    }
    float *b1 = reinterpret_cast<float *>(sm + s.o_b1);
    for (int j = tid; j < s.N1; j += kBThreads) b1[j] = __ldg(w + head_off(s, j / H) + H * s.Din + j % H);
    float *b2 = reinterpret_cast<float *>(sm + s.o_b2);
    for (int o = tid; o < s.NZ; o += kBThreads) {
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

// Adds the tensor-memory weight-gradient accumulators of partition p to
// global memory.  Thread t reads accumulator lane t: output unit t (permuted
// layout) of dW2 and hidden unit t of dW1.
__device__ void tb_flush(const TbShape &s, uint32_t tmem, float *__restrict__ g)
{
    const int tid = threadIdx.x, warp = tid >> 5, H = s.H;
    // dW2 [NZ (lanes) x NH1]: columns 0..3H-1 hidden units of all heads, 3H = bias
    int h = -1, lo = 0;
    if (tid < s.Noc) {
        const int i = tid >> 2, c = tid & 3;
        if (i < s.k) { h = c == 0 ? 0 : 1; lo = c == 0 ? i : 3 * i + c - 1; }
    } else if (tid < s.NZ) {
        const int oo = tid - s.Noc, i = oo >> 3, j = oo & 7;
        if (i < s.k && j < 7) { h = 2; lo = 7 * i + j; }
    }
    for (int c0 = 0; c0 < s.NH1; c0 += 16) {
        float v[16];
        tc::tmem_ld16(tc::tmem_addr(tmem, warp, s.c_dW2 + c0), v);
        if (h < 0) continue;
        const int ho = head_off(s, h), dout = h == 0 ? s.dout[0] : (h == 1 ? s.dout[1] : s.dout[2]);
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            const int col = c0 + j;
            if (col >= h * H && col < (h + 1) * H)
                atomicAdd(g + ho + H * s.Din + H + lo * H + (col - h * H), v[j]);
            else if (col == s.N1)
                atomicAdd(g + ho + H * s.Din + H + dout * H + lo, v[j]);
        }
    }
    // dW1 [N1 (lanes) x KP] in U column order; the bias column gives db1
    const int hj = tid / H, jj = tid % H;
    const int ho1 = tid < s.N1 ? head_off(s, hj) : 0;
    for (int c0 = 0; c0 < s.KP; c0 += 16) {
        float v[16];
        tc::tmem_ld16(tc::tmem_addr(tmem, warp, s.c_dW1 + c0), v);
        if (tid >= s.N1) continue;
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            const int i = u_input(s, c0 + j);
            if (i >= 0 && i < s.Din) atomicAdd(g + ho1 + jj * s.Din + i, v[j]);
            else if (i == s.Din) atomicAdd(g + ho1 + H * s.Din + jj, v[j]);
        }
    }
}

// Issues the MMAs of one step from thread 0 and waits for them (bounded);
// false (uniformly over the CTA) if the wait ran out.
template <typename F>
__device__ __forceinline__ bool tb_mma_step(uint64_t *bar, uint32_t &phase, unsigned long long wait_ns, F issue)
{
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (threadIdx.x == 0) {
        issue();
        tc::mma_commit(bar);
    }
    const bool ok = tc::mbar_wait(bar, phase, wait_ns);
    if (__syncthreads_or(!ok)) return false;
    phase ^= 1u;
    tc::fence_after_sync();
    return true;
}

__global__ void __launch_bounds__(kBThreads) decode_bwd_tc_kernel(DecodeBwdArgsB a, TbShape s)
{
    const DecodeArgs &f = a.f;
    if (__syncthreads_or(has_error(f.st))) return;   // block-uniform exit
    extern __shared__ __align__(1024) char sm[];
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t tslot;
    __shared__ int s_p, s_staged, s_accp;
    const int tid = threadIdx.x, warp = tid >> 5;
    const int k = s.k, H = s.H;
    if (warp == 0) {
        tc::tmem_alloc(&tslot, (uint32_t)s.tcols);
        tc::tmem_relinquish();
    }
    if (tid == 0) {
        tc::mbar_init(&bar, 1);
        s_staged = -1;
        s_accp = -1;
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = tslot;
    const uint32_t sUh = tc::smem_u32(sm + s.o_Uh), sA = tc::smem_u32(sm + s.o_A), sHX = tc::smem_u32(sm + s.o_HX);
    const uint32_t sW1h = tc::smem_u32(sm + s.o_W1h), sW1l = tc::smem_u32(sm + s.o_W1l);
    const uint32_t sW2oc = tc::smem_u32(sm + s.o_W2oc), sW2cov = tc::smem_u32(sm + s.o_W2cov);
    const float *b1 = reinterpret_cast<const float *>(sm + s.o_b1);
    const float *b2 = reinterpret_cast<const float *>(sm + s.o_b2);
    const int rows = __ldg(f.view_start + f.V);
    const int ntiles = (rows + kBRows - 1) / kBRows;
    const long long P = f.mlp_floats;
    uint32_t phase = 0;
    bool failed = false, fresh = true;   // fresh: the accumulators hold nothing yet

    // each CTA takes a contiguous range of tiles: rows are view-major and partition-sorted inside a
    // view, so a CTA meets few partitions (the weights are staged, and the weight gradients flushed,
    // only when the partition changes)
    const int per_cta = (ntiles + (int)gridDim.x - 1) / (int)gridDim.x;
    const int tile_end = min(ntiles, ((int)blockIdx.x + 1) * per_cta);
    for (int tile = (int)blockIdx.x * per_cta; tile < tile_end && !failed; ++tile) {
        // ---- row setup: anchor, partition, (d, |d|) of Eq. 2; U = [f, d/|d|, |d|, 1] as hi + lo
        const int row = tile * kBRows + tid;
        int an = -1, pm = -1, vw = 0;
        float d0 = 0.f, d1 = 0.f, d2 = 0.f, dl = 1.f;
        Cam cam;
        if (row < rows) {
            an = __ldg(f.row_anchor + row);
            if (!idx_ok(f.st, an, f.N, 63)) an = -1;
        }
        if (an >= 0) {
            pm = __ldg(f.part + an);
            if (!idx_ok(f.st, pm, f.M, 64)) { pm = -1; an = -1; }
        }
        if (an >= 0) {
            vw = view_of_row(f.view_start, f.V, row);
            cam = load_cam(f.cams, vw);
            const Cam &c = cam;
            float xc[3];
#pragma unroll
            for (int i = 0; i < 3; ++i) xc[i] = -(c.R[i] * c.t[0] + c.R[3 + i] * c.t[1] + c.R[6 + i] * c.t[2]);
            d0 = __ldg(f.xyz + 3 * an) - xc[0];
            d1 = __ldg(f.xyz + 3 * an + 1) - xc[1];
            d2 = __ldg(f.xyz + 3 * an + 2) - xc[2];
            dl = sqrtf(d0 * d0 + d1 * d1 + d2 * d2);
        }
        const float inv_dl = 1.f / dl;
        // U row (hi into Uh; lo into region A, where later steps of a pass
        // overwrite it, so every further pass of the tile writes it again)
        auto write_u = [&](bool hi_too) {
            const float *fr = f.feat + (size_t)(an >= 0 ? an : 0) * s.F;
            // 16-byte feature loads where the rows allow them (fewer requests of this uncoalesced read)
            const bool fvec = (s.F & 3) == 0 && (reinterpret_cast<uintptr_t>(f.feat) & 15) == 0;
            for (int kc = 0; kc < s.KP; kc += 8) {
                float u[8], lo[8], fv[8];
                if (an >= 0 && fvec && kc >= 8 && kc + 8 <= 8 + s.F) {
                    const float4 q0 = __ldg(reinterpret_cast<const float4 *>(fr + (kc - 8)));
                    const float4 q1 = __ldg(reinterpret_cast<const float4 *>(fr + (kc - 4)));
                    fv[0] = q0.x; fv[1] = q0.y; fv[2] = q0.z; fv[3] = q0.w;
                    fv[4] = q1.x; fv[5] = q1.y; fv[6] = q1.z; fv[7] = q1.w;
                } else {
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        const int c = kc + j;
                        fv[j] = (an >= 0 && c >= 8 && c < 8 + s.F) ? __ldg(fr + (c - 8)) : 0.f;
                    }
                }
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const int c = kc + j;
                    float x = 0.f;
                    if (an >= 0) {
                        if (c == 0) x = d0 * inv_dl;
                        else if (c == 1) x = d1 * inv_dl;
                        else if (c == 2) x = d2 * inv_dl;
                        else if (c == 3) x = dl;
                        else if (c == 4) x = 1.f;
                        else if (c >= 8 && c < 8 + s.F) x = fv[j];
                    }
                    u[j] = x;
                    lo[j] = x - __bfloat162float(__float2bfloat16_rn(x));
                }
                const uint32_t off = tc::kmajor_offset(tid, kc, s.KP);
                if (hi_too) put8_bf16(sm + s.o_Uh, off, u);
                put8_bf16(sm + s.o_A, off, lo);
            }
        };
        write_u(true);
        bool done = pm < 0, first_pass = true;

        for (;;) {
            if (tid == 0) s_p = 0x7fffffff;
            __syncthreads();
            if (!done) atomicMin(&s_p, pm);
            __syncthreads();
            const int p = s_p;
            if (p == 0x7fffffff) break;
            if (!first_pass) write_u(false);   // region A held dZ / dPRE of the previous pass
            first_pass = false;
            if (p != s_accp) {   // the accumulators belong to another partition: add them out
                if (s_accp >= 0) tb_flush(s, tmem, a.dmlp + (size_t)s_accp * P);
                fresh = true;
                tc::fence_before_sync();
                __syncthreads();
                if (tid == 0) s_accp = p;
            }
            if (p != s_staged) {
                tb_stage_weights(s, sm, f.mlp + (size_t)p * P);
                if (tid == 0) s_staged = p;
            }
            const bool mine = !done && pm == p;

            // ---- 1. PRE (split BF16)
            if (!tb_mma_step(&bar, phase, f.wait_ns, [&] {
                    const uint32_t id = tc::idesc_bf16(kBRows, s.N1);
                    const uint32_t sbo = s.KP * 16;
                    for (int ks = 0; ks < s.KP / 16; ++ks) {
                        const uint64_t uh = tc::sdesc(sUh + 256 * ks, 128, sbo), ul = tc::sdesc(sA + 256 * ks, 128, sbo);
                        const uint64_t wh = tc::sdesc(sW1h + 256 * ks, 128, sbo), wl = tc::sdesc(sW1l + 256 * ks, 128, sbo);
                        tc::mma_bf16(tmem, uh, wh, id, ks > 0);
                        tc::mma_bf16(tmem, ul, wh, id, 1);
                        tc::mma_bf16(tmem, uh, wl, id, 1);
                    }
                })) { failed = true; break; }
            // ---- 2. relu masks and [HID | 1] in BF16
            uint32_t mask[4] = {0u, 0u, 0u, 0u};   // bit j of hidden unit j: PRE > 0 (N1 <= 128)
#pragma unroll
            for (int cc = 0; cc < 8; ++cc) {
                const int c = 16 * cc;
                if (c >= s.N1) break;
                float v[16], hv[16];
                tc::tmem_ld16(tc::tmem_addr(tmem, warp, c), v);
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const float pre = v[j] + b1[c + j];
                    if (pre > 0.f) mask[cc >> 1] |= 1u << ((cc & 1) * 16 + j);
                    hv[j] = fmaxf(pre, 0.f);
                }
                put8_bf16(sm + s.o_HX, tc::kmajor_offset(tid, c, s.NH1), hv);
                put8_bf16(sm + s.o_HX, tc::kmajor_offset(tid, c + 8, s.NH1), hv + 8);
            }
            {
                const float one[8] = {mine ? 1.f : 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
                const float zero[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
                put8_bf16(sm + s.o_HX, tc::kmajor_offset(tid, s.N1, s.NH1), one);
                put8_bf16(sm + s.o_HX, tc::kmajor_offset(tid, s.N1 + 8, s.NH1), zero);
            }
            // ---- Z_oc = HID[:, 0:2H] W2oc^T
            if (!tb_mma_step(&bar, phase, f.wait_ns, [&] {
                    const uint32_t id = tc::idesc_bf16(kBRows, s.Noc), sbo = s.NH1 * 16;
                    for (int ks = 0; ks < 2 * H / 16; ++ks)
                        tc::mma_bf16(tmem, tc::sdesc(sHX + 256 * ks, 128, sbo),
                                     tc::sdesc(sW2oc + 256 * ks, 128, 2 * H * 16), id, ks > 0);
                })) { failed = true; break; }
            float zoc[64];   // Noc <= 64
#pragma unroll
            for (int cc = 0; cc < 4; ++cc)
                if (16 * cc < s.Noc) tc::tmem_ld16(tc::tmem_addr(tmem, warp, 16 * cc), zoc + 16 * cc);
            // ---- Z_cov = HID[:, 2H:3H] W2cov^T (runs while dZ_oc is computed)
            tc::fence_before_sync();
            __syncthreads();
            tc::fence_after_sync();
            if (tid == 0) {
                const uint32_t id = tc::idesc_bf16(kBRows, s.Ncov), sbo = s.NH1 * 16;
                const uint32_t hcov = sHX + (2 * H / 8) * 128;
                for (int ks = 0; ks < H / 16; ++ks)
                    tc::mma_bf16(tmem, tc::sdesc(hcov + 256 * ks, 128, sbo), tc::sdesc(sW2cov + 256 * ks, 128, H * 16),
                                 id, ks > 0);
                tc::mma_commit(&bar);
            }
            // ---- 3a. dZ of opacity (tanh) and colour (sigmoid); live = decoded opacity > 0
            uint32_t live = 0u;
            const size_t c0 = (size_t)row * k;
#pragma unroll
            for (int cc = 0; cc < 4; ++cc) {
                if (16 * cc >= s.Noc) break;
                float dz[16];
                // d opacity, d colour of the chunk's candidates: from their splat gradients (fused
                // with the projection's reverse; zero for a splat that covers no tile) or given --
                // every load issued before any is used
                float gin[16];
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int i = 4 * cc + j;
                    const bool ok = mine && i < k;
                    const size_t ci = c0 + (ok ? i : 0);
                    if (a.sgT) {   // row-tiled splat gradients: one coalesced load per value and warp
                        const float *sgp = a.sgT + ((size_t)tile * k + (ok ? i : 0)) * 9 * kBRows + tid;
#pragma unroll
                        for (int ch = 0; ch < 4; ++ch) gin[4 * j + ch] = ok ? __ldg(sgp + (5 + ch) * kBRows) : 0.f;
                    } else {
                        gin[4 * j] = ok ? __ldg(a.dopacity + ci) : 0.f;
#pragma unroll
                        for (int ch = 0; ch < 3; ++ch) gin[4 * j + 1 + ch] = ok ? __ldg(a.dcolour + 3 * ci + ch) : 0.f;
                    }
                }
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int i = 4 * cc + j, o = 16 * cc + 4 * j;
                    dz[4 * j] = dz[4 * j + 1] = dz[4 * j + 2] = dz[4 * j + 3] = 0.f;
                    if (!mine || i >= k) continue;
                    const float op = tanh_fast(zoc[o] + b2[o]);
                    if (!(op > 0.f)) continue;   // culled by decoding: no gradient
                    live |= 1u << i;
                    const float gop = gin[4 * j], gcol[3] = {gin[4 * j + 1], gin[4 * j + 2], gin[4 * j + 3]};
                    dz[4 * j] = gop * (1.f - op * op);
#pragma unroll
                    for (int ch = 0; ch < 3; ++ch) {
                        const float sg = sigmoid_fast(zoc[o + 1 + ch] + b2[o + 1 + ch]);
                        dz[4 * j + 1 + ch] = gcol[ch] * sg * (1.f - sg);
                    }
                }
                put8_bf16(sm + s.o_A, tc::kmajor_offset(tid, 16 * cc, s.NZ), dz);
                put8_bf16(sm + s.o_A, tc::kmajor_offset(tid, 16 * cc + 8, s.NZ), dz + 8);
            }
            {
                const bool ok = tc::mbar_wait(&bar, phase, f.wait_ns);
                if (__syncthreads_or(!ok)) { failed = true; break; }
                phase ^= 1u;
                tc::fence_after_sync();
            }
            // ---- 3b. dZ of scale (exp(l) sigmoid) and rotation (normalisation); per-anchor terms
            float el[6], gls[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f}, gx[3] = {0.f, 0.f, 0.f}, xa[3];
#pragma unroll
            for (int j = 0; j < 6; ++j) el[j] = mine ? expf(__ldg(f.log_scaling + 6 * an + j)) : 0.f;
#pragma unroll
            for (int j = 0; j < 3; ++j) xa[j] = mine ? __ldg(f.xyz + 3 * an + j) : 0.f;
            for (int cc = 0; cc < s.Ncov; cc += 16) {
                float v[16], dz[16];
                tc::tmem_ld16(tc::tmem_addr(tmem, warp, cc), v);
                // inputs of the chunk's two candidates, every load issued before any is used: the
                // offsets, and the splat gradients (d mean2d, d conic) or the given 3D gradients
                float pin[2][10], ofv[2][3];
                bool drawn[2];
#pragma unroll
                for (int j = 0; j < 2; ++j) {
                    const int i = cc / 8 + j;
                    const bool ok = i < k && (live >> i & 1u);
                    const size_t ci = c0 + (ok ? i : 0);
                    const float *off = f.offsets + ((size_t)(ok ? an : 0) * k + (ok ? i : 0)) * 3;
#pragma unroll
                    for (int e = 0; e < 3; ++e) ofv[j][e] = ok ? __ldg(off + e) : 0.f;
                    if (a.sgT) {
                        const float *sgp = a.sgT + ((size_t)tile * k + (ok ? i : 0)) * 9 * kBRows + tid;
#pragma unroll
                        for (int e = 0; e < 5; ++e) pin[j][e] = ok ? __ldg(sgp + e * kBRows) : 0.f;
#pragma unroll
                        for (int e = 5; e < 10; ++e) pin[j][e] = 0.f;
                        // zero for a splat that covers no tile: no projection reverse (and no
                        // arithmetic on a culled candidate's projection)
                        drawn[j] = ok && (pin[j][0] != 0.f || pin[j][1] != 0.f || pin[j][2] != 0.f ||
                                          pin[j][3] != 0.f || pin[j][4] != 0.f);
                    } else {
                        drawn[j] = ok;
#pragma unroll
                        for (int e = 0; e < 3; ++e) {
                            pin[j][e] = ok ? __ldg(a.dscale + 3 * ci + e) : 0.f;
                            pin[j][3 + e] = ok ? __ldg(a.dmu + 3 * ci + e) : 0.f;
                        }
#pragma unroll
                        for (int e = 0; e < 4; ++e) pin[j][6 + e] = ok ? __ldg(a.dquat + 4 * ci + e) : 0.f;
                    }
                }
#pragma unroll
                for (int j = 0; j < 2; ++j) {
                    const int i = cc / 8 + j, o = s.Noc + cc + 8 * j;
#pragma unroll
                    for (int e = 0; e < 8; ++e) dz[8 * j + e] = 0.f;
                    if (i >= k || !(live >> i & 1u)) continue;
                    float sgv[3], q[4], dsv[3], dq[4], dmv[3], qd = 0.f;
#pragma unroll
                    for (int e = 0; e < 3; ++e) sgv[e] = sigmoid_fast(v[8 * j + e] + b2[o + e]);
#pragma unroll
                    for (int e = 0; e < 4; ++e) q[e] = v[8 * j + 3 + e] + b2[o + 3 + e];
                    const float inv = rsqrtf(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
                    if (a.sgT) {
                        // the projection's reverse on the recomputed Gaussian: mean x_a + offset *
                        // exp(l[0:3]), scale exp(l[3:6]) sigmoid, unit quaternion
#pragma unroll
                        for (int e = 0; e < 3; ++e) dsv[e] = dmv[e] = 0.f;
#pragma unroll
                        for (int e = 0; e < 4; ++e) dq[e] = 0.f;
                        if (drawn[j]) {
                            const float sc[3] = {el[3] * sgv[0], el[4] * sgv[1], el[5] * sgv[2]};
                            const float qu[4] = {q[0] * inv, q[1] * inv, q[2] * inv, q[3] * inv};
                            proj_bwd_one(cam, (float)a.W[vw], (float)a.H[vw], xa[0] + ofv[j][0] * el[0],
                                         xa[1] + ofv[j][1] * el[1], xa[2] + ofv[j][2] * el[2], sc, qu, pin[j][0],
                                         pin[j][1], pin[j][2], pin[j][3], pin[j][4], dmv, dsv, dq);
                        }
                    } else {
#pragma unroll
                        for (int e = 0; e < 3; ++e) {
                            dsv[e] = pin[j][e];
                            dmv[e] = pin[j][3 + e];
                        }
#pragma unroll
                        for (int e = 0; e < 4; ++e) dq[e] = pin[j][6 + e];
                    }
#pragma unroll
                    for (int e = 0; e < 3; ++e) {
                        dz[8 * j + e] = dsv[e] * el[3 + e] * sgv[e] * (1.f - sgv[e]);
                        gls[3 + e] += dsv[e] * el[3 + e] * sgv[e];
                    }
#pragma unroll
                    for (int e = 0; e < 4; ++e) qd += q[e] * inv * dq[e];
#pragma unroll
                    for (int e = 0; e < 4; ++e) dz[8 * j + 3 + e] = (dq[e] - q[e] * inv * qd) * inv;
#pragma unroll
                    for (int e = 0; e < 3; ++e) {
                        const float gm = dmv[e];
                        gx[e] += gm;
                        atomicAdd(a.doff + ((size_t)an * k + i) * 3 + e, gm * el[e]);
                        gls[e] += gm * ofv[j][e] * el[e];
                    }
                }
                put8_bf16(sm + s.o_A, tc::kmajor_offset(tid, s.Noc + cc, s.NZ), dz);
                put8_bf16(sm + s.o_A, tc::kmajor_offset(tid, s.Noc + cc + 8, s.NZ), dz + 8);
            }
            if (mine) {
#pragma unroll
                for (int j = 0; j < 6; ++j) atomicAdd(a.dls + 6 * an + j, gls[j]);
            }
            // ---- 4. dHID = dZ W2 (W2 read MN-major); dW2 += dZ^T [HID | 1]
            const uint32_t acc = fresh ? 0u : 1u;
            if (!tb_mma_step(&bar, phase, f.wait_ns, [&] {
                    const uint32_t ioc = tc::idesc_bf16(kBRows, 2 * H, 0, 1), icov = tc::idesc_bf16(kBRows, H, 0, 1);
                    const uint32_t zsbo = s.NZ * 16;
                    for (int ks = 0; ks < s.Noc / 16; ++ks)
                        tc::mma_bf16(tmem, tc::sdesc(sA + 256 * ks, 128, zsbo),
                                     tc::sdesc(sW2oc + 2 * ks * (2 * H * 16), 2 * H * 16, 128), ioc, ks > 0);
                    const uint32_t zcov = sA + (s.Noc / 8) * 128;
                    for (int ks = 0; ks < s.Ncov / 16; ++ks)
                        tc::mma_bf16(tmem + 2 * H, tc::sdesc(zcov + 256 * ks, 128, zsbo),
                                     tc::sdesc(sW2cov + 2 * ks * (H * 16), H * 16, 128), icov, ks > 0);
                    const uint32_t iw2 = tc::idesc_bf16(kBRows, s.NH1, 1, 1);
                    for (int ks = 0; ks < kBRows / 16; ++ks)
                        tc::mma_bf16(tmem + s.c_dW2, tc::sdesc(sA + 2 * ks * zsbo, zsbo, 128),
                                     tc::sdesc(sHX + 2 * ks * (s.NH1 * 16), s.NH1 * 16, 128), iw2, acc | (ks > 0));
                })) { failed = true; break; }
            // ---- 5. dPRE = dHID * mask (region A: dZ is no longer read)
#pragma unroll
            for (int cc = 0; cc < 8; ++cc) {
                const int c = 16 * cc;
                if (c >= s.N1) break;
                float v[16];
                tc::tmem_ld16(tc::tmem_addr(tmem, warp, c), v);
#pragma unroll
                for (int j = 0; j < 16; ++j)
                    if (!mine || !(mask[cc >> 1] >> ((cc & 1) * 16 + j) & 1u)) v[j] = 0.f;
                put8_bf16(sm + s.o_A, tc::kmajor_offset(tid, c, s.N1), v);
                put8_bf16(sm + s.o_A, tc::kmajor_offset(tid, c + 8, s.N1), v + 8);
            }
            // dU = dPRE W1 (W1 read MN-major); dW1 += dPRE^T [U | 1]
            if (!tb_mma_step(&bar, phase, f.wait_ns, [&] {
                    const uint32_t iu = tc::idesc_bf16(kBRows, s.KP, 0, 1), psbo = s.N1 * 16, usbo = s.KP * 16;
                    for (int ks = 0; ks < s.N1 / 16; ++ks)
                        tc::mma_bf16(tmem, tc::sdesc(sA + 256 * ks, 128, psbo), tc::sdesc(sW1h + 2 * ks * usbo, usbo, 128),
                                     iu, ks > 0);
                    const uint32_t iw1 = tc::idesc_bf16(kBRows, s.KP, 1, 1);
                    for (int ks = 0; ks < kBRows / 16; ++ks)
                        tc::mma_bf16(tmem + s.c_dW1, tc::sdesc(sA + 2 * ks * psbo, psbo, 128),
                                     tc::sdesc(sUh + 2 * ks * usbo, usbo, 128), iw1, acc | (ks > 0));
                })) { failed = true; break; }
            fresh = false;
            // ---- 6. features, and the view inputs of Eq. 2 -> position
            for (int c = 0; c < s.KP; c += 16) {
                float v[16];
                tc::tmem_ld16(tc::tmem_addr(tmem, warp, c), v);   // all lanes: a warp-collective load
                if (!mine) continue;
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const int i = c + j - 8;
                    if (i >= 0 && i < s.F) atomicAdd(a.dfeat + (size_t)an * s.F + i, v[j]);
                }
                if (c == 0) {   // columns 0..3: d/|d| and |d|
                    const float dir[3] = {d0 * inv_dl, d1 * inv_dl, d2 * inv_dl};
                    const float dd = v[0] * dir[0] + v[1] * dir[1] + v[2] * dir[2];
#pragma unroll
                    for (int e = 0; e < 3; ++e)
                        atomicAdd(a.dxyz + 3 * an + e, (v[e] - dir[e] * dd) * inv_dl + v[3] * dir[e] + gx[e]);
                }
            }
            if (pm == p) done = true;
            tc::fence_before_sync();
        }
    }
    if (failed) {
        if (tid == 0) set_error(f.st, GS_ERR_TIMEOUT, 65);
        tc::mbar_wait(&bar, phase);   // MMAs still in flight (bounded by the default limit)
    } else {
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
        if (s_accp >= 0) tb_flush(s, tmem, a.dmlp + (size_t)s_accp * P);
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (warp == 0) tc::tmem_dealloc(tmem, (uint32_t)s.tcols);
}

int launch_decode_bwd_bf16(const DecodeBwdArgsB &a, cudaStream_t st)
{
    const TbShape s = tb_shape(a.f.F, a.f.k, a.f.H);
    if (a.f.H % 16 != 0 || s.N1 > 128 || s.NZ > 128 || s.Noc > 64 || s.KP > 256 || s.tcols > 512 ||
        s.k > 32 || s.smem > 200 * 1024)
        return GS_ERR_UNSUPPORTED;
    static int dev_smem = 0, dev_reserve = 0, static_smem = 0, regs = 0;
    if (dev_smem == 0) {
        int dev = 0;
        cudaFuncAttributes fa;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&dev_smem, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&dev_reserve, cudaDevAttrReservedSharedMemoryPerBlock, dev) != cudaSuccess ||
            cudaFuncGetAttributes(&fa, decode_bwd_tc_kernel) != cudaSuccess)
            return GS_ERR_CUDA;
        static_smem = (int)fa.sharedSizeBytes;
        regs = fa.numRegs;
    }
    // at most 512 / tcols CTAs with tensor memory per SM (see the forward decoder)
    const int max_res = 512 / s.tcols;
    const size_t per_cta = (size_t)static_smem + dev_reserve;
    size_t smem = s.smem;
    const size_t floor_bytes = (size_t)dev_smem / (max_res + 1) + 16 - std::min(per_cta, (size_t)dev_smem / (max_res + 1));
    if (smem < floor_bytes) smem = floor_bytes;
    if (smem + per_cta > (size_t)dev_smem) return GS_ERR_UNSUPPORTED;
    static size_t configured = 0;
    if (smem > configured) {
        if (cudaFuncSetAttribute(decode_bwd_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
                cudaSuccess ||
            cudaFuncSetAttribute(decode_bwd_tc_kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 cudaSharedmemCarveoutMaxShared) != cudaSuccess)
            return GS_ERR_UNSUPPORTED;
        configured = smem;
    }
    int occ = (int)(dev_smem / (smem + per_cta));
    occ = std::min(occ, 65536 / std::max(1, regs * kBThreads));
    occ = std::min(occ, max_res);
    if (occ < 1) return GS_ERR_UNSUPPORTED;
    const long long tiles = (a.f.cap_rows + kBRows - 1) / kBRows;
    const int grid = (int)std::max<long long>(1, std::min<long long>(tiles, (long long)sm_count() * occ));
    decode_bwd_tc_kernel<<<grid, kBThreads, smem, st>>>(a, s);
    count_launches(1);
    return cudaPeekAtLastError() == cudaSuccess ? GS_OK : GS_ERR_CUDA;
}

}  // namespace gs
