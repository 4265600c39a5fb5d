// decode_bwd_bf16.cu -- reverse of the partitioned anchor decoder on BF16
// tensor cores (mma.sync m16n8k16, FP32 accumulation).
//
// Per tile of 64 rows (4 warps x 16 rows), for each partition present:
//   1. recompute PRE = U W1^T + b1 and Z = relu(PRE) W2^T + b2   (split-BF16 MMA)
//   2. dZ through the activations from the candidates' gradients (FP32), with
//      the per-anchor terms of scale and position (atomics)
//   3. dHID = dZ_h W2_h, dPRE = dHID * [PRE > 0]        (split-BF16 MMA)
//   4. dU = dPRE W1 -> d feature, and through d_ac, delta_ac (Eq. 2) -> d x_a
//                                                         (split-BF16 MMA)
//   5. dW1 += dPRE^T [U | 1], dW2 += dZ^T [HID | 1]      (BF16 MMA, K = rows)
// Steps 1, 3 and 4 sum ~100 terms with cancellation (and step 1 decides the
// relu masks), so their operands are split into BF16 hi + lo parts (three MMAs
// per product, ~2^-16 relative error) from FP32 copies in shared memory: the
// gradients are those of the decoder at the anchors' FP32 parameters.
// The weight-gradient accumulators stay in registers across tiles of the same
// partition and are added to global memory when the partition changes and at
// the end.  Constant-one columns give the bias gradients from the same MMAs.
#include "gs_internal.cuh"
#include "mma_bf16.cuh"

namespace gs {

constexpr int kBRows = 64;
constexpr int kBThreads = 128;
constexpr int kBLdr = kBRows + 8;   // row stride of the [feature][row] (transposed) tiles

struct BwdShape {
    int F, Din, KP, H, k, H3;
    int dout[3], dpad[3], off[3], NZ;   // head output blocks padded to 16 (k-step aligned)
    int hoff[3];
    int ldw1, ldw1t, ldw2, ldw2t[3], ldu, ldz, lddu;
    // smem offsets (bytes); W2T holds one [H][dpad_h] block per head
    size_t o_W1s, o_W1T, o_W2s, o_W2T, o_W2Th[3], o_Us, o_UT, o_HT, o_dZT, o_Zs, o_dPT, o_dUs, o_b1, o_b2, o_rd, o_ri;
    size_t smem;
};

static BwdShape bwd_shape(int F, int k, int H)
{
    BwdShape s;
    s.F = F; s.Din = F + 4; s.KP = (s.Din + 1 + 15) / 16 * 16;   // + the constant-one column
    s.H = H; s.k = k; s.H3 = 3 * H;
    const int d[3] = {k, 3 * k, 7 * k};
    int o = 0, h = 0;
    for (int i = 0; i < 3; ++i) {
        s.dout[i] = d[i];
        s.dpad[i] = (d[i] + 15) / 16 * 16;
        s.off[i] = o;
        o += s.dpad[i];
        s.hoff[i] = h;
        h += H * s.Din + H + d[i] * H + d[i];
    }
    s.NZ = o;
    s.ldw1 = s.KP + 4;        // W1s  [3H][KP] fp32
    s.ldw1t = s.H3 + 4;       // W1T  [KP][3H] fp32
    s.ldw2 = H + 4;           // W2s  [NZ][H]  fp32
    for (int i = 0; i < 3; ++i) s.ldw2t[i] = s.dpad[i] + 4;   // W2T_h [H][dpad_h] fp32
    s.ldu = s.KP + 4;         // Us   [64][KP] fp32
    s.ldz = s.NZ + 4;         // Zs   [64][NZ] fp32: Z, then dZ in place
    s.lddu = s.KP + 4;        // dUs  [64][KP] fp32
    size_t b = 0;
    auto take = [&](size_t bytes) { size_t at = b; b = (b + bytes + 15) / 16 * 16; return at; };
    s.o_W1s = take(4ull * s.H3 * s.ldw1);
    s.o_W1T = take(4ull * s.KP * s.ldw1t);
    s.o_W2s = take(4ull * s.NZ * s.ldw2);
    s.o_W2T = 0;
    for (int i = 0; i < 3; ++i) s.o_W2Th[i] = take(4ull * H * s.ldw2t[i]);
    s.o_Us = take(4ull * kBRows * s.ldu);
    s.o_UT = take(2ull * s.KP * kBLdr);
    s.o_HT = take(2ull * 3 * (H + 8) * kBLdr);           // [head][H + 8][row]: HID^T plus a row of ones
    s.o_dZT = take(2ull * s.NZ * kBLdr);
    s.o_Zs = take(4ull * kBRows * s.ldz);
    s.o_dPT = take(2ull * s.H3 * kBLdr);
    s.o_dUs = take(4ull * kBRows * s.lddu);
    s.o_b1 = take(4ull * s.H3);
    s.o_b2 = take(4ull * s.NZ);
    s.o_rd = take(4ull * kBRows * 7);   // per row: d (3), delta, then the position gradient via mu (3)
    s.o_ri = take(4ull * kBRows * 3);
    s.smem = b;
    return s;
}

struct BwdSmem {
    __nv_bfloat16 *UT, *HT, *dZT, *dPT;
    float *W1s, *W1T, *W2s, *W2T[3], *Us, *Zs, *dUs, *b1, *b2, *rd, *gxs;
    int *ran, *rpart, *rdone;
};

__device__ __forceinline__ BwdSmem bwd_smem(char *base, const BwdShape &s)
{
    BwdSmem m;
    m.W1s = reinterpret_cast<float *>(base + s.o_W1s);
    m.W1T = reinterpret_cast<float *>(base + s.o_W1T);
    m.W2s = reinterpret_cast<float *>(base + s.o_W2s);
    for (int i = 0; i < 3; ++i) m.W2T[i] = reinterpret_cast<float *>(base + s.o_W2Th[i]);
    m.Us = reinterpret_cast<float *>(base + s.o_Us);
    m.UT = reinterpret_cast<__nv_bfloat16 *>(base + s.o_UT);
    m.HT = reinterpret_cast<__nv_bfloat16 *>(base + s.o_HT);
    m.dZT = reinterpret_cast<__nv_bfloat16 *>(base + s.o_dZT);
    m.Zs = reinterpret_cast<float *>(base + s.o_Zs);
    m.dPT = reinterpret_cast<__nv_bfloat16 *>(base + s.o_dPT);
    m.dUs = reinterpret_cast<float *>(base + s.o_dUs);
    m.b1 = reinterpret_cast<float *>(base + s.o_b1);
    m.b2 = reinterpret_cast<float *>(base + s.o_b2);
    m.rd = reinterpret_cast<float *>(base + s.o_rd);
    m.gxs = m.rd + 4 * kBRows;
    int *ri = reinterpret_cast<int *>(base + s.o_ri);
    m.ran = ri;
    m.rpart = ri + kBRows;
    m.rdone = ri + 2 * kBRows;
    return m;
}

__device__ __forceinline__ int head_of(const BwdShape &s, int o) { return o < s.off[1] ? 0 : (o < s.off[2] ? 1 : 2); }

__device__ void bwd_stage_weights(const BwdShape &s, const BwdSmem &m, const float *__restrict__ mlp_p)
{
    const int tid = threadIdx.x;
    for (int idx = tid; idx < s.H3 * s.KP; idx += kBThreads) {
        const int j = idx / s.KP, i = idx % s.KP, h = j / s.H, jj = j % s.H;
        const float w = i < s.Din ? __ldg(mlp_p + s.hoff[h] + jj * s.Din + i) : 0.f;
        m.W1s[j * s.ldw1 + i] = w;
        m.W1T[i * s.ldw1t + j] = w;
    }
    for (int j = tid; j < s.H3; j += kBThreads) {
        const int h = j / s.H, jj = j % s.H;
        m.b1[j] = __ldg(mlp_p + s.hoff[h] + s.H * s.Din + jj);
    }
    for (int idx = tid; idx < s.NZ * s.H; idx += kBThreads) {
        const int o = idx / s.H, j = idx % s.H;
        const int h = head_of(s, o), lo = o - s.off[h];
        const float w = lo < s.dout[h] ? __ldg(mlp_p + s.hoff[h] + s.H * s.Din + s.H + lo * s.H + j) : 0.f;
        m.W2s[o * s.ldw2 + j] = w;
        float *wt = h == 0 ? m.W2T[0] : (h == 1 ? m.W2T[1] : m.W2T[2]);
        const int ld = h == 0 ? s.ldw2t[0] : (h == 1 ? s.ldw2t[1] : s.ldw2t[2]);
        wt[j * ld + lo] = w;
    }
    for (int o = tid; o < s.NZ; o += kBThreads) {
        const int h = head_of(s, o), lo = o - s.off[h];
        m.b2[o] = lo < s.dout[h] ? __ldg(mlp_p + s.hoff[h] + s.H * s.Din + s.H + s.dout[h] * s.H + lo) : 0.f;
    }
}

__device__ void bwd_load_rows(const DecodeArgs &a, const BwdShape &s, const BwdSmem &m, int tile, int rows)
{
    const int tid = threadIdx.x;
    if (tid < kBRows) {
        const int r = tile * kBRows + tid;
        int an = -1, pm = -1;
        float d0 = 0.f, d1 = 0.f, d2 = 0.f, dl = 1.f;
        if (r < rows) {
            an = __ldg(a.row_anchor + r);
            if (!idx_ok(a.st, an, a.N, 63)) an = -1;
        }
        if (an >= 0) {
            pm = __ldg(a.part + an);
            if (!idx_ok(a.st, pm, a.M, 64)) { pm = -1; an = -1; }
        }
        if (an >= 0) {
            const int v = view_of_row(a.view_start, a.V, r);
            const Cam c = load_cam(a.cams, v);
            float xc[3];
#pragma unroll
            for (int i = 0; i < 3; ++i) xc[i] = -(c.R[i] * c.t[0] + c.R[3 + i] * c.t[1] + c.R[6 + i] * c.t[2]);
            d0 = __ldg(a.xyz + 3 * an) - xc[0];
            d1 = __ldg(a.xyz + 3 * an + 1) - xc[1];
            d2 = __ldg(a.xyz + 3 * an + 2) - xc[2];
            dl = sqrtf(d0 * d0 + d1 * d1 + d2 * d2);
        }
        m.ran[tid] = an;
        m.rpart[tid] = pm;
        m.rdone[tid] = pm < 0;
        m.rd[4 * tid] = d0; m.rd[4 * tid + 1] = d1; m.rd[4 * tid + 2] = d2; m.rd[4 * tid + 3] = dl;
    }
    __syncthreads();
    // thread (r = tid / 2, half = tid % 2) fills columns half, half + 2, ... of row r
    {
        const int r = tid >> 1, h0 = tid & 1;
        const int an = m.ran[r];
        const float inv = 1.f / m.rd[4 * r + 3];
        for (int i = h0; i < s.KP; i += 2) {
            float u = 0.f;
            if (an >= 0) {
                if (i < s.F) u = __ldg(a.feat + (size_t)an * s.F + i);
                else if (i < s.F + 3) u = m.rd[4 * r + (i - s.F)] * inv;
                else if (i == s.F + 3) u = m.rd[4 * r + 3];
                else if (i == s.Din) u = 1.f;   // constant input: gives the bias gradient of layer 1
            }
            m.Us[r * s.ldu + i] = u;
            m.UT[i * kBLdr + r] = __float2bfloat16_rn(u);
        }
    }
}

template <int KS, int HT, int NT1, int NT2, int NH>
struct BwdAcc {
    float w1[NT1][4];   // dW1 output tiles owned by this warp
    float w2[NT2][4];   // dW2 output tiles owned by this warp
};

// Output tiles of the weight-gradient GEMMs, distributed round-robin over warps.
//   dW1: (3H/16) x (KP/8) tiles of 16x8;  dW2: per head (dpad/16) x ((H+8)/8) tiles.
__device__ __forceinline__ void w1_tile(const BwdShape &s, int idx, int *m0, int *n0)
{
    const int nt = s.KP / 8;
    *m0 = (idx / nt) * 16;
    *n0 = (idx % nt) * 8;
}
__device__ __forceinline__ bool w2_tile(const BwdShape &s, int idx, int *h, int *m0, int *n0)
{
    const int nt = (s.H + 8) / 8;
    int base = 0;
    for (int hh = 0; hh < 3; ++hh) {
        const int cnt = (s.dpad[hh] / 16) * nt;
        if (idx < base + cnt) {
            const int l = idx - base;
            *h = hh;
            *m0 = s.off[hh] + (l / nt) * 16;
            *n0 = (l % nt) * 8;
            return true;
        }
        base += cnt;
    }
    return false;
}

template <int KS, int HT, int NT1, int NT2, int NH>
__device__ void flush_acc(const BwdShape &s, BwdAcc<KS, HT, NT1, NT2, NH> &acc, float *__restrict__ dmlp_p)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, q = lane & 3;
    const int n1 = (s.H3 / 16) * (s.KP / 8);
#pragma unroll
    for (int t = 0; t < NT1; ++t) {
        const int idx = warp + 4 * t;
        if (idx < n1) {
            int m0, n0;
            w1_tile(s, idx, &m0, &n0);
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int j = m0 + g + (e >= 2 ? 8 : 0), i = n0 + 2 * q + (e & 1);
                const int h = j / s.H, jj = j % s.H;
                const float v = acc.w1[t][e];
                if (i < s.Din) atomicAdd(dmlp_p + s.hoff[h] + jj * s.Din + i, v);
                else if (i == s.Din) atomicAdd(dmlp_p + s.hoff[h] + s.H * s.Din + jj, v);
                acc.w1[t][e] = 0.f;
            }
        }
    }
#pragma unroll
    for (int t = 0; t < NT2; ++t) {
        int h, m0, n0;
        if (w2_tile(s, warp + 4 * t, &h, &m0, &n0)) {
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int o = m0 + g + (e >= 2 ? 8 : 0), jj = n0 + 2 * q + (e & 1);
                const int lo = o - s.off[h];
                const float v = acc.w2[t][e];
                if (lo < s.dout[h]) {
                    if (jj < s.H) atomicAdd(dmlp_p + s.hoff[h] + s.H * s.Din + s.H + lo * s.H + jj, v);
                    else if (jj == s.H) atomicAdd(dmlp_p + s.hoff[h] + s.H * s.Din + s.H + s.dout[h] * s.H + lo, v);
                }
                acc.w2[t][e] = 0.f;
            }
        }
    }
}

template <int KS, int HT, int NT1, int NT2, int NH>
__global__ void __launch_bounds__(kBThreads) decode_bwd_bf16_kernel(DecodeBwdArgsB a, BwdShape s)
{
    if (has_error(a.f.st)) return;
    extern __shared__ __align__(16) char smem_raw[];
    const BwdSmem m = bwd_smem(smem_raw, s);
    __shared__ int s_p, s_staged, s_accp;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, g = lane >> 2, q = lane & 3;
    const int m0w = warp * 16;
    const int rows = __ldg(a.f.view_start + a.f.V);
    const int ntiles = (rows + kBRows - 1) / kBRows;
    const long long P = a.f.mlp_floats;
    const int k = s.k;
    if (tid == 0) { s_staged = -1; s_accp = -1; }
    BwdAcc<KS, HT, NT1, NT2, NH> acc;
#pragma unroll
    for (int t = 0; t < NT1; ++t)
#pragma unroll
        for (int e = 0; e < 4; ++e) acc.w1[t][e] = 0.f;
#pragma unroll
    for (int t = 0; t < NT2; ++t)
#pragma unroll
        for (int e = 0; e < 4; ++e) acc.w2[t][e] = 0.f;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        __syncthreads();
        bwd_load_rows(a.f, s, m, tile, rows);
        __syncthreads();
        for (;;) {
            if (tid == 0) {
                int p = -1;
                for (int r = 0; r < kBRows; ++r)
                    if (!m.rdone[r]) { p = m.rpart[r]; break; }
                s_p = p;
            }
            __syncthreads();
            const int p = s_p;
            if (p < 0) break;
            if (p != s_accp) {   // the accumulators belong to another partition: add them out
                const int old = s_accp;
                if (old >= 0) flush_acc<KS, HT, NT1, NT2, NH>(s, acc, a.dmlp + (size_t)old * P);
                __syncthreads();
                if (tid == 0) s_accp = p;
            }
            if (p != s_staged) {
                bwd_stage_weights(s, m, a.f.mlp + (size_t)p * P);
                __syncthreads();
                if (tid == 0) s_staged = p;
            }
            // ---- 1. recompute both layers (split-BF16); HID^T (+ ones) to smem, relu masks kept
            uint32_t uh[KS][4], ul[KS][4];
#pragma unroll
            for (int ks = 0; ks < KS; ++ks) load_a_split(uh[ks], ul[ks], m.Us, s.ldu, m0w, 16 * ks);
            uint32_t mask[NH];   // bit (2*t+half)*4+e of head h: PRE > 0
#pragma unroll
            for (int h = 0; h < NH; ++h) {
                mask[h] = 0u;
                uint32_t hh[HT][4], hl[HT][4];
#pragma unroll
                for (int t = 0; t < HT; ++t) {
                    float c[2][4];
                    const int n0 = h * s.H + 16 * t;
#pragma unroll
                    for (int hf = 0; hf < 2; ++hf) {
                        c[hf][0] = c[hf][2] = m.b1[n0 + 8 * hf + 2 * q];
                        c[hf][1] = c[hf][3] = m.b1[n0 + 8 * hf + 2 * q + 1];
#pragma unroll
                        for (int ks = 0; ks < KS; ++ks) {
                            uint32_t bh[2], bl[2];
                            load_b_split(bh, bl, m.W1s, s.ldw1, 16 * ks, n0 + 8 * hf);
                            mma_split(c[hf], uh[ks], ul[ks], bh, bl);
                        }
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            if (c[hf][e] > 0.f) mask[h] |= 1u << ((2 * t + hf) * 4 + e);
                            c[hf][e] = fmaxf(c[hf][e], 0.f);
                        }
                        // HID^T rows (hidden unit) x cols (row of the tile)
                        const int jl = 16 * t + 8 * hf + 2 * q;
                        __nv_bfloat16 *ht = m.HT + (size_t)(h * (s.H + 8)) * kBLdr;
                        ht[jl * kBLdr + m0w + g] = __float2bfloat16_rn(c[hf][0]);
                        ht[(jl + 1) * kBLdr + m0w + g] = __float2bfloat16_rn(c[hf][1]);
                        ht[jl * kBLdr + m0w + g + 8] = __float2bfloat16_rn(c[hf][2]);
                        ht[(jl + 1) * kBLdr + m0w + g + 8] = __float2bfloat16_rn(c[hf][3]);
                    }
                    split_bf16(c[0][0], c[0][1], hh[t][0], hl[t][0]);
                    split_bf16(c[0][2], c[0][3], hh[t][1], hl[t][1]);
                    split_bf16(c[1][0], c[1][1], hh[t][2], hl[t][2]);
                    split_bf16(c[1][2], c[1][3], hh[t][3], hl[t][3]);
                }
                {   // ones row (bias of layer 2) and zero padding rows of HID^T
                    __nv_bfloat16 *ht = m.HT + (size_t)(h * (s.H + 8) + s.H) * kBLdr;
                    for (int idx = lane; idx < 8 * 16; idx += 32) {
                        const int jr = idx / 16, rr = m0w + idx % 16;
                        ht[jr * kBLdr + rr] = __float2bfloat16_rn(jr == 0 && m.rpart[rr] == p ? 1.f : 0.f);
                    }
                }
                for (int n0 = s.off[h]; n0 < s.off[h] + s.dpad[h]; n0 += 8) {
                    float z[4];
                    z[0] = z[2] = m.b2[n0 + 2 * q];
                    z[1] = z[3] = m.b2[n0 + 2 * q + 1];
#pragma unroll
                    for (int t = 0; t < HT; ++t) {
                        uint32_t bh[2], bl[2];
                        load_b_split(bh, bl, m.W2s, s.ldw2, 16 * t, n0);
                        mma_split(z, hh[t], hl[t], bh, bl);
                    }
                    m.Zs[(m0w + g) * s.ldz + n0 + 2 * q] = z[0];
                    m.Zs[(m0w + g) * s.ldz + n0 + 2 * q + 1] = z[1];
                    m.Zs[(m0w + g + 8) * s.ldz + n0 + 2 * q] = z[2];
                    m.Zs[(m0w + g + 8) * s.ldz + n0 + 2 * q + 1] = z[3];
                }
            }
            __syncthreads();
            // ---- 2. dZ through the activations, in place of Z, and dZ^T in BF16 for the
            //         dW2 GEMM.  Two threads per row (candidates of one parity each); every
            //         output column of the row, padding and foreign rows included, is written.
            {
                const int r = tid >> 1, par = tid & 1;
                const int an = m.ran[r];
                const bool mine = an >= 0 && m.rpart[r] == p;
                float *z = m.Zs + r * s.ldz;
                auto put = [&](int o, float v) {
                    z[o] = v;
                    m.dZT[o * kBLdr + r] = __float2bfloat16_rn(v);
                };
                float gls[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f}, gx[3] = {0.f, 0.f, 0.f};
                const float *ls = a.f.log_scaling + 6 * (an >= 0 ? an : 0);
                float el[6];
#pragma unroll
                for (int j = 0; j < 6; ++j) el[j] = mine ? expf(__ldg(ls + j)) : 0.f;
                for (int i = par; i < k; i += 2) {
                    const float op = mine ? tanhf(z[s.off[0] + i]) : 0.f;
                    if (!(op > 0.f)) {   // culled by decoding (or not this partition): no gradient
                        put(s.off[0] + i, 0.f);
#pragma unroll
                        for (int ch = 0; ch < 3; ++ch) put(s.off[1] + 3 * i + ch, 0.f);
#pragma unroll
                        for (int j = 0; j < 7; ++j) put(s.off[2] + 7 * i + j, 0.f);
                        continue;
                    }
                    const size_t c = ((size_t)tile * kBRows + r) * k + i;
                    put(s.off[0] + i, __ldg(a.dopacity + c) * (1.f - op * op));
#pragma unroll
                    for (int ch = 0; ch < 3; ++ch) {
                        const int o = s.off[1] + 3 * i + ch;
                        const float sg = sigmoidf_(z[o]);
                        put(o, __ldg(a.dcolour + 3 * c + ch) * sg * (1.f - sg));
                    }
                    float zq[7];
#pragma unroll
                    for (int j = 0; j < 7; ++j) zq[j] = z[s.off[2] + 7 * i + j];
#pragma unroll
                    for (int j = 0; j < 3; ++j) {
                        const float sg = sigmoidf_(zq[j]);
                        const float ds = __ldg(a.dscale + 3 * c + j);
                        put(s.off[2] + 7 * i + j, ds * el[3 + j] * sg * (1.f - sg));
                        gls[3 + j] += ds * el[3 + j] * sg;
                    }
                    const float qn = sqrtf(zq[3] * zq[3] + zq[4] * zq[4] + zq[5] * zq[5] + zq[6] * zq[6]);
                    const float inv = 1.f / qn;
                    float dq[4], qd = 0.f;
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        dq[j] = __ldg(a.dquat + 4 * c + j);
                        qd += zq[3 + j] * inv * dq[j];
                    }
#pragma unroll
                    for (int j = 0; j < 4; ++j) put(s.off[2] + 7 * i + 3 + j, (dq[j] - zq[3 + j] * inv * qd) * inv);
                    const float *off = a.f.offsets + ((size_t)an * k + i) * 3;
#pragma unroll
                    for (int j = 0; j < 3; ++j) {
                        const float gm = __ldg(a.dmu + 3 * c + j);
                        gx[j] += gm;
                        atomicAdd(a.doff + ((size_t)an * k + i) * 3 + j, gm * el[j]);
                        gls[j] += gm * __ldg(off + j) * el[j];
                    }
                }
                // padding columns of each head block
#pragma unroll
                for (int h = 0; h < 3; ++h)
                    for (int o = s.off[h] + s.dout[h] + par; o < s.off[h] + s.dpad[h]; o += 2) put(o, 0.f);
                // combine the two threads of the row, one atomic per anchor quantity
#pragma unroll
                for (int j = 0; j < 6; ++j) gls[j] += __shfl_xor_sync(0xffffffffu, gls[j], 1);
#pragma unroll
                for (int j = 0; j < 3; ++j) gx[j] += __shfl_xor_sync(0xffffffffu, gx[j], 1);
                if (mine && par == 0) {
#pragma unroll
                    for (int j = 0; j < 6; ++j) atomicAdd(a.dls + 6 * an + j, gls[j]);
                    // position gradient through mu = x_a + ..., combined with the Eq. 2 part below
#pragma unroll
                        m.gxs[3 * r] = gx[0]; m.gxs[3 * r + 1] = gx[1]; m.gxs[3 * r + 2] = gx[2];
                }
            }
            __syncthreads();
            // ---- 3./4. dHID = dZ_h W2_h, dPRE = dHID * mask, dU = dPRE W1 (split-BF16)
            {
                uint32_t ph[NH][HT][4], pl[NH][HT][4];   // dPRE as hi/lo A fragments
#pragma unroll
                for (int h = 0; h < NH; ++h) {
#pragma unroll
                    for (int t = 0; t < HT; ++t) {
                        float c[2][4];
#pragma unroll
                        for (int hf = 0; hf < 2; ++hf) {
                            c[hf][0] = c[hf][1] = c[hf][2] = c[hf][3] = 0.f;
                            const int n0 = h * s.H + 16 * t + 8 * hf;
                            const float *w2t = h == 0 ? m.W2T[0] : (h == 1 ? m.W2T[1] : m.W2T[2]);
                            const int ldt = h == 0 ? s.ldw2t[0] : (h == 1 ? s.ldw2t[1] : s.ldw2t[2]);
                            for (int k0 = s.off[h]; k0 < s.off[h] + s.dpad[h]; k0 += 16) {
                                uint32_t ah[4], al[4], bh[2], bl[2];
                                load_a_split(ah, al, m.Zs, s.ldz, m0w, k0);
                                load_b_split(bh, bl, w2t, ldt, k0 - s.off[h], n0 - h * s.H);
                                mma_split(c[hf], ah, al, bh, bl);
                            }
#pragma unroll
                            for (int e = 0; e < 4; ++e)
                                if (!(mask[h] >> ((2 * t + hf) * 4 + e) & 1u)) c[hf][e] = 0.f;
                            const int j = n0 + 2 * q;   // dPRE^T for the dW1 GEMM
                            m.dPT[j * kBLdr + m0w + g] = __float2bfloat16_rn(c[hf][0]);
                            m.dPT[(j + 1) * kBLdr + m0w + g] = __float2bfloat16_rn(c[hf][1]);
                            m.dPT[j * kBLdr + m0w + g + 8] = __float2bfloat16_rn(c[hf][2]);
                            m.dPT[(j + 1) * kBLdr + m0w + g + 8] = __float2bfloat16_rn(c[hf][3]);
                        }
                        split_bf16(c[0][0], c[0][1], ph[h][t][0], pl[h][t][0]);
                        split_bf16(c[0][2], c[0][3], ph[h][t][1], pl[h][t][1]);
                        split_bf16(c[1][0], c[1][1], ph[h][t][2], pl[h][t][2]);
                        split_bf16(c[1][2], c[1][3], ph[h][t][3], pl[h][t][3]);
                    }
                }
                for (int n0 = 0; n0 < s.KP; n0 += 8) {
                    float c[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
                    for (int h = 0; h < NH; ++h)
#pragma unroll
                        for (int t = 0; t < HT; ++t) {
                            uint32_t bh[2], bl[2];
                            load_b_split(bh, bl, m.W1T, s.ldw1t, h * s.H + 16 * t, n0);
                            mma_split(c, ph[h][t], pl[h][t], bh, bl);
                        }
                    m.dUs[(m0w + g) * s.lddu + n0 + 2 * q] = c[0];
                    m.dUs[(m0w + g) * s.lddu + n0 + 2 * q + 1] = c[1];
                    m.dUs[(m0w + g + 8) * s.lddu + n0 + 2 * q] = c[2];
                    m.dUs[(m0w + g + 8) * s.lddu + n0 + 2 * q + 1] = c[3];
                }
            }
            __syncthreads();
            // ---- 5. weight gradients over the tile's rows (K = 64)
            {
                const int n1 = (s.H3 / 16) * (s.KP / 8);
#pragma unroll
                for (int t = 0; t < NT1; ++t) {
                    const int idx = warp + 4 * t;
                    if (idx < n1) {
                        int mm, nn;
                        w1_tile(s, idx, &mm, &nn);
#pragma unroll
                        for (int kk = 0; kk < kBRows; kk += 16) {
                            uint32_t af[4], b0, b1;
                            load_a(af, m.dPT, kBLdr, mm, kk);
                            load_b(b0, b1, m.UT, kBLdr, kk, nn);
                            mma_bf16_16816(acc.w1[t], af, b0, b1);
                        }
                    }
                }
#pragma unroll
                for (int t = 0; t < NT2; ++t) {
                    int h, mm, nn;
                    if (w2_tile(s, warp + 4 * t, &h, &mm, &nn)) {
                        const __nv_bfloat16 *ht = m.HT + (size_t)(h * (s.H + 8)) * kBLdr;
#pragma unroll
                        for (int kk = 0; kk < kBRows; kk += 16) {
                            uint32_t af[4], b0, b1;
                            load_a(af, m.dZT, kBLdr, mm, kk);
                            load_b(b0, b1, ht, kBLdr, kk, nn);
                            mma_bf16_16816(acc.w2[t], af, b0, b1);
                        }
                    }
                }
            }
            // ---- per-row: features and the view inputs of Eq. 2
            if (tid < kBRows && m.rpart[tid] == p && m.ran[tid] >= 0) {
                const int an = m.ran[tid];
                const float *du = m.dUs + tid * s.lddu;
                for (int i = 0; i < s.F; ++i) atomicAdd(a.dfeat + (size_t)an * s.F + i, du[i]);
                const float inv = 1.f / m.rd[4 * tid + 3];
                const float dir[3] = {m.rd[4 * tid] * inv, m.rd[4 * tid + 1] * inv, m.rd[4 * tid + 2] * inv};
                const float g0 = du[s.F], g1 = du[s.F + 1], g2 = du[s.F + 2], gd = du[s.F + 3];
                const float dd = g0 * dir[0] + g1 * dir[1] + g2 * dir[2];
                atomicAdd(a.dxyz + 3 * an, (g0 - dir[0] * dd) * inv + gd * dir[0] + m.gxs[3 * tid]);
                atomicAdd(a.dxyz + 3 * an + 1, (g1 - dir[1] * dd) * inv + gd * dir[1] + m.gxs[3 * tid + 1]);
                atomicAdd(a.dxyz + 3 * an + 2, (g2 - dir[2] * dd) * inv + gd * dir[2] + m.gxs[3 * tid + 2]);
            }
            __syncthreads();
            if (tid < kBRows && m.rpart[tid] == p) m.rdone[tid] = 1;
            __syncthreads();
        }
    }
    __syncthreads();
    if (s_accp >= 0) flush_acc<KS, HT, NT1, NT2, NH>(s, acc, a.dmlp + (size_t)s_accp * P);
}

template <int KS, int HT, int NT2>
static int launch_bwd_t(const DecodeBwdArgsB &a, const BwdShape &s, cudaStream_t st)
{
    constexpr int NH = 3;
    constexpr int NT1 = ((3 * 16 * HT / 16) * (KS * 16 / 8) + 3) / 4;   // dW1 tiles per warp
    static size_t configured = 0;
    if (s.smem > 48 * 1024 && s.smem > configured) {
        if (cudaFuncSetAttribute(decode_bwd_bf16_kernel<KS, HT, NT1, NT2, NH>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s.smem) != cudaSuccess)
            return GS_ERR_UNSUPPORTED;
        configured = s.smem;
    }
    const long long tiles = (a.f.cap_rows + kBRows - 1) / kBRows;
    const int grid = (int)std::max<long long>(1, std::min<long long>(tiles, (long long)sm_count()));
    decode_bwd_bf16_kernel<KS, HT, NT1, NT2, NH><<<grid, kBThreads, s.smem, st>>>(a, s);
    count_launches(1);
    return cudaPeekAtLastError() == cudaSuccess ? GS_OK : GS_ERR_CUDA;
}

int launch_decode_bwd_bf16(const DecodeBwdArgsB &a, cudaStream_t st)
{
    const BwdShape s = bwd_shape(a.f.F, a.f.k, a.f.H);
    const int KS = s.KP / 16, HT = a.f.H / 16;
    if (a.f.H % 16 != 0 || HT < 1 || HT > 2 || KS < 1 || KS > 4 || s.smem > 220 * 1024) return GS_ERR_UNSUPPORTED;
    // dW2 output tiles per warp: 4, 10 or 14 register tiles
    const int n2 = ((s.dpad[0] + s.dpad[1] + s.dpad[2]) / 16) * ((s.H + 8) / 8);
    const int per = (n2 + 3) / 4;
    const int NT2 = per <= 4 ? 4 : (per <= 10 ? 10 : (per <= 14 ? 14 : 0));
    if (NT2 == 0) return GS_ERR_UNSUPPORTED;
#define GS_BWD_CASE(ks, ht) \
    if (KS == ks && HT == ht) {                                                   \
        if (NT2 == 4) return launch_bwd_t<ks, ht, 4>(a, s, st);                   \
        if (NT2 == 10) return launch_bwd_t<ks, ht, 10>(a, s, st);                 \
        return launch_bwd_t<ks, ht, 14>(a, s, st);                                \
    }
    GS_BWD_CASE(1, 1) GS_BWD_CASE(2, 1) GS_BWD_CASE(3, 1) GS_BWD_CASE(4, 1)
    GS_BWD_CASE(1, 2) GS_BWD_CASE(2, 2) GS_BWD_CASE(3, 2) GS_BWD_CASE(4, 2)
#undef GS_BWD_CASE
    return GS_ERR_UNSUPPORTED;
}

}  // namespace gs
