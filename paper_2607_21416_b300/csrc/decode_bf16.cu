// decode_bf16.cu -- BF16 tensor-core anchor decoding (FP32 accumulation).
//
// Same arithmetic as the FP32 decoder (Sec. III-A, Eq. 2; partition MLP sets
// of Eq. 6) with the two MLP layers run as warp MMAs (m16n8k16, BF16 inputs,
// FP32 accumulation) and an FP32 epilogue:
//   PRE = U W1^T + b1 (all three heads stacked, K = F + 4 padded to 16s),
//   HID = relu(PRE) rounded to BF16 -- kept in registers: the C fragments of
//         two 8-wide n-tiles are the A fragment of one k-step of layer 2,
//   Z_h = HID_h W2_h^T + b2_h, staged in shared memory for the epilogue.
// A CTA of 4 warps decodes tiles of 64 rows (16 per warp), persistent over
// the row range.  The partition's weights are converted to BF16 into shared
// memory once and re-staged only when the partition changes; a tile whose rows
// span several partitions is run once per partition with the other rows'
// results discarded.
#include "gs_internal.cuh"
#include "mma_bf16.cuh"

namespace gs {

constexpr int kDRows = 64;
constexpr int kDThreads = 128;

struct DecShape {
    int F, Din, KP, H, k;
    int dout[3], dpad[3], off[3], NZ;   // layer-2 outputs per head, padded to 8, stacked offsets
    int hoff[3];                        // offsets of the heads in the packed FP32 MLP set
    int ldw1, ldw2, ldu, ldz;
    size_t smem;
};

static DecShape dec_shape(int F, int k, int H)
{
    DecShape s;
    s.F = F; s.Din = F + 4; s.KP = (s.Din + 15) / 16 * 16; s.H = H; s.k = k;
    const int d[3] = {k, 3 * k, 7 * k};
    int o = 0, h = 0;
    for (int i = 0; i < 3; ++i) {
        s.dout[i] = d[i];
        s.dpad[i] = (d[i] + 7) / 8 * 8;
        s.off[i] = o;
        o += s.dpad[i];
        s.hoff[i] = h;
        h += H * s.Din + H + d[i] * H + d[i];
    }
    s.NZ = o;
    s.ldw1 = s.KP + 8;
    s.ldw2 = H + 8;
    s.ldu = s.KP + 8;
    s.ldz = s.NZ + 4;
    size_t b = 0;
    b += sizeof(__nv_bfloat16) * (size_t)3 * H * s.ldw1;   // W1s
    b += sizeof(__nv_bfloat16) * (size_t)s.NZ * s.ldw2;    // W2s
    b += sizeof(__nv_bfloat16) * (size_t)kDRows * s.ldu;   // Us
    b = (b + 15) / 16 * 16;
    b += sizeof(float) * (size_t)(3 * H + s.NZ);           // b1s, b2s
    b += sizeof(float) * (size_t)kDRows * s.ldz;           // Zs
    b += sizeof(float) * (size_t)kDRows * 4;               // per-row (d, delta)
    b += sizeof(int) * (size_t)kDRows * 3;                 // anchor, partition, done
    s.smem = b;
    return s;
}

struct DecSmem {
    __nv_bfloat16 *W1s, *W2s, *Us;
    float *b1s, *b2s, *Zs, *rd;
    int *ran, *rpart, *rdone;
};

__device__ __forceinline__ DecSmem dec_smem(char *base, const DecShape &s)
{
    DecSmem m;
    size_t o = 0;
    m.W1s = reinterpret_cast<__nv_bfloat16 *>(base + o); o += sizeof(__nv_bfloat16) * (size_t)3 * s.H * s.ldw1;
    m.W2s = reinterpret_cast<__nv_bfloat16 *>(base + o); o += sizeof(__nv_bfloat16) * (size_t)s.NZ * s.ldw2;
    m.Us = reinterpret_cast<__nv_bfloat16 *>(base + o); o += sizeof(__nv_bfloat16) * (size_t)kDRows * s.ldu;
    o = (o + 15) / 16 * 16;
    m.b1s = reinterpret_cast<float *>(base + o); o += sizeof(float) * 3 * s.H;
    m.b2s = reinterpret_cast<float *>(base + o); o += sizeof(float) * s.NZ;
    m.Zs = reinterpret_cast<float *>(base + o); o += sizeof(float) * (size_t)kDRows * s.ldz;
    m.rd = reinterpret_cast<float *>(base + o); o += sizeof(float) * kDRows * 4;
    m.ran = reinterpret_cast<int *>(base + o); o += sizeof(int) * kDRows;
    m.rpart = reinterpret_cast<int *>(base + o); o += sizeof(int) * kDRows;
    m.rdone = reinterpret_cast<int *>(base + o);
    return m;
}

// Converts partition p's FP32 weights into the BF16 / padded shared layout.
__device__ void stage_weights(const DecShape &s, const DecSmem &m, const float *__restrict__ mlp_p)
{
    const int tid = threadIdx.x;
    for (int idx = tid; idx < 3 * s.H * s.KP; idx += kDThreads) {
        const int j = idx / s.KP, i = idx % s.KP, h = j / s.H, jj = j % s.H;
        const float w = i < s.Din ? __ldg(mlp_p + s.hoff[h] + jj * s.Din + i) : 0.f;
        m.W1s[j * s.ldw1 + i] = __float2bfloat16_rn(w);
    }
    for (int j = tid; j < 3 * s.H; j += kDThreads) {
        const int h = j / s.H, jj = j % s.H;
        m.b1s[j] = __ldg(mlp_p + s.hoff[h] + s.H * s.Din + jj);
    }
    for (int idx = tid; idx < s.NZ * s.H; idx += kDThreads) {
        const int o = idx / s.H, j = idx % s.H;
        const int h = o < s.off[1] ? 0 : (o < s.off[2] ? 1 : 2);
        const int lo = o - s.off[h];
        const float w = lo < s.dout[h] ? __ldg(mlp_p + s.hoff[h] + s.H * s.Din + s.H + lo * s.H + j) : 0.f;
        m.W2s[o * s.ldw2 + j] = __float2bfloat16_rn(w);
    }
    for (int o = tid; o < s.NZ; o += kDThreads) {
        const int h = o < s.off[1] ? 0 : (o < s.off[2] ? 1 : 2);
        const int lo = o - s.off[h];
        m.b2s[o] = lo < s.dout[h] ? __ldg(mlp_p + s.hoff[h] + s.H * s.Din + s.H + s.dout[h] * s.H + lo) : 0.f;
    }
}

// Loads the tile's rows (anchor, partition, view inputs) and builds U in BF16.
__device__ void load_rows(const DecodeArgs &a, const DecShape &s, const DecSmem &m, int tile, int rows)
{
    const int tid = threadIdx.x;
    if (tid < kDRows) {
        const int r = tile * kDRows + tid;
        int an = -1, pm = -1;
        float d0 = 0.f, d1 = 0.f, d2 = 0.f, dl = 1.f;
        if (r < rows) {
            an = __ldg(a.row_anchor + r);
            if (!idx_ok(a.st, an, a.N, 13)) an = -1;
        }
        if (an >= 0) {
            pm = __ldg(a.part + an);
            if (!idx_ok(a.st, pm, a.M, 14)) { pm = -1; an = -1; }
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
    for (int idx = tid; idx < kDRows * s.KP; idx += kDThreads) {
        const int r = idx / s.KP, i = idx % s.KP;
        const int an = m.ran[r];
        float u = 0.f;
        if (an >= 0) {
            if (i < s.F) u = __ldg(a.feat + (size_t)an * s.F + i);
            else if (i < s.F + 3) u = m.rd[4 * r + (i - s.F)] / m.rd[4 * r + 3];
            else if (i == s.F + 3) u = m.rd[4 * r + 3];
        }
        m.Us[r * s.ldu + i] = __float2bfloat16_rn(u);
    }
}

// Layers 1 and 2 of the tile's 16 rows of this warp for the staged partition;
// Z rows of partition p are written to Zs.
template <int KS, int HT>
__device__ void mlp_tile(const DecShape &s, const DecSmem &m, int p)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, q = lane & 3;
    const int m0 = warp * 16;
    uint32_t ua[KS][4];
#pragma unroll
    for (int ks = 0; ks < KS; ++ks) load_a(ua[ks], m.Us, s.ldu, m0, 16 * ks);
    const bool keep_lo = m.rpart[m0 + g] == p, keep_hi = m.rpart[m0 + g + 8] == p;
#pragma unroll
    for (int h = 0; h < 3; ++h) {
        uint32_t ha[HT][4];
        const int hb = h * s.H;
#pragma unroll
        for (int t = 0; t < HT; ++t) {
            float c0[4], c1[4];
            const int n0 = hb + 16 * t;
            c0[0] = c0[2] = m.b1s[n0 + 2 * q];
            c0[1] = c0[3] = m.b1s[n0 + 2 * q + 1];
            c1[0] = c1[2] = m.b1s[n0 + 8 + 2 * q];
            c1[1] = c1[3] = m.b1s[n0 + 8 + 2 * q + 1];
#pragma unroll
            for (int ks = 0; ks < KS; ++ks) {
                uint32_t b0, b1;
                load_b(b0, b1, m.W1s, s.ldw1, 16 * ks, n0);
                mma_bf16_16816(c0, ua[ks], b0, b1);
                load_b(b0, b1, m.W1s, s.ldw1, 16 * ks, n0 + 8);
                mma_bf16_16816(c1, ua[ks], b0, b1);
            }
            ha[t][0] = pack_bf16(fmaxf(c0[0], 0.f), fmaxf(c0[1], 0.f));
            ha[t][1] = pack_bf16(fmaxf(c0[2], 0.f), fmaxf(c0[3], 0.f));
            ha[t][2] = pack_bf16(fmaxf(c1[0], 0.f), fmaxf(c1[1], 0.f));
            ha[t][3] = pack_bf16(fmaxf(c1[2], 0.f), fmaxf(c1[3], 0.f));
        }
        for (int n0 = s.off[h]; n0 < s.off[h] + s.dpad[h]; n0 += 8) {
            float z[4];
            z[0] = z[2] = m.b2s[n0 + 2 * q];
            z[1] = z[3] = m.b2s[n0 + 2 * q + 1];
#pragma unroll
            for (int t = 0; t < HT; ++t) {
                uint32_t b0, b1;
                load_b(b0, b1, m.W2s, s.ldw2, 16 * t, n0);
                mma_bf16_16816(z, ha[t], b0, b1);
            }
            if (keep_lo) {
                m.Zs[(m0 + g) * s.ldz + n0 + 2 * q] = z[0];
                m.Zs[(m0 + g) * s.ldz + n0 + 2 * q + 1] = z[1];
            }
            if (keep_hi) {
                m.Zs[(m0 + g + 8) * s.ldz + n0 + 2 * q] = z[2];
                m.Zs[(m0 + g + 8) * s.ldz + n0 + 2 * q + 1] = z[3];
            }
        }
    }
}

template <int KS, int HT>
__global__ void __launch_bounds__(kDThreads) decode_bf16_kernel(DecodeArgs a, DecShape s)
{
    if (has_error(a.st)) return;
    extern __shared__ __align__(16) char smem_raw[];
    const DecSmem m = dec_smem(smem_raw, s);
    __shared__ int s_p, s_staged;
    const int tid = threadIdx.x;
    const int rows = __ldg(a.view_start + a.V);
    const int ntiles = (rows + kDRows - 1) / kDRows;
    if (tid == 0) s_staged = -1;
    const long long P = a.mlp_floats;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        __syncthreads();
        load_rows(a, s, m, tile, rows);
        __syncthreads();
        for (;;) {
            if (tid == 0) {
                int p = -1;
                for (int r = 0; r < kDRows; ++r)
                    if (!m.rdone[r]) { p = m.rpart[r]; break; }
                s_p = p;
            }
            __syncthreads();
            const int p = s_p;
            if (p < 0) break;
            if (p != s_staged) {
                stage_weights(s, m, a.mlp + (size_t)p * P);
                __syncthreads();
                if (tid == 0) s_staged = p;
            }
            mlp_tile<KS, HT>(s, m, p);
            __syncthreads();
            if (tid < kDRows && m.rpart[tid] == p) m.rdone[tid] = 1;
            __syncthreads();
        }
        // epilogue: one (row, candidate) per thread-iteration
        const int k = s.k;
        for (int idx = tid; idx < kDRows * k; idx += kDThreads) {
            const int r = idx / k, i = idx % k;
            const int an = m.ran[r];
            if (an < 0) continue;
            const float *z = m.Zs + r * s.ldz;
            const size_t c = ((size_t)tile * kDRows + r) * k + i;
            a.opacity[c] = tanhf(z[s.off[0] + i]);
#pragma unroll
            for (int ch = 0; ch < 3; ++ch) a.colour[3 * c + ch] = sigmoidf_(z[s.off[1] + 3 * i + ch]);
            const float *zc = z + s.off[2] + 7 * i;
            const float *ls = a.log_scaling + 6 * an;
#pragma unroll
            for (int j = 0; j < 3; ++j) a.scale[3 * c + j] = expf(__ldg(ls + 3 + j)) * sigmoidf_(zc[j]);
            const float qn = sqrtf(zc[3] * zc[3] + zc[4] * zc[4] + zc[5] * zc[5] + zc[6] * zc[6]);
            const float inv = 1.f / qn;
#pragma unroll
            for (int j = 0; j < 4; ++j) a.quat[4 * c + j] = zc[3 + j] * inv;
            const float *off = a.offsets + ((size_t)an * k + i) * 3;
#pragma unroll
            for (int j = 0; j < 3; ++j) a.mu[3 * c + j] = __ldg(a.xyz + 3 * an + j) + __ldg(off + j) * expf(__ldg(ls + j));
        }
    }
}

template <int KS, int HT>
static int launch_t(const DecodeArgs &a, const DecShape &s, cudaStream_t st)
{
    static size_t configured = 0;
    if (s.smem > 48 * 1024 && s.smem > configured) {
        if (cudaFuncSetAttribute(decode_bf16_kernel<KS, HT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)s.smem) != cudaSuccess)
            return GS_ERR_UNSUPPORTED;
        configured = s.smem;
    }
    const long long tiles = (a.cap_rows + kDRows - 1) / kDRows;
    const int grid = (int)std::max<long long>(1, std::min<long long>(tiles, (long long)sm_count() * 4));
    decode_bf16_kernel<KS, HT><<<grid, kDThreads, s.smem, st>>>(a, s);
    count_launches(1);
    return cudaPeekAtLastError() == cudaSuccess ? GS_OK : GS_ERR_CUDA;
}

int launch_decode_bf16(const DecodeArgs &a, cudaStream_t st)
{
    const DecShape s = dec_shape(a.F, a.k, a.H);
    const int KS = s.KP / 16, HT = a.H / 16;
    if (a.H % 16 != 0 || HT < 1 || HT > 2 || KS < 1 || KS > 4 || s.smem > 200 * 1024) return GS_ERR_UNSUPPORTED;
#define GS_DEC_CASE(ks, ht) \
    if (KS == ks && HT == ht) return launch_t<ks, ht>(a, s, st);
    GS_DEC_CASE(1, 1) GS_DEC_CASE(2, 1) GS_DEC_CASE(3, 1) GS_DEC_CASE(4, 1)
    GS_DEC_CASE(1, 2) GS_DEC_CASE(2, 2) GS_DEC_CASE(3, 2) GS_DEC_CASE(4, 2)
#undef GS_DEC_CASE
    return GS_ERR_UNSUPPORTED;
}

}  // namespace gs
