// mma_bf16.cuh -- warp-level BF16 tensor-core helpers (mma.sync m16n8k16,
// FP32 accumulation) and fragment loaders for the anchor-decoder GEMMs.
//
// Fragment layouts (per lane: g = lane / 4, q = lane % 4):
//   A 16x16 (row-major): r0 = A[g][2q..2q+1], r1 = A[g+8][2q..], r2 = A[g][8+2q..],
//                        r3 = A[g+8][8+2q..]   (two bf16 per register, low half = lower column)
//   B 16x8  (k x n):     r0 = B[2q..2q+1][g],  r1 = B[8+2q..][g]
//   C 16x8  (fp32):      c0,c1 = C[g][2q..2q+1], c2,c3 = C[g+8][2q..2q+1]
// A C fragment pair (n-tiles 2t, 2t+1) therefore is, after rounding, the A
// fragment of k-step t of a following GEMM: layers chain in registers.
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>

namespace gs {

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi)
{
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t *>(&v);
}

__device__ __forceinline__ void mma_bf16_16816(float c[4], const uint32_t a[4], uint32_t b0, uint32_t b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
        "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// A fragment of the 16x16 block at (m0, k0) of a row-major bf16 matrix with a
// row stride of `ld` elements (ld even, m0/k0 multiples of 16 resp. 8).
__device__ __forceinline__ void load_a(uint32_t a[4], const __nv_bfloat16 *X, int ld, int m0, int k0)
{
    const int lane = threadIdx.x & 31, g = lane >> 2, q = lane & 3;
    const __nv_bfloat16 *p = X + (size_t)(m0 + g) * ld + k0 + 2 * q;
    a[0] = *reinterpret_cast<const uint32_t *>(p);
    a[1] = *reinterpret_cast<const uint32_t *>(p + 8 * ld);
    a[2] = *reinterpret_cast<const uint32_t *>(p + 8);
    a[3] = *reinterpret_cast<const uint32_t *>(p + 8 * ld + 8);
}

// B fragment of the 16x8 block at (k0, n0) of B[k][n] = Wt[n][k] with Wt a
// row-major bf16 matrix of row stride `ld` (a linear layer's weight [out][in]).
__device__ __forceinline__ void load_b(uint32_t &b0, uint32_t &b1, const __nv_bfloat16 *Wt, int ld, int k0, int n0)
{
    const int lane = threadIdx.x & 31, g = lane >> 2, q = lane & 3;
    const __nv_bfloat16 *p = Wt + (size_t)(n0 + g) * ld + k0 + 2 * q;
    b0 = *reinterpret_cast<const uint32_t *>(p);
    b1 = *reinterpret_cast<const uint32_t *>(p + 8);
}

// x = hi + lo with hi, lo in BF16 (about 16 significant bits together).
__device__ __forceinline__ void split_bf16(float x0, float x1, uint32_t &hi, uint32_t &lo)
{
    __nv_bfloat162 h = __floats2bfloat162_rn(x0, x1);
    const float2 hf = __bfloat1622float2(h);
    __nv_bfloat162 l = __floats2bfloat162_rn(x0 - hf.x, x1 - hf.y);
    hi = *reinterpret_cast<uint32_t *>(&h);
    lo = *reinterpret_cast<uint32_t *>(&l);
}

// Split (hi/lo) A fragment of an FP32 row-major matrix (ld even).
__device__ __forceinline__ void load_a_split(uint32_t ah[4], uint32_t al[4], const float *X, int ld, int m0, int k0)
{
    const int lane = threadIdx.x & 31, g = lane >> 2, q = lane & 3;
    const float *p = X + (size_t)(m0 + g) * ld + k0 + 2 * q;
    const float2 v0 = *reinterpret_cast<const float2 *>(p);
    const float2 v1 = *reinterpret_cast<const float2 *>(p + 8 * ld);
    const float2 v2 = *reinterpret_cast<const float2 *>(p + 8);
    const float2 v3 = *reinterpret_cast<const float2 *>(p + 8 * ld + 8);
    split_bf16(v0.x, v0.y, ah[0], al[0]);
    split_bf16(v1.x, v1.y, ah[1], al[1]);
    split_bf16(v2.x, v2.y, ah[2], al[2]);
    split_bf16(v3.x, v3.y, ah[3], al[3]);
}

// Split (hi/lo) B fragment of B[k][n] = Wt[n][k], Wt FP32 row-major (ld even).
__device__ __forceinline__ void load_b_split(uint32_t bh[2], uint32_t bl[2], const float *Wt, int ld, int k0, int n0)
{
    const int lane = threadIdx.x & 31, g = lane >> 2, q = lane & 3;
    const float *p = Wt + (size_t)(n0 + g) * ld + k0 + 2 * q;
    const float2 v0 = *reinterpret_cast<const float2 *>(p);
    const float2 v1 = *reinterpret_cast<const float2 *>(p + 8);
    split_bf16(v0.x, v0.y, bh[0], bl[0]);
    split_bf16(v1.x, v1.y, bh[1], bl[1]);
}

// c += (ah + al)(bh + bl) without the al*bl term: three BF16 MMAs, FP32 accumulation.
__device__ __forceinline__ void mma_split(float c[4], const uint32_t ah[4], const uint32_t al[4], const uint32_t bh[2],
                                          const uint32_t bl[2])
{
    mma_bf16_16816(c, al, bh[0], bh[1]);
    mma_bf16_16816(c, ah, bl[0], bl[1]);
    mma_bf16_16816(c, ah, bh[0], bh[1]);
}

}  // namespace gs
