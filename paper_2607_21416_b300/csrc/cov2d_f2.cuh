// cov2d_f2.cuh -- the EWA 2D covariance of a near-degenerate splat in
// compensated single precision, for the FP64 determinant and conic inverse
// of the projection and of its reverse pass.
//
// The inverse of a 2x2 covariance with condition number c amplifies the
// relative rounding of its entries c times, so entries formed in plain FP32
// leave a conic error of about c 2^-24 however the inverse is taken.  Here the
// entries are formed as float-float values: an unevaluated sum hi + lo of two
// floats (Dekker's double-length arithmetic): products get their exact
// rounding error from a fused multiply-add, sums from Knuth's two-sum, which
// carries about 44 significant bits through the chain.  Only the determinant
// and the inverse are then taken in FP64, from hi + lo.
#pragma once

#include "gs_internal.cuh"

namespace gs {

struct f2 {
    float hi, lo;
};

__device__ __forceinline__ f2 f2_of(float x) { return {x, 0.f}; }

// s + e = a + b exactly (Knuth).
__device__ __forceinline__ f2 f2_two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}
// s + e = a + b exactly when |a| >= |b| (Dekker).
__device__ __forceinline__ f2 f2_fast_two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ f2 f2_add(f2 a, f2 b)
{
    f2 s = f2_two_sum(a.hi, b.hi);
    const f2 t = f2_two_sum(a.lo, b.lo);
    s = f2_fast_two_sum(s.hi, __fadd_rn(s.lo, t.hi));
    return f2_fast_two_sum(s.hi, __fadd_rn(s.lo, t.lo));
}
__device__ __forceinline__ f2 f2_neg(f2 a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ f2 f2_mul(f2 a, f2 b)
{
    const float p = __fmul_rn(a.hi, b.hi);
    float e = fmaf(a.hi, b.hi, -p);   // exact error of the product
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    return f2_fast_two_sum(p, e);
}
// a / b: one correction of the quotient by its exact remainder.
__device__ __forceinline__ f2 f2_div(f2 a, f2 b)
{
    const float q1 = __fdiv_rn(a.hi, b.hi);
    const f2 r = f2_add(a, f2_neg(f2_mul(b, f2_of(q1))));
    return f2_fast_two_sum(q1, __fdiv_rn(r.hi, b.hi));
}
__device__ __forceinline__ double f2_to_double(f2 a) { return (double)a.hi + (double)a.lo; }

// 2D covariance (a, b, c) = J W R_q S^2 R_q^T W^T J^T + 0.3 I of a splat with
// FP32 mean m, scales s, quaternion (w, x, y, z) under camera cm (the
// Jacobian at the clamped tangent, as the FP32 path forms it), returned as
// FP64 values of the float-float results.
static __device__ __noinline__ void cov2d_compensated(const Cam &cm, float m0, float m1, float m2, float w, float x,
                                                      float y, float z, float s0, float s1, float s2, float limx,
                                                      float limy, double *ca, double *cb, double *cc)
{
    f2 p[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        f2 acc = f2_of(cm.t[i]);
        acc = f2_add(acc, f2_mul(f2_of(cm.R[3 * i]), f2_of(m0)));
        acc = f2_add(acc, f2_mul(f2_of(cm.R[3 * i + 1]), f2_of(m1)));
        p[i] = f2_add(acc, f2_mul(f2_of(cm.R[3 * i + 2]), f2_of(m2)));
    }
    // rotation of the unit quaternion, entries as 1 - 2(..) and 2(.. +- ..)
    const f2 W = f2_of(w), X = f2_of(x), Y = f2_of(y), Z = f2_of(z), one = f2_of(1.f);
    const f2 xx = f2_mul(X, X), yy = f2_mul(Y, Y), zz = f2_mul(Z, Z);
    const f2 xy = f2_mul(X, Y), xz = f2_mul(X, Z), yz = f2_mul(Y, Z);
    const f2 wx = f2_mul(W, X), wy = f2_mul(W, Y), wz = f2_mul(W, Z);
    auto twice = [](f2 a) { return f2{2.f * a.hi, 2.f * a.lo}; };
    f2 Rq[9];
    Rq[0] = f2_add(one, f2_neg(twice(f2_add(yy, zz))));
    Rq[1] = twice(f2_add(xy, f2_neg(wz)));
    Rq[2] = twice(f2_add(xz, wy));
    Rq[3] = twice(f2_add(xy, wz));
    Rq[4] = f2_add(one, f2_neg(twice(f2_add(xx, zz))));
    Rq[5] = twice(f2_add(yz, f2_neg(wx)));
    Rq[6] = twice(f2_add(xz, f2_neg(wy)));
    Rq[7] = twice(f2_add(yz, wx));
    Rq[8] = f2_add(one, f2_neg(twice(f2_add(xx, yy))));
    const f2 q[3] = {f2_mul(f2_of(s0), f2_of(s0)), f2_mul(f2_of(s1), f2_of(s1)), f2_mul(f2_of(s2), f2_of(s2))};
    f2 S[6];   // Sigma3: 00 01 02 11 12 22
    {
        const int ij[6][2] = {{0, 0}, {0, 1}, {0, 2}, {1, 1}, {1, 2}, {2, 2}};
#pragma unroll
        for (int e = 0; e < 6; ++e) {
            const int i = ij[e][0], j = ij[e][1];
            f2 acc = f2_mul(f2_mul(Rq[3 * i], Rq[3 * j]), q[0]);
            acc = f2_add(acc, f2_mul(f2_mul(Rq[3 * i + 1], Rq[3 * j + 1]), q[1]));
            S[e] = f2_add(acc, f2_mul(f2_mul(Rq[3 * i + 2], Rq[3 * j + 2]), q[2]));
        }
    }
    // Jacobian at the clamped tangent
    f2 tx = f2_div(p[0], p[2]), ty = f2_div(p[1], p[2]);
    if (tx.hi < -limx) tx = f2_of(-limx);
    if (tx.hi > limx) tx = f2_of(limx);
    if (ty.hi < -limy) ty = f2_of(-limy);
    if (ty.hi > limy) ty = f2_of(limy);
    const f2 j00 = f2_div(f2_of(cm.fx), p[2]), j11 = f2_div(f2_of(cm.fy), p[2]);
    const f2 j02 = f2_neg(f2_mul(j00, tx)), j12 = f2_neg(f2_mul(j11, ty));
    f2 T0[3], T1[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        T0[j] = f2_add(f2_mul(j00, f2_of(cm.R[j])), f2_mul(j02, f2_of(cm.R[6 + j])));
        T1[j] = f2_add(f2_mul(j11, f2_of(cm.R[3 + j])), f2_mul(j12, f2_of(cm.R[6 + j])));
    }
    // U = Sigma3 T^T
    const f2 Sm[9] = {S[0], S[1], S[2], S[1], S[3], S[4], S[2], S[4], S[5]};
    f2 U0[3], U1[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        U0[i] = f2_add(f2_add(f2_mul(Sm[3 * i], T0[0]), f2_mul(Sm[3 * i + 1], T0[1])), f2_mul(Sm[3 * i + 2], T0[2]));
        U1[i] = f2_add(f2_add(f2_mul(Sm[3 * i], T1[0]), f2_mul(Sm[3 * i + 1], T1[1])), f2_mul(Sm[3 * i + 2], T1[2]));
    }
    const f2 low = f2_of(kLowpass);
    const f2 a = f2_add(f2_add(f2_add(f2_mul(T0[0], U0[0]), f2_mul(T0[1], U0[1])), f2_mul(T0[2], U0[2])), low);
    const f2 b = f2_add(f2_add(f2_mul(T0[0], U1[0]), f2_mul(T0[1], U1[1])), f2_mul(T0[2], U1[2]));
    const f2 c = f2_add(f2_add(f2_add(f2_mul(T1[0], U1[0]), f2_mul(T1[1], U1[1])), f2_mul(T1[2], U1[2])), low);
    *ca = f2_to_double(a);
    *cb = f2_to_double(b);
    *cc = f2_to_double(c);
}

}  // namespace gs
