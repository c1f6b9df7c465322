// Device-side complex helpers shared by the gate kernels.
#pragma once

#include "common.cuh"

namespace gbvqc {

template <typename R> struct CT;
template <> struct CT<float> { typedef float2 T; };
template <> struct CT<double> { typedef double2 T; };

template <typename R> __device__ __forceinline__ const R *mat_of(const MatRec *r);
template <> __device__ __forceinline__ const float *mat_of<float>(const MatRec *r) { return r->f; }
template <> __device__ __forceinline__ const double *mat_of<double>(const MatRec *r) { return r->d; }

template <typename T, typename R>
__device__ __forceinline__ T cmul(R mr, R mi, T a)
{
    T o;
    o.x = mr * a.x - mi * a.y;
    o.y = mr * a.y + mi * a.x;
    return o;
}

template <typename T, typename R>
__device__ __forceinline__ void cfma(R mr, R mi, T a, T &acc)
{
    acc.x = fma(mr, a.x, fma(-mi, a.y, acc.x));
    acc.y = fma(mr, a.y, fma(mi, a.x, acc.y));
}

// a <- (mr + i mi) a, written so the results can reuse a's registers: both products of
// the old value go to temporaries first, then the final FMAs overwrite a.
template <typename T, typename R>
__device__ __forceinline__ void cmul_ip(R mr, R mi, T &a)
{
    const R p = mi * a.y, q = mi * a.x;
    a.x = fma(mr, a.x, -p);
    a.y = fma(mr, a.y, q);
}

// (a, b) <- M (a, b) for a 2x2 matrix of the given structure (row-major re/im).  The
// update is in place: every product of an old value that a later output needs is taken
// before that value's register is overwritten, so the compiler can keep a and b in the
// same registers across gates.
template <typename R, int SH>
__device__ __forceinline__ void apply2(const R *m, typename CT<R>::T &a, typename CT<R>::T &b)
{
    if (SH == SH_DENSE1) {
        if constexpr (sizeof(R) == 4) {
            // packed FP32x2 without swapped operands: for an output row (u, v) the packed
            // P = Re(u) a + Re(v) b and Q = Im(u) a + Im(v) b give the output as
            // (P.x - Q.y, P.y + Q.x): four packed operations and two adds per output, none
            // of them a register move
            const float2 pa = __ffma2_rn(make_float2(m[2], m[2]), b, __fmul2_rn(make_float2(m[0], m[0]), a));
            const float2 qa = __ffma2_rn(make_float2(m[3], m[3]), b, __fmul2_rn(make_float2(m[1], m[1]), a));
            const float2 pb = __ffma2_rn(make_float2(m[6], m[6]), b, __fmul2_rn(make_float2(m[4], m[4]), a));
            const float2 qb = __ffma2_rn(make_float2(m[7], m[7]), b, __fmul2_rn(make_float2(m[5], m[5]), a));
            a = make_float2(pa.x - qa.y, pa.y + qa.x);
            b = make_float2(pb.x - qb.y, pb.y + qb.x);
        } else {
            // contributions of the old a to a' and b'
            const R a1x = fma(m[0], a.x, -m[1] * a.y), a1y = fma(m[0], a.y, m[1] * a.x);
            const R b1x = fma(m[4], a.x, -m[5] * a.y), b1y = fma(m[4], a.y, m[5] * a.x);
            // a' = a1 + m01 b
            a.x = fma(m[2], b.x, fma(-m[3], b.y, a1x));
            a.y = fma(m[2], b.y, fma(m[3], b.x, a1y));
            // b' = b1 + m11 b
            const R bx = fma(-m[7], b.y, b1x), by = fma(m[7], b.x, b1y);
            b.x = fma(m[6], b.x, bx);
            b.y = fma(m[6], b.y, by);
        }
    } else if (SH == SH_ROT1) {
        // R(phi) = [[1, alpha], [0, 1]] [[1, 0], [beta, 1]] [[1, alpha], [0, 1]] with
        // alpha = -tan(phi / 2), beta = sin(phi): three fmas per component pair
        if constexpr (sizeof(R) == 4) {
            const float2 al = make_float2(m[0], m[0]), be = make_float2(m[1], m[1]);
            a = __ffma2_rn(al, b, a);
            b = __ffma2_rn(be, a, b);
            a = __ffma2_rn(al, b, a);
        } else {
            a.x = fma(m[0], b.x, a.x);
            a.y = fma(m[0], b.y, a.y);
            b.x = fma(m[1], a.x, b.x);
            b.y = fma(m[1], a.y, b.y);
            a.x = fma(m[0], b.x, a.x);
            a.y = fma(m[0], b.y, a.y);
        }
    } else if (SH == SH_RDIAG1) {
        // real diagonal (m[1] = m[7] = 0): the diagonal term of each output is one packed
        // multiply (complex64) or two multiplies
        if constexpr (sizeof(R) == 4) {
            const float2 pa = __ffma2_rn(make_float2(m[2], m[2]), b, __fmul2_rn(make_float2(m[0], m[0]), a));
            const float2 qa = __fmul2_rn(make_float2(m[3], m[3]), b);
            const float2 pb = __ffma2_rn(make_float2(m[4], m[4]), a, __fmul2_rn(make_float2(m[6], m[6]), b));
            const float2 qb = __fmul2_rn(make_float2(m[5], m[5]), a);
            a = make_float2(pa.x - qa.y, pa.y + qa.x);
            b = make_float2(pb.x - qb.y, pb.y + qb.x);
        } else {
            const R ax = fma(m[2], b.x, fma(-m[3], b.y, m[0] * a.x)), ay = fma(m[2], b.y, fma(m[3], b.x, m[0] * a.y));
            const R bx = fma(m[4], a.x, fma(-m[5], a.y, m[6] * b.x)), by = fma(m[4], a.y, fma(m[5], a.x, m[6] * b.y));
            a.x = ax;
            a.y = ay;
            b.x = bx;
            b.y = by;
        }
    } else if (SH == SH_DIAG1) {
        cmul_ip(m[0], m[1], a);
        cmul_ip(m[6], m[7], b);
    } else if (SH == SH_IMAG1) {
        // [[p, i q], [i r, s]] with p = m[0], q = m[3], r = m[5], s = m[6] real:
        // a' = p a + i q b, b' = i r a + s b
        if constexpr (sizeof(R) == 4) {
            const float2 t = make_float2(-m[3] * b.y, m[3] * b.x);
            const float2 u = make_float2(-m[5] * a.y, m[5] * a.x);
            a = __ffma2_rn(make_float2(m[0], m[0]), a, t);
            b = __ffma2_rn(make_float2(m[6], m[6]), b, u);
        } else {
            const R tx = -m[3] * b.y, ty = m[3] * b.x, ux = -m[5] * a.y, uy = m[5] * a.x;
            a.x = fma(m[0], a.x, tx);
            a.y = fma(m[0], a.y, ty);
            b.x = fma(m[6], b.x, ux);
            b.y = fma(m[6], b.y, uy);
        }
    } else if (SH == SH_ANTI1) {
        const R x = fma(m[2], b.x, -m[3] * b.y), y = fma(m[2], b.y, m[3] * b.x);
        b.x = fma(m[4], a.x, -m[5] * a.y);
        b.y = fma(m[4], a.y, m[5] * a.x);
        a.x = x;
        a.y = y;
    } else {  // SH_REAL1
        if constexpr (sizeof(R) == 4) {
            // both components of an amplitude take the same real coefficient: one packed
            // FP32x2 multiply or fma per coefficient (same IEEE operations per lane)
            const float2 m0 = make_float2(m[0], m[0]), m2 = make_float2(m[2], m[2]);
            const float2 m4 = make_float2(m[4], m[4]), m6 = make_float2(m[6], m[6]);
            const float2 t = __fmul2_rn(m0, a), u = __fmul2_rn(m4, a);
            a = __ffma2_rn(m2, b, t);
            b = __ffma2_rn(m6, b, u);
        } else {
            const R t0 = m[0] * a.x, t1 = m[0] * a.y, u0 = m[4] * a.x, u1 = m[4] * a.y;
            a.x = fma(m[2], b.x, t0);
            a.y = fma(m[2], b.y, t1);
            b.x = fma(m[6], b.x, u0);
            b.y = fma(m[6], b.y, u1);
        }
    }
}

}  // namespace gbvqc
