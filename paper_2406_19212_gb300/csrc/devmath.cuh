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

// (a, b) <- M (a, b) for a 2x2 matrix of the given structure (row-major re/im).
template <typename R, int SH>
__device__ __forceinline__ void apply2(const R *m, typename CT<R>::T &a, typename CT<R>::T &b)
{
    typedef typename CT<R>::T T;
    if (SH == SH_DENSE1) {
        T x = cmul<T, R>(m[0], m[1], a), y = cmul<T, R>(m[4], m[5], a);
        cfma<T, R>(m[2], m[3], b, x);
        cfma<T, R>(m[6], m[7], b, y);
        a = x;
        b = y;
    } else if (SH == SH_DIAG1) {
        a = cmul<T, R>(m[0], m[1], a);
        b = cmul<T, R>(m[6], m[7], b);
    } else if (SH == SH_ANTI1) {
        T x = cmul<T, R>(m[2], m[3], b), y = cmul<T, R>(m[4], m[5], a);
        a = x;
        b = y;
    } else {  // SH_REAL1
        T x, y;
        x.x = m[0] * a.x + m[2] * b.x;
        x.y = m[0] * a.y + m[2] * b.y;
        y.x = m[4] * a.x + m[6] * b.x;
        y.y = m[4] * a.y + m[6] * b.y;
        a = x;
        b = y;
    }
}

}  // namespace gbvqc
