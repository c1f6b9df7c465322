// Device code of the fused tile passes (shared by the single-circuit and batched kernels).
//
// Fused tile passes: one HBM read and one write of the state apply a whole run of gates.
//
// A pass names a set S of t "tile" qubits (the lowest `low` qubits are always in S, so
// every tile is made of contiguous 2^low-amplitude segments).  CTA i owns the 2^t
// amplitudes whose non-tile bits spell i, stages them in shared memory together with
// the pass's gate records and matrices, applies the gates and writes the tile back.
// Inside the tile, gates run in "sub-runs": each sub-run names NR tile positions that
// every thread gathers into registers (2^NR amplitudes per thread), applies all of the
// sub-run's gates on them with no further memory traffic, and scatters back.
//
// Diagonal gates need no register position: a run of them is applied as one phase per
// amplitude, the product of a per-CTA constant (tile-index bits), a per-thread constant
// (tile bits outside the registers) and tables over the register bits built by doubling.
//
// This is the GPU counterpart of the paper's gate fusion for compute density (Sec. III.B,
// citing gate fusion) and of its aggregation of independent amplitude groups (Fig. 3):
// the 2^low contiguous amplitudes of a segment play the role of the paper's
// vectorisable inner dimension.
//
// The reverse variant (Algorithm 2) carries Phi and Psi tiles together: for every gate
// in reverse order it accumulates the gradient term coef * Im <Psi|P|Phi> of the gate's
// Pauli generator P (dQ/dtheta = -i/2 P Q for Q = exp(-i theta P/2), so
// 2 Re <Psi|dQ|Phi_{j-1}> = Im <Psi|P|Phi_j>), then uncomputes Phi with Q^{-1} and Psi
// with Q^dag.  In a diagonal run every Z generator is read from the states after the
// whole run (diagonal matrices commute with Z).  Per-thread partials over 2^NR terms
// are summed across the warp with shuffles (FP32 for complex64, FP64 for complex128) and
// across warps in FP64 in fixed order, giving one FP64 partial per (gradient slot, tile).
#pragma once

#include "devmath.cuh"
#include "kernels.h"

namespace gbvqc {

template <typename R> struct SwzBits;
template <> struct SwzBits<float> { static constexpr int B = 4; };   // 16 x 8 B = 128 B
template <> struct SwzBits<double> { static constexpr int B = 3; };  // 8 x 16 B = 128 B

// XOR swizzle of the shared-memory slot of local amplitude l: folds bits [B, 2B) onto
// bits [0, B) so strided register gathers spread over all banks.
template <typename R>
__device__ __forceinline__ int swz(int l)
{
    constexpr int B = SwzBits<R>::B;
    return l ^ ((l >> B) & ((1 << B) - 1));
}

// --------------------------------------------------------------- register-slot gates

template <typename R, int NR, int K, int SH>
__device__ __forceinline__ void rg1(typename CT<R>::T *a, const R *m)
{
#pragma unroll
    for (int j = 0; j < (1 << NR); j++)
        if (!(j & (1 << K))) apply2<R, SH>(m, a[j], a[j | (1 << K)]);
}

template <typename R, int NR, int SH>
__device__ __forceinline__ void rg1_dispatch(int k, typename CT<R>::T *a, const R *m)
{
#define GBVQC_RG1(K) \
    case K:          \
        if constexpr (K < NR) rg1<R, NR, K, SH>(a, m); \
        break;
    switch (k) {
        GBVQC_RG1(0) GBVQC_RG1(1) GBVQC_RG1(2) GBVQC_RG1(3) GBVQC_RG1(4) GBVQC_RG1(5)
    }
#undef GBVQC_RG1
}

// Two-qubit gate on register slots (K0 = matrix bit 0, K1 = matrix bit 1).
template <typename R, int NR, int K0, int K1, int SH>
__device__ __forceinline__ void rg2(typename CT<R>::T *a, const R *m, int perm)
{
    typedef typename CT<R>::T T;
#pragma unroll
    for (int j = 0; j < (1 << NR); j++) {
        if (j & ((1 << K0) | (1 << K1))) continue;
        const int i1 = j | (1 << K0), i2 = j | (1 << K1), i3 = j | (1 << K0) | (1 << K1);
        if (SH == SH_CTRL2) {
            R u[8] = {m[10], m[11], m[14], m[15], m[26], m[27], m[30], m[31]};
            apply2<R, SH_DENSE1>(u, a[i1], a[i3]);
            continue;
        }
        if (SH == SH_BLOCK2) {
            R u[8] = GBVQC_BLOCK2_U(m);
            apply2<R, SH_DENSE1>(u, a[i1], a[i2]);
            cmul_ip<T, R>(m[0], m[1], a[j]);
            cmul_ip<T, R>(m[30], m[31], a[i3]);
            continue;
        }
        if (SH == SH_PAR2 || SH == SH_RPAR2) {
            R o[8] = GBVQC_OUTER_U(m), u[8] = GBVQC_BLOCK2_U(m);
            apply2<R, SH == SH_PAR2 ? SH_DENSE1 : SH_REAL1>(o, a[j], a[i3]);
            apply2<R, SH == SH_PAR2 ? SH_DENSE1 : SH_REAL1>(u, a[i1], a[i2]);
            continue;
        }
        T v[4] = {a[j], a[i1], a[i2], a[i3]}, w[4];
        if (SH == SH_DENSE2) {
#pragma unroll
            for (int r = 0; r < 4; r++) {
                T acc = cmul<T, R>(m[8 * r], m[8 * r + 1], v[0]);
#pragma unroll
                for (int c = 1; c < 4; c++) cfma<T, R>(m[8 * r + 2 * c], m[8 * r + 2 * c + 1], v[c], acc);
                w[r] = acc;
            }
        } else {  // SH_PERM2
#pragma unroll
            for (int r = 0; r < 4; r++) {
                const int c = (perm >> (2 * r)) & 3;
                T x = c == 0 ? v[0] : c == 1 ? v[1] : c == 2 ? v[2] : v[3];
                R mr = m[8 * r + 2 * c], mi = m[8 * r + 2 * c + 1];
                w[r] = cmul<T, R>(mr, mi, x);
            }
        }
        a[j] = w[0];
        a[i1] = w[1];
        a[i2] = w[2];
        a[i3] = w[3];
    }
}

// SH_BLOCK2 with a plan-time variant (a fixed matrix): the 2x2 on {|01>, |10>} applied
// in its INNER shape, the |00> / |11> phases skipped where they are exactly 1 (P00 /
// P11 false).  The skipped terms are exact zeros or unit factors.
template <typename R, int NR, int K0, int K1, int INNER, bool P00, bool P11>
__device__ __forceinline__ void rg2_block2v(typename CT<R>::T *a, const R *m)
{
    typedef typename CT<R>::T T;
    const R u[8] = GBVQC_BLOCK2_U(m);
#pragma unroll
    for (int j = 0; j < (1 << NR); j++) {
        if (j & ((1 << K0) | (1 << K1))) continue;
        const int i1 = j | (1 << K0), i2 = j | (1 << K1), i3 = i1 | i2;
        apply2<R, INNER>(u, a[i1], a[i2]);
        if (P00) cmul_ip<T, R>(m[0], m[1], a[j]);
        if (P11) cmul_ip<T, R>(m[30], m[31], a[i3]);
    }
}

template <typename R, int NR, int SH>
__device__ __forceinline__ void rg2_dispatch(int k0, int k1, typename CT<R>::T *a, const R *m, int perm)
{
#define GBVQC_RG2(K0, K1) \
    case K0 * 8 + K1:     \
        if constexpr (K0 < NR && K1 < NR) rg2<R, NR, K0, K1, SH>(a, m, perm); \
        break;
    switch (k0 * 8 + k1) {
        GBVQC_RG2(0, 1) GBVQC_RG2(0, 2) GBVQC_RG2(0, 3) GBVQC_RG2(0, 4)
        GBVQC_RG2(1, 0) GBVQC_RG2(1, 2) GBVQC_RG2(1, 3) GBVQC_RG2(1, 4)
        GBVQC_RG2(2, 0) GBVQC_RG2(2, 1) GBVQC_RG2(2, 3) GBVQC_RG2(2, 4)
        GBVQC_RG2(3, 0) GBVQC_RG2(3, 1) GBVQC_RG2(3, 2) GBVQC_RG2(3, 4)
        GBVQC_RG2(4, 0) GBVQC_RG2(4, 1) GBVQC_RG2(4, 2) GBVQC_RG2(4, 3)
    }
#undef GBVQC_RG2
}

// Gradient probe: sum over the register quadruples of Re sum_r conj(p_r) (K f)_r with the
// 4x4 K (row-major re/im; K0 = matrix bit 0, K1 = matrix bit 1), f = Phi, p = Psi.
template <typename R, int NR, int K0, int K1>
__device__ __forceinline__ R probe2(const typename CT<R>::T *f, const typename CT<R>::T *p, const R *m)
{
    typedef typename CT<R>::T T;
    R s = 0;
#pragma unroll
    for (int j = 0; j < (1 << NR); j++) {
        if (j & ((1 << K0) | (1 << K1))) continue;
        const int idx[4] = {j, j | (1 << K0), j | (1 << K1), j | (1 << K0) | (1 << K1)};
#pragma unroll
        for (int r = 0; r < 4; r++) {
            T w = cmul<T, R>(m[8 * r], m[8 * r + 1], f[idx[0]]);
#pragma unroll
            for (int c = 1; c < 4; c++) cfma<T, R>(m[8 * r + 2 * c], m[8 * r + 2 * c + 1], f[idx[c]], w);
            s += p[idx[r]].x * w.x + p[idx[r]].y * w.y;
        }
    }
    return s;
}

template <typename R, int NR>
__device__ __forceinline__ R probe2_dispatch(int k0, int k1, const typename CT<R>::T *f, const typename CT<R>::T *p,
                                             const R *m)
{
#define GBVQC_PR2(K0, K1) \
    case K0 * 8 + K1:     \
        if constexpr (K0 < NR && K1 < NR) return probe2<R, NR, K0, K1>(f, p, m); \
        break;
    switch (k0 * 8 + k1) {
        GBVQC_PR2(0, 1) GBVQC_PR2(0, 2) GBVQC_PR2(0, 3) GBVQC_PR2(0, 4)
        GBVQC_PR2(1, 0) GBVQC_PR2(1, 2) GBVQC_PR2(1, 3) GBVQC_PR2(1, 4)
        GBVQC_PR2(2, 0) GBVQC_PR2(2, 1) GBVQC_PR2(2, 3) GBVQC_PR2(2, 4)
        GBVQC_PR2(3, 0) GBVQC_PR2(3, 1) GBVQC_PR2(3, 2) GBVQC_PR2(3, 4)
        GBVQC_PR2(4, 0) GBVQC_PR2(4, 1) GBVQC_PR2(4, 2) GBVQC_PR2(4, 3)
    }
#undef GBVQC_PR2
    return 0;
}

// Bit of a non-register position code (constant over the thread's amplitudes).
template <int NR>
__device__ __forceinline__ int const_bit(int code, int base, int64_t tilebase)
{
    if (code < 0) return (int)((tilebase >> (-1 - code)) & 1);
    return (base >> (code - NR)) & 1;
}

// Non-diagonal gate on register slots.  Kernels compiled without TWOQ never see
// two-qubit gates (the planner flags every pass that holds one), which keeps their
// code paths out of the common one-qubit loop.
template <typename R, int NR, bool TWOQ>
__device__ __forceinline__ void apply_fgate(int type, int ga, int gb, int perm, const R *m,
                                            typename CT<R>::T *a)
{
    switch (type) {
    case FT_DENSE1: rg1_dispatch<R, NR, SH_DENSE1>(ga, a, m); break;
    case FT_REAL1: rg1_dispatch<R, NR, SH_REAL1>(ga, a, m); break;
    case FT_ANTI1: rg1_dispatch<R, NR, SH_ANTI1>(ga, a, m); break;
    case FT_IMAG1: rg1_dispatch<R, NR, SH_IMAG1>(ga, a, m); break;
    default:
        if constexpr (TWOQ) {
            switch (type) {
            case FT_DENSE2: rg2_dispatch<R, NR, SH_DENSE2>(ga, gb, a, m, 0); break;
            case FT_PERM2: rg2_dispatch<R, NR, SH_PERM2>(ga, gb, a, m, perm); break;
            case FT_BLOCK2: rg2_dispatch<R, NR, SH_BLOCK2>(ga, gb, a, m, 0); break;
            case FT_RPAR2: rg2_dispatch<R, NR, SH_RPAR2>(ga, gb, a, m, 0); break;
            case FT_PAR2: rg2_dispatch<R, NR, SH_PAR2>(ga, gb, a, m, 0); break;
            default: rg2_dispatch<R, NR, SH_CTRL2>(ga, gb, a, m, 0); break;
            }
        }
        break;
    }
}

// ------------------------------------------------------------- diagonal phase blocks

// Element r of the diagonal of a k-qubit matrix staged as 2x2 (one unit) or 4x4 (four).
template <typename R>
__device__ __forceinline__ void diag_elem(const R *m, int k, int r, R &re, R &im)
{
    const int o = k == 1 ? 6 * r : 10 * r;
    re = m[o];
    im = m[o + 1];
}

template <typename R>
__device__ __forceinline__ void cmul_inplace(R &xr, R &xi, R yr, R yi)
{
    R t = xr * yr - xi * yi;
    xi = xr * yi + xi * yr;
    xr = t;
}

// Factor pairs (f0, f1) of the register bits: the phase of register amplitude j is the
// product over bits k of f_{bit k of j}[k].
template <typename R, int NR>
struct RegPairs {
    R p0r[NR], p0i[NR], p1r[NR], p1i[NR];
    __device__ __forceinline__ void init()
    {
#pragma unroll
        for (int k = 0; k < NR; k++) {
            p0r[k] = 1; p0i[k] = 0; p1r[k] = 1; p1i[k] = 0;
        }
    }
    // multiply (e0, e1) into register bit k (k uniform; one case runs)
    __device__ __forceinline__ void mul(int k, R e0r, R e0i, R e1r, R e1i)
    {
#define GBVQC_PM(K)                                              \
    case K:                                                      \
        if constexpr (K < NR) {                                  \
            cmul_inplace<R>(p0r[K], p0i[K], e0r, e0i);           \
            cmul_inplace<R>(p1r[K], p1i[K], e1r, e1i);           \
        }                                                        \
        break;
        switch (k) { GBVQC_PM(0) GBVQC_PM(1) GBVQC_PM(2) GBVQC_PM(3) GBVQC_PM(4) GBVQC_PM(5) }
#undef GBVQC_PM
    }
};

// a[j] *= c (or -a[j] for NEG) on the register amplitudes whose bits K0 and K1 are both 1.
template <typename R, int NR, int K0, int K1, bool NEG>
__device__ __forceinline__ void cphase(typename CT<R>::T *a, R cr, R ci)
{
    typedef typename CT<R>::T T;
#pragma unroll
    for (int j = 0; j < (1 << NR); j++) {
        if (!(((j >> K0) & 1) && ((j >> K1) & 1))) continue;
        if (NEG) {
            a[j].x = -a[j].x;
            a[j].y = -a[j].y;
        } else {
            cmul_ip<T, R>(cr, ci, a[j]);
        }
    }
}

template <typename R, int NR, bool NEG>
__device__ __forceinline__ void cphase_dispatch(int k0, int k1, typename CT<R>::T *a, R cr, R ci)
{
    const int lo = k0 < k1 ? k0 : k1, hi = k0 < k1 ? k1 : k0;
#define GBVQC_CP(L, H) \
    case L * 8 + H:    \
        if constexpr (H < NR) cphase<R, NR, L, H, NEG>(a, cr, ci); \
        break;
    switch (lo * 8 + hi) {
        GBVQC_CP(0, 1) GBVQC_CP(0, 2) GBVQC_CP(0, 3) GBVQC_CP(0, 4) GBVQC_CP(1, 2)
        GBVQC_CP(1, 3) GBVQC_CP(1, 4) GBVQC_CP(2, 3) GBVQC_CP(2, 4) GBVQC_CP(3, 4)
    }
#undef GBVQC_CP
}

template <typename R>
__device__ __forceinline__ void cdiv(R ar, R ai, R br, R bi, R &qr, R &qi)
{
    const R inv = R(1) / (br * br + bi * bi);
    qr = (ar * br + ai * bi) * inv;
    qi = (ai * br - ar * bi) * inv;
}

// Apply one phase block to a (and b, if given).  `ents` points after the Z entries; the
// tile-constant entries (the first nt) are already folded into (c0r, c0i).  The phase
// of register amplitude j is c * TL[j & lo] * TH[j >> H] with c the product of the
// tile-constant and thread-local entries and TL, TH tables over the low and high halves
// of the register bits built by doubling from the factor pairs; PAIR entries are split
// into factor pairs d0 (1, d1/d0) (1, d2/d0) and the controlled phase d3 d0 / (d1 d2).
template <typename R, int NR>
__device__ __forceinline__ void phase_block(const DEnt *ents, int counts, const R *smat, bool second,
                                            R c0r, R c0i, typename CT<R>::T *a, typename CT<R>::T *b,
                                            int base, int64_t tilebase)
{
    typedef typename CT<R>::T T;
    constexpr int H = NR / 2;
    const int nt = counts & 255, nl = (counts >> 8) & 255, nr = (counts >> 16) & 255, np = (counts >> 24) & 255;
    const DEnt *e = ents + nt;
    R cr = c0r, ci = c0i;
    for (int i = 0; i < nl; i++, e++) {  // thread-local constants
        const R *m = smat + 8 * (second ? e->mat2 : e->mat);
        const int idx = e->k == 1 ? const_bit<NR>(e->ca, base, tilebase)
                                  : const_bit<NR>(e->ca, base, tilebase) | (const_bit<NR>(e->cb, base, tilebase) << 1);
        R er, ei;
        diag_elem<R>(m, e->k, idx, er, ei);
        cmul_inplace<R>(cr, ci, er, ei);
    }
    RegPairs<R, NR> P;
    P.init();
    for (int i = 0; i < nr; i++, e++) {  // one register bit
        const R *m = smat + 8 * (second ? e->mat2 : e->mat);
        R e0r, e0i, e1r, e1i;
        int k;
        if (e->k == 1) {
            k = e->ca;
            diag_elem<R>(m, 1, 0, e0r, e0i);
            diag_elem<R>(m, 1, 1, e1r, e1i);
        } else {
            const bool ra = e->ca >= 0 && e->ca < NR;
            k = ra ? e->ca : e->cb;
            const int cbit = ra ? const_bit<NR>(e->cb, base, tilebase) : const_bit<NR>(e->ca, base, tilebase);
            diag_elem<R>(m, 2, ra ? 2 * cbit : cbit, e0r, e0i);
            diag_elem<R>(m, 2, ra ? 1 + 2 * cbit : cbit + 2, e1r, e1i);
        }
        P.mul(k, e0r, e0i, e1r, e1i);
    }
    for (int i = 0; i < np; i++, e++) {  // two register bits
        if (e->cls == DC_PAIR_CZ) {
            cphase_dispatch<R, NR, true>(e->ca, e->cb, a, R(0), R(0));
            if (b) cphase_dispatch<R, NR, true>(e->ca, e->cb, b, R(0), R(0));
            continue;
        }
        const R *m = smat + 8 * (second ? e->mat2 : e->mat);
        R d0r, d0i, d1r, d1i, d2r, d2i, d3r, d3i;
        diag_elem<R>(m, 2, 0, d0r, d0i);
        diag_elem<R>(m, 2, 1, d1r, d1i);
        diag_elem<R>(m, 2, 2, d2r, d2i);
        diag_elem<R>(m, 2, 3, d3r, d3i);
        R qr, qi;
        cmul_inplace<R>(cr, ci, d0r, d0i);
        cdiv<R>(d1r, d1i, d0r, d0i, qr, qi);
        P.mul(e->ca, R(1), R(0), qr, qi);
        cdiv<R>(d2r, d2i, d0r, d0i, qr, qi);
        P.mul(e->cb, R(1), R(0), qr, qi);
        R nr_ = d3r, ni_ = d3i, dr_ = d1r, di_ = d1i;
        cmul_inplace<R>(nr_, ni_, d0r, d0i);
        cmul_inplace<R>(dr_, di_, d2r, d2i);
        cdiv<R>(nr_, ni_, dr_, di_, qr, qi);
        cphase_dispatch<R, NR, false>(e->ca, e->cb, a, qr, qi);
        if (b) cphase_dispatch<R, NR, false>(e->ca, e->cb, b, qr, qi);
    }
    R lr[1 << H], li[1 << H], hr[1 << (NR - H)], hi[1 << (NR - H)];
    lr[0] = 1;
    li[0] = 0;
#pragma unroll
    for (int k = 0; k < H; k++) {
#pragma unroll
        for (int j = 0; j < (1 << k); j++) {
            lr[j | (1 << k)] = lr[j] * P.p1r[k] - li[j] * P.p1i[k];
            li[j | (1 << k)] = lr[j] * P.p1i[k] + li[j] * P.p1r[k];
            R x = lr[j] * P.p0r[k] - li[j] * P.p0i[k];
            li[j] = lr[j] * P.p0i[k] + li[j] * P.p0r[k];
            lr[j] = x;
        }
    }
    hr[0] = cr;
    hi[0] = ci;
#pragma unroll
    for (int k = 0; k < NR - H; k++) {
#pragma unroll
        for (int j = 0; j < (1 << k); j++) {
            hr[j | (1 << k)] = hr[j] * P.p1r[H + k] - hi[j] * P.p1i[H + k];
            hi[j | (1 << k)] = hr[j] * P.p1i[H + k] + hi[j] * P.p1r[H + k];
            R x = hr[j] * P.p0r[H + k] - hi[j] * P.p0i[H + k];
            hi[j] = hr[j] * P.p0i[H + k] + hi[j] * P.p0r[H + k];
            hr[j] = x;
        }
    }
#pragma unroll
    for (int j = 0; j < (1 << NR); j++) {
        const int jl = j & ((1 << H) - 1), jh = j >> H;
        const R pr = lr[jl] * hr[jh] - li[jl] * hi[jh], pi = lr[jl] * hi[jh] + li[jl] * hr[jh];
        cmul_ip<T, R>(pr, pi, a[j]);
        if (b) cmul_ip<T, R>(pr, pi, b[j]);
    }
}

// Bit j of the result: parity of the register bits of j selected by sm (sign pattern of
// the mixed CZ entries), for the 2^NR register indices.
template <int NR>
__device__ __forceinline__ uint32_t parity_bits(uint32_t sm)
{
    constexpr uint32_t col[5] = {0xAAAAAAAAu, 0xCCCCCCCCu, 0xF0F0F0F0u, 0xFF00FF00u, 0xFFFF0000u};
    uint32_t par = 0;
#pragma unroll
    for (int k = 0; k < NR; k++)
        if ((sm >> k) & 1) par ^= col[k];
    return par;
}

// Table-mode phase block (FLAG_TABLE): amplitude j is multiplied by c * table[j] * (-1)^(j . sm)
// with c the product of the tile-constant (c0) and thread-local entries, table the block's
// register phase table in shared memory (written per step by k_phase_tables) and sm the
// register bits of the mixed CZ entries whose constant bit is 1 in this thread.  `ents`
// points after the Z entries; b (if given) takes the same phases.
template <typename R, int NR>
__device__ __forceinline__ void phase_table(const DEnt *ents, int counts, const R *smat, int tab, bool second,
                                            R c0r, R c0i, typename CT<R>::T *a, typename CT<R>::T *b, int base,
                                            int64_t tilebase)
{
    typedef typename CT<R>::T T;
    const int nt = counts & 255, nl = (counts >> 8) & 255, nm = (counts >> 16) & 255;
    const DEnt *e = ents + nt;
    R cr = c0r, ci = c0i;
    for (int i = 0; i < nl; i++, e++) {  // thread-local constants
        const R *m = smat + 8 * (second ? e->mat2 : e->mat);
        const int idx = e->k == 1 ? const_bit<NR>(e->ca, base, tilebase)
                                  : const_bit<NR>(e->ca, base, tilebase) | (const_bit<NR>(e->cb, base, tilebase) << 1);
        R er, ei;
        diag_elem<R>(m, e->k, idx, er, ei);
        cmul_inplace<R>(cr, ci, er, ei);
    }
    uint32_t sm = 0;
    for (int i = 0; i < nm; i++, e++) {  // mixed CZ: sign on register bit k where the constant bit is 1
        const bool ra = e->ca >= 0 && e->ca < NR;
        const int k = ra ? e->ca : e->cb, c = ra ? e->cb : e->ca;
        sm ^= (uint32_t)const_bit<NR>(c, base, tilebase) << k;
    }
    const uint32_t par = parity_bits<NR>(sm);
    const bool has_c = (nt | nl) != 0;
    const T *tb = reinterpret_cast<const T *>(smat + 8 * tab);
#pragma unroll
    for (int j = 0; j < (1 << NR); j++) {
        T t = tb[j];
        if ((par >> j) & 1) {
            t.x = -t.x;
            t.y = -t.y;
        }
        if (has_c) {
            const R x = cr * t.x - ci * t.y;
            t.y = cr * t.y + ci * t.x;
            t.x = x;
        }
        cmul_ip<T, R>(t.x, t.y, a[j]);
        if (b) cmul_ip<T, R>(t.x, t.y, b[j]);
    }
}

// ------------------------------------------------------------ generator inner products

// Im <Psi| P_K |Phi> over the thread's register amplitudes, P = X or Y on slot K.
template <typename R, int NR, int K, int G>
__device__ __forceinline__ R gen_xy(const typename CT<R>::T *f, const typename CT<R>::T *p)
{
    if constexpr (sizeof(R) == 4 && G == GEN_Y) {
        // Re(conj(p1) f0) - Re(conj(p0) f1) as two packed accumulators of
        // (re*re, im*im) products
        float2 sp = make_float2(0.f, 0.f), sm = make_float2(0.f, 0.f);
#pragma unroll
        for (int j = 0; j < (1 << NR); j++) {
            if (j & (1 << K)) continue;
            const int j1 = j | (1 << K);
            sp = __ffma2_rn(p[j1], f[j], sp);
            sm = __ffma2_rn(p[j], f[j1], sm);
        }
        return (sp.x + sp.y) - (sm.x + sm.y);
    }
    R s = 0;
#pragma unroll
    for (int j = 0; j < (1 << NR); j++) {
        if (j & (1 << K)) continue;
        const int j1 = j | (1 << K);
        if (G == GEN_X) {  // Im(conj(p0) f1 + conj(p1) f0)
            s += (p[j].x * f[j1].y - p[j].y * f[j1].x) + (p[j1].x * f[j].y - p[j1].y * f[j].x);
        } else {           // Re(conj(p1) f0) - Re(conj(p0) f1)
            s += (p[j1].x * f[j].x + p[j1].y * f[j].y) - (p[j].x * f[j1].x + p[j].y * f[j1].y);
        }
    }
    return s;
}

template <typename R, int NR, int G>
__device__ __forceinline__ R gen_xy_dispatch(int k, const typename CT<R>::T *f, const typename CT<R>::T *p)
{
#define GBVQC_GXY(K) \
    case K:          \
        if constexpr (K < NR) return gen_xy<R, NR, K, G>(f, p); \
        break;
    switch (k) {
        GBVQC_GXY(0) GBVQC_GXY(1) GBVQC_GXY(2) GBVQC_GXY(3) GBVQC_GXY(4) GBVQC_GXY(5)
    }
#undef GBVQC_GXY
    return 0;
}

template <typename R>
struct RedCtx {
    R *sgrad;  // per (slot, warp) partials in the state's precision (exact in FP64 later)
    int slot_begin, nwarps, warp, lane, lanes;
    unsigned lanemask;
};

// Sum a per-thread partial over the warp (shuffles in the state's precision: FP32 for
// complex64, FP64 for complex128) and store it for its slot.
template <typename R>
__device__ __forceinline__ void emit_partial(const RedCtx<R> &c, int slot, R v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        if (o < c.lanes) v += __shfl_xor_sync(c.lanemask, v, o);
    if (c.lane == 0) c.sgrad[(slot - c.slot_begin) * c.nwarps + c.warp] = v;
}

// Several per-thread partials at once (specialised passes): N interleaved warp reductions,
// lane 0 stores each for its pass-local slot.
template <typename R, int N>
__device__ __forceinline__ void emit_partials(const RedCtx<R> &c, const int (&local_slot)[N], R (&v)[N])
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int k = 0; k < N; k++)
            if (o < c.lanes) v[k] += __shfl_xor_sync(c.lanemask, v[k], o);
    if (c.lane == 0)
#pragma unroll
        for (int k = 0; k < N; k++) c.sgrad[local_slot[k] * c.nwarps + c.warp] = v[k];
}

// N per-thread partials (N <= 32) summed over the warp by a transpose reduction, for the
// pass-local slots first_slot .. first_slot + N - 1: each of the first log2(N') steps
// (N' = N rounded up to a power of two) halves the values a lane holds, exchanging the
// half it gives up with its partner, so N values cost about 2 N' shuffles and adds
// instead of 5 N; the remaining steps are a plain butterfly.  Lane l then holds the sum
// of value index (its high lane bits), and the lanes whose low bits are zero store it.
// Blocks narrower than a warp take the plain form.
template <typename R, int N>
__device__ __forceinline__ void emit_partials_seq(const RedCtx<R> &c, int first_slot, R (&v)[N])
{
    constexpr int S = N <= 1 ? 0 : N <= 2 ? 1 : N <= 4 ? 2 : N <= 8 ? 3 : N <= 16 ? 4 : 5;
    if (c.lanes < 32) {
        int ls[N];
#pragma unroll
        for (int k = 0; k < N; k++) ls[k] = first_slot + k;
        emit_partials<R, N>(c, ls, v);
        return;
    }
    R w[1 << S];
#pragma unroll
    for (int k = 0; k < (1 << S); k++) w[k] = k < N ? v[k] : R(0);
#pragma unroll
    for (int t = 0; t < S; t++) {
        const int o = 16 >> t, half = 1 << (S - t - 1);
        const bool hi = (c.lane & o) != 0;
#pragma unroll
        for (int i = 0; i < half; i++) {
            const R send = hi ? w[i] : w[i + half];
            const R keep = hi ? w[i + half] : w[i];
            w[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
        }
    }
#pragma unroll
    for (int o = 16 >> S; o > 0; o >>= 1) w[0] += __shfl_xor_sync(0xffffffffu, w[0], o);
    int idx = 0;
#pragma unroll
    for (int t = 0; t < S; t++)
        if (c.lane & (16 >> t)) idx |= 1 << (S - t - 1);
    if ((c.lane & ((1 << (5 - S)) - 1)) == 0 && idx < N) c.sgrad[(first_slot + idx) * c.nwarps + c.warp] = w[0];
}

// A 2x2 matrix unit (8 reals) from shared memory as 16-byte vector loads.
template <typename R>
__device__ __forceinline__ void load_unit(const R *p, R (&m)[8])
{
    if constexpr (sizeof(R) == 4) {
        const float4 x = reinterpret_cast<const float4 *>(p)[0], y = reinterpret_cast<const float4 *>(p)[1];
        m[0] = x.x; m[1] = x.y; m[2] = x.z; m[3] = x.w; m[4] = y.x; m[5] = y.y; m[6] = y.z; m[7] = y.w;
    } else {
#pragma unroll
        for (int i = 0; i < 4; i++) {
            const double2 v = reinterpret_cast<const double2 *>(p)[i];
            m[2 * i] = v.x;
            m[2 * i + 1] = v.y;
        }
    }
}

// One-qubit gate of layer shape code sh (0 dense, 1 real, 2 imaginary off-diagonal,
// 3 anti-diagonal) on register slot K.
template <typename R, int NR, int K>
__device__ __forceinline__ void layer_gate(int sh, const R *m, typename CT<R>::T *a)
{
    if (sh == 1) rg1<R, NR, K, SH_REAL1>(a, m);
    else if (sh == 2) rg1<R, NR, K, SH_IMAG1>(a, m);
    else if (sh == 0) rg1<R, NR, K, SH_DENSE1>(a, m);
    else if (sh == 4) rg1<R, NR, K, SH_ROT1>(a, m);
    else rg1<R, NR, K, SH_ANTI1>(a, m);
}

// FT_LAYER1: one-qubit gates on distinct register slots, slot loop unrolled at compile
// time (no per-gate dispatch on the slot).  Entry-driven form: each entry names its
// shape, generator class, gradient slot and matrix units.  Reverse: generator read, then
// Phi and Psi.
template <typename R, int NR, bool REV, int K>
__device__ __forceinline__ void layer_slot_ent(int mask, const DEnt *le, int &idx, const R *smat, typename CT<R>::T *a,
                                               typename CT<R>::T *b, R (&gv)[NR], int (&gs)[NR])
{
    if constexpr (K < NR) {
        if ((mask >> K) & 1) {
            const DEnt d = le[idx++];
            if constexpr (REV) {  // the read is reduced over the warp after the layer
                gs[K] = d.cls == GEN_NONE ? -1 : d.slot;
                if (d.cls == GEN_X) gv[K] = gen_xy<R, NR, K, GEN_X>(a, b) * (R)d.coef;
                else if (d.cls == GEN_Y) gv[K] = gen_xy<R, NR, K, GEN_Y>(a, b) * (R)d.coef;
            }
            const R *m = smat + 8 * d.mat;
            const R *m2 = smat + 8 * d.mat2;
            if (d.k == SH_REAL1) {
                rg1<R, NR, K, SH_REAL1>(a, m);
                if constexpr (REV) rg1<R, NR, K, SH_REAL1>(b, m2);
            } else if (d.k == SH_IMAG1) {
                rg1<R, NR, K, SH_IMAG1>(a, m);
                if constexpr (REV) rg1<R, NR, K, SH_IMAG1>(b, m2);
            } else if (d.k == SH_ROT1) {
                rg1<R, NR, K, SH_ROT1>(a, m);
                if constexpr (REV) rg1<R, NR, K, SH_ROT1>(b, m2);
            } else if (d.k == SH_DENSE1 || d.k == SH_RDIAG1) {  // (general form for both)
                rg1<R, NR, K, SH_DENSE1>(a, m);
                if constexpr (REV) rg1<R, NR, K, SH_DENSE1>(b, m2);
            } else {
                rg1<R, NR, K, SH_ANTI1>(a, m);
                if constexpr (REV) rg1<R, NR, K, SH_ANTI1>(b, m2);
            }
        }
        layer_slot_ent<R, NR, REV, K + 1>(mask, le, idx, smat, a, b, gv, gs);
    }
}

// Forward form for kernels without two-qubit gates: the record carries each slot's shape
// (codes, 3 bits per slot) and the first of the layer's consecutive matrix units, so no
// matrix address waits for an entry load, and the next entry's matrix is loaded into
// registers while the current one is applied.
template <typename R, int NR, int K>
__device__ __forceinline__ void layer_slot_pf(int mask, int codes, const R *mp, int last, int &idx, R (&cur)[8],
                                              typename CT<R>::T *a)
{
    if constexpr (K < NR) {
        if ((mask >> K) & 1) {
            R nxt[8];
            load_unit<R>(mp + 8 * (idx + 1 < last ? idx + 1 : last), nxt);
            layer_gate<R, NR, K>((codes >> (3 * K)) & 7, cur, a);
#pragma unroll
            for (int i = 0; i < 8; i++) cur[i] = nxt[i];
            idx++;
        }
        layer_slot_pf<R, NR, K + 1>(mask, codes, mp, last, idx, cur, a);
    }
}

// PF: the prefetching forward form (the other kernels are at their register bound)
template <typename R, int NR, bool REV, bool PF>
__device__ __forceinline__ void apply_layer(const FGate &g, const DEnt *le, const R *smat, typename CT<R>::T *a,
                                            typename CT<R>::T *b, const RedCtx<R> &rc)
{
    int idx = 0;
    if constexpr (!REV && PF) {
        R cur[8];
        const R *mp = smat + 8 * g.mat;
        load_unit<R>(mp, cur);
        layer_slot_pf<R, NR, 0>(g.a, g.perm, mp, g.b - 1, idx, cur, a);
    } else {
        R gv[NR];
        int gs[NR];
#pragma unroll
        for (int k = 0; k < NR; k++) {
            gv[k] = R(0);
            gs[k] = -1;
        }
        layer_slot_ent<R, NR, REV, 0>(g.a, le, idx, smat, a, b, gv, gs);
        if constexpr (REV) {
            // the layer's generator reads: NR independent warp reductions, interleaved
#pragma unroll
            for (int o = 16; o > 0; o >>= 1)
#pragma unroll
                for (int k = 0; k < NR; k++)
                    if (o < rc.lanes) gv[k] += __shfl_xor_sync(rc.lanemask, gv[k], o);
#pragma unroll
            for (int k = 0; k < NR; k++)
                if (gs[k] >= 0 && rc.lane == 0) rc.sgrad[(gs[k] - rc.slot_begin) * rc.nwarps + rc.warp] = gv[k];
        }
    }
}

// ----------------------------------------------------------------------- the kernel



// Tile <-> shared memory.  Every thread moves CNT 16-byte words (two complex64 or one
// complex128 amplitude each): tile_fetch issues all of its global loads into registers
// (so their latencies overlap with each other and with the gate staging), tile_put
// writes them to shared memory.  The block has exactly 2^t * size(T) / 16 / CNT threads.
//
// Word c of a thread starts at tile position l = A | B_c, A = AW * thread and B_c = AW * c *
// blockDim on disjoint bits.  Its global offset tilebase | hitab[l >> low] | (l & lowmask)
// and its swizzled slot are both linear over such a split (OR of disjoint deposits, XOR),
// so the thread part is computed once and the part of word c is a block-uniform value.
template <typename R>
struct TileAddr {
    int64_t g;  // global offset of the thread part (tilebase included)
    int s;      // swizzled slot of the thread part
};

// The swizzle only touches bits below 2B (SwzBits): slot(X ^ H) = swz(X) + H for H on bits
// >= 2B that X does not use, so such a part of an index is an address offset.
template <typename R>
__device__ __forceinline__ int swz_lo_mask() { return (1 << (2 * SwzBits<R>::B)) - 1; }

template <int THREADS>
__device__ __forceinline__ int tile_threads() { return THREADS ? THREADS : (int)blockDim.x; }

template <typename R, int THREADS>
__device__ __forceinline__ TileAddr<R> tile_addr(int low, int64_t tilebase, const int64_t *hitab)
{
    constexpr int AW = sizeof(typename CT<R>::T) == 8 ? 2 : 1;
    const int A = (int)threadIdx.x * AW;
    return TileAddr<R>{tilebase | hitab[A >> low] | (A & ((1 << low) - 1)), swz<R>(A)};
}

// Word c's part B = AW * c * threads: its global offset (B's deposit) and its slot split
// into swz(B's bits below 2B) (XORed with the thread part) and B's higher bits (added:
// the thread part A < AW * threads never holds them).
template <typename R, int THREADS>
__device__ __forceinline__ void tile_word(int c, int low, const int64_t *hitab, int64_t &g, int &slo, int &shi)
{
    constexpr int AW = sizeof(typename CT<R>::T) == 8 ? 2 : 1;
    const int B = c * tile_threads<THREADS>() * AW;
    g = c ? (hitab[B >> low] | (B & ((1 << low) - 1))) : 0;
    slo = swz<R>(B & swz_lo_mask<R>());
    shi = B & ~swz_lo_mask<R>();
}

template <typename R, int CNT, int THREADS = 0>
__device__ __forceinline__ void tile_fetch(const typename CT<R>::T *gmem, float4 (&w)[CNT], int low, int64_t tilebase,
                                           const int64_t *hitab)
{
    const TileAddr<R> ta = tile_addr<R, THREADS>(low, tilebase, hitab);
#pragma unroll
    for (int c = 0; c < CNT; c++) {
        int64_t g;
        int slo, shi;
        tile_word<R, THREADS>(c, low, hitab, g, slo, shi);
        w[c] = *reinterpret_cast<const float4 *>(gmem + (ta.g | g));
    }
}

template <typename R, int CNT, int THREADS = 0>
__device__ __forceinline__ void tile_put(typename CT<R>::T *sm, const float4 (&w)[CNT])
{
    constexpr int AW = sizeof(typename CT<R>::T) == 8 ? 2 : 1;
    const int sA = swz<R>((int)threadIdx.x * AW);
#pragma unroll
    for (int c = 0; c < CNT; c++) {
        const int B = c * tile_threads<THREADS>() * AW;
        const int l = (sA ^ swz<R>(B & swz_lo_mask<R>())) + (B & ~swz_lo_mask<R>());
        if constexpr (AW == 2) {  // l ^ 1 = slot of the odd amplitude (swz(1) = 1)
            float2 *s2 = reinterpret_cast<float2 *>(sm);
            s2[l] = make_float2(w[c].x, w[c].y);
            s2[l ^ 1] = make_float2(w[c].z, w[c].w);
        } else {
            reinterpret_cast<float4 *>(sm)[l] = w[c];
        }
    }
}

template <typename R, int CNT, int THREADS = 0>
__device__ __forceinline__ void tile_store(typename CT<R>::T *gmem, const typename CT<R>::T *sm, int low,
                                           int64_t tilebase, const int64_t *hitab)
{
    constexpr int AW = sizeof(typename CT<R>::T) == 8 ? 2 : 1;
    const TileAddr<R> ta = tile_addr<R, THREADS>(low, tilebase, hitab);
#pragma unroll
    for (int c = 0; c < CNT; c++) {
        int64_t g;
        int slo, shi;
        tile_word<R, THREADS>(c, low, hitab, g, slo, shi);
        const int l = (ta.s ^ slo) + shi;
        float4 w;
        if constexpr (AW == 2) {
            const float2 *s2 = reinterpret_cast<const float2 *>(sm);
            const float2 a = s2[l], b = s2[l ^ 1];
            w = make_float4(a.x, a.y, b.x, b.y);
        } else {
            w = reinterpret_cast<const float4 *>(sm)[l];
        }
        *reinterpret_cast<float4 *>(gmem + (ta.g | g)) = w;
    }
}

// Zeros to every amplitude of the tile (the words tile_store would write).
template <typename R, int CNT, int THREADS = 0>
__device__ __forceinline__ void tile_zero(typename CT<R>::T *gmem, int low, int64_t tilebase, const int64_t *hitab)
{
    const TileAddr<R> ta = tile_addr<R, THREADS>(low, tilebase, hitab);
#pragma unroll
    for (int c = 0; c < CNT; c++) {
        int64_t g;
        int slo, shi;
        tile_word<R, THREADS>(c, low, hitab, g, slo, shi);
        *reinterpret_cast<float4 *>(gmem + (ta.g | g)) = make_float4(0.f, 0.f, 0.f, 0.f);
    }
}

__host__ __device__ inline size_t align16(size_t x) { return (x + 15) & ~size_t(15); }

// Element e of matrix unit m: a record part, or the shear parameters of a rotation record
// (kUnitShear), computed from its FP64 entries c = m[0], s = m[4].
template <typename R>
__device__ __forceinline__ R unit_elem(const MatUnit &m, int e, const MatRec *__restrict__ recs)
{
    if (m.part != kUnitShear) return mat_of<R>(&recs[m.rec])[8 * m.part + e];
    if (e > 1) return R(0);
    const double c = recs[m.rec].d[0], s = recs[m.rec].d[4];
    if (e == 0) return (R)(c >= 0.0 ? -s / (1.0 + c) : s / (1.0 - c));
    return (R)(c >= 0.0 ? s : -s);
}

// Shared-memory layout and per-CTA state of one tile pass, built by tile_begin and used
// by the sub-runs (interpreted from the pass's records, or specialised code) and tile_end.
template <typename R, int NR, bool REV>
struct TileCtx {
    typedef typename CT<R>::T T;
    T *sphi, *spsi;
    int64_t *hitab;
    FGate *sgates;
    DEnt *sents;
    R *sconst;
    R *smat;
    int64_t tilebase;
    int t, low, n_slots, slot_begin;
    RedCtx<R> rc;
};

// Prologue of a tile pass: the tile's base offset and strided address table, the tile's
// global loads (issued first), the staging of the pass's gate records, diagonal entries
// and matrices, the tile into shared memory, and the tile-constant products of every
// phase block.  Ends with the block synchronised.  Returns false, with nothing staged,
// for a tile of a pass started from |0...0> (args.init) that is not tile 0: the tile's
// amplitudes are written as zeros and the CTA has nothing more to do.
// Geometry of a pass read from its descriptor at run time (the interpreter).  The
// specialised passes pass their own provider with kStatic = true and the pass's tile
// positions compiled in: tilebase(tile) deposits the tile index on the physical qubits
// outside the tile, hi(h) the high local bits h on the tile's qubits low..t-1.
struct RuntimeGeom {
    static constexpr bool kStatic = false;
    static constexpr int kThreads = 0;  // block size (0: read blockDim.x)
    __device__ static int64_t tilebase(int64_t) { return 0; }
    __device__ static int64_t hi(int) { return 0; }
};

template <typename R, int NR, bool REV, class Geom = RuntimeGeom>
__device__ __forceinline__ bool tile_begin(const typename CT<R>::T *__restrict__ phi,
                                           const typename CT<R>::T *__restrict__ psi, const FusedArgs &args,
                                           const int64_t tile, TileCtx<R, NR, REV> &c)
{
    typedef typename CT<R>::T T;
    extern __shared__ __align__(16) unsigned char smem[];
    const PassDesc &pdg = *args.pd;
    struct {
        int t, n, low, n_sub, sub_begin, slot_begin, n_slots, gate_begin, n_gates, ent_begin, n_ent,
            unit_begin, n_units, n_blocks;
    } pd = {pdg.t, pdg.n, pdg.low, pdg.n_sub, pdg.sub_begin, pdg.slot_begin, pdg.n_slots, pdg.gate_begin,
            pdg.n_gates, pdg.ent_begin, pdg.n_ent, pdg.unit_begin, pdg.n_units, pdg.n_blocks};
    const int t = pd.t, n = pd.n, low = pd.low;
    const int L = 1 << t;
    const int nhi = 1 << (t - low);
    const int lanes = blockDim.x < 32 ? blockDim.x : 32;
    const int nwarps = (blockDim.x + 31) >> 5, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const unsigned lanemask = lanes == 32 ? 0xffffffffu : ((1u << lanes) - 1u);

    unsigned char *p = smem;
    T *sphi = reinterpret_cast<T *>(p);
    p += align16((size_t)(REV ? 2 : 1) * L * sizeof(T));
    T *spsi = sphi + (REV ? L : 0);
    int64_t *hitab = reinterpret_cast<int64_t *>(p);
    p += align16(sizeof(int64_t) * nhi);
    R *sgrad = reinterpret_cast<R *>(p);
    if (REV) p += align16(sizeof(R) * (size_t)pd.n_slots * nwarps);
    FGate *sgates = reinterpret_cast<FGate *>(p);
    p += align16(sizeof(FGate) * (size_t)pd.n_gates);
    DEnt *sents = reinterpret_cast<DEnt *>(p);
    p += align16(sizeof(DEnt) * (size_t)pd.n_ent);
    R *sconst = reinterpret_cast<R *>(p);  // per phase block: tile-constant products (Phi, Psi)
    p += align16((size_t)4 * sizeof(R) * pd.n_blocks);
    R *smat = reinterpret_cast<R *>(p);

    int64_t tilebase = 0;
    if constexpr (Geom::kStatic) {
        tilebase = Geom::tilebase(tile);
        for (int h = threadIdx.x; h < nhi; h += blockDim.x) hitab[h] = Geom::hi(h);
    } else {
        // S as two 64-bit words: byte j = physical qubit of tile position j (j < t <= 16)
        const int4 sw = *reinterpret_cast<const int4 *>(pdg.S);
        const uint64_t s_lo = (uint64_t)(uint32_t)sw.x | ((uint64_t)(uint32_t)sw.y << 32);
        const uint64_t s_hi = (uint64_t)(uint32_t)sw.z | ((uint64_t)(uint32_t)sw.w << 32);
        uint64_t smask = 0;
#pragma unroll
        for (int j = 0; j < 16; j++)
            if (j < t) smask |= uint64_t(1) << (((j < 8 ? s_lo : s_hi) >> (8 * (j & 7))) & 0xff);
        // tile-index bit i -> i-th lowest physical qubit outside S (bit deposit, no loads)
        uint64_t rest = ~smask & (n >= 64 ? ~uint64_t(0) : ((uint64_t(1) << n) - 1));
        for (uint64_t x = (uint64_t)tile; rest; rest &= rest - 1, x >>= 1)
            if (x & 1) tilebase |= (int64_t)(rest & (~rest + 1));
        // hitab[h] = sum over bits i of h of 2^S[low + i]; h = threadIdx.x + c * blockDim:
        // the thread bits give one constant part, the bits of c a small second one
        const int sh = 8 * low;  // S shifted down by low bytes (low <= 6)
        const uint64_t p_lo = sh ? (s_lo >> sh) | (s_hi << (64 - sh)) : s_lo, p_hi = s_hi >> sh;
        const int tb = __ffs(blockDim.x) - 1;  // log2(threads)
        const int hb = t - low;                // bits of h
        int64_t o_t = 0;
#pragma unroll
        for (int i = 0; i < 15; i++)
            if (i < tb && i < hb && ((threadIdx.x >> i) & 1))
                o_t |= int64_t(1) << (((i < 8 ? p_lo : p_hi) >> (8 * (i & 7))) & 0xff);
        for (int c = 0, h = threadIdx.x; h < nhi; c++, h += blockDim.x) {
            int64_t o = o_t;
#pragma unroll
            for (int i = 0; i < 6; i++)  // bits of c (h >> tb), fewer than 2^6 entries per thread
                if (tb + i < hb && ((c >> i) & 1)) {
                    const int k = tb + i;
                    o |= int64_t(1) << (((k < 8 ? p_lo : p_hi) >> (8 * (k & 7))) & 0xff);
                }
            hitab[h] = o;
        }
    }
    if (REV)
        for (int i = threadIdx.x; i < pd.n_slots * nwarps; i += blockDim.x) sgrad[i] = R(0);
    __syncthreads();
    // words of 16 bytes per thread: 2^t amplitudes over 2^(t - NR) threads
    constexpr int CNT = sizeof(T) == 8 ? (1 << (NR - 1)) : (1 << NR);
    float4 wphi[CNT], wpsi[REV ? CNT : 1];
    if (!REV && args.init) {
#pragma unroll
        for (int k = 0; k < CNT; k++) wphi[k] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (tile != 0) {  // uniform over the CTA; a prefetch launch runs tile 0 only
            tile_zero<R, CNT, Geom::kThreads>(const_cast<T *>(phi), low, tilebase, hitab);
            return false;
        }
        if (threadIdx.x == 0) *reinterpret_cast<T *>(&wphi[0]) = T{R(1), R(0)};  // local 0 = global 0
    } else {
        tile_fetch<R, CNT, Geom::kThreads>(phi, wphi, low, tilebase, hitab);
    }
    if constexpr (REV) tile_fetch<R, CNT, Geom::kThreads>(psi, wpsi, low, tilebase, hitab);
    // stage the pass's gates, diagonal entries and matrices while the tile loads are in flight
    {
        const int4 *src = reinterpret_cast<const int4 *>(args.gates + pd.gate_begin);
        int4 *dst = reinterpret_cast<int4 *>(sgates);
        for (int i = threadIdx.x; i < pd.n_gates * 2; i += blockDim.x) dst[i] = src[i];
        const int4 *esrc = reinterpret_cast<const int4 *>(args.ents + pd.ent_begin);
        int4 *edst = reinterpret_cast<int4 *>(sents);
        for (int i = threadIdx.x; i < pd.n_ent; i += blockDim.x) edst[i] = esrc[i];
        if (args.img) {  // contiguous copy of the pass's run of the matrix image
            const int4 *msrc = reinterpret_cast<const int4 *>(reinterpret_cast<const R *>(args.img) +
                                                              (size_t)8 * pd.unit_begin);
            int4 *mdst = reinterpret_cast<int4 *>(smat);
            const int words = pd.n_units * (int)(8 * sizeof(R) / 16);
            for (int i = threadIdx.x; i < words; i += blockDim.x) mdst[i] = msrc[i];
        } else {
            for (int i = threadIdx.x; i < pd.n_units * 8; i += blockDim.x) {
                const MatUnit u = args.units[pd.unit_begin + (i >> 3)];
                smat[i] = u.rec >= 0 ? unit_elem<R>(u, i & 7, args.recs) : R(0);
            }
        }
    }
    tile_put<R, CNT, Geom::kThreads>(sphi, wphi);
    if constexpr (REV) tile_put<R, CNT, Geom::kThreads>(spsi, wpsi);
    __syncthreads();
    // tile-constant phase products of every phase block (bits fixed by the tile index)
    for (int gi = threadIdx.x; gi < pd.n_gates; gi += blockDim.x) {
        const FGate g = sgates[gi];
        if (g.type != FT_DIAGB) continue;
        const DEnt *e = sents + g.ent + g.nz;
        R r0 = 1, i0 = 0, r1 = 1, i1 = 0;
        for (int i = 0; i < (g.perm & 255); i++, e++) {
            const int idx = e->k == 1 ? (int)((tilebase >> (-1 - e->ca)) & 1)
                                      : (int)((tilebase >> (-1 - e->ca)) & 1) | ((int)((tilebase >> (-1 - e->cb)) & 1) << 1);
            R er, ei;
            diag_elem<R>(smat + 8 * e->mat, e->k, idx, er, ei);
            cmul_inplace<R>(r0, i0, er, ei);
            diag_elem<R>(smat + 8 * e->mat2, e->k, idx, er, ei);
            cmul_inplace<R>(r1, i1, er, ei);
        }
        sconst[4 * g.slot] = r0;
        sconst[4 * g.slot + 1] = i0;
        sconst[4 * g.slot + 2] = r1;
        sconst[4 * g.slot + 3] = i1;
    }
    __syncthreads();
    c.sphi = sphi;
    c.spsi = spsi;
    c.hitab = hitab;
    c.sgates = sgates;
    c.sents = sents;
    c.sconst = sconst;
    c.smat = smat;
    c.tilebase = tilebase;
    c.t = t;
    c.low = low;
    c.n_slots = pd.n_slots;
    c.slot_begin = pd.slot_begin;
    c.rc = RedCtx<R>{sgrad, pd.slot_begin, nwarps, warp, lane, lanes, lanemask};
    return true;
}

// A sub-run's thread base position: tile positions Rp[0..NR-1] are the register bits,
// the thread index spells the other positions (below t) in ascending order.
template <int NR>
__device__ __forceinline__ int subrun_base(int t, const int (&Rp)[NR])
{
    int rmask = 0;
#pragma unroll
    for (int k = 0; k < NR; k++) rmask |= 1 << Rp[k];
    int base = 0;
    for (int q = 0, i = 0; q < t; q++) {
        if ((rmask >> q) & 1) continue;
        if ((threadIdx.x >> i) & 1) base |= 1 << q;
        i++;
    }
    return base;
}

// Gather the register amplitudes of the thread at base with register offsets off[k] =
// 1 << Rp[k].  base and the register offsets occupy disjoint bits, so base | C = base ^ C,
// and the swizzle is linear over XOR: slot(base | C_j) = swz(base) ^ swz(C_j) with swz(C_j)
// a constant of the sub-run (a literal in the specialised passes).
template <typename R, int NR, bool REV>
__device__ __forceinline__ void subrun_gather(const TileCtx<R, NR, REV> &c, int base, const int (&off)[NR],
                                              typename CT<R>::T *a, typename CT<R>::T *b)
{
    const int sb = swz<R>(base);
#pragma unroll
    for (int j = 0; j < (1 << NR); j++) {
        int cj = 0;
#pragma unroll
        for (int k = 0; k < NR; k++)
            if ((j >> k) & 1) cj |= off[k];
        // register bits at or above 2B are an offset (base never holds them)
        const int l = (sb ^ swz<R>(cj & swz_lo_mask<R>())) + (cj & ~swz_lo_mask<R>());
        a[j] = c.sphi[l];
        if constexpr (REV) b[j] = c.spsi[l];
    }
}

// Base position, register offsets and gather of a sub-run (returns the base).
template <typename R, int NR, bool REV>
__device__ __forceinline__ int subrun_load(const TileCtx<R, NR, REV> &c, const int (&Rp)[NR], int (&off)[NR],
                                           typename CT<R>::T *a, typename CT<R>::T *b)
{
#pragma unroll
    for (int k = 0; k < NR; k++) off[k] = 1 << Rp[k];
    const int base = subrun_base<NR>(c.t, Rp);
    subrun_gather<R, NR, REV>(c, base, off, a, b);
    return base;
}

// Scatter the register amplitudes back and synchronise the block.
template <typename R, int NR, bool REV>
__device__ __forceinline__ void subrun_store(const TileCtx<R, NR, REV> &c, int base, const int (&off)[NR],
                                             const typename CT<R>::T *a, const typename CT<R>::T *b)
{
    const int sb = swz<R>(base);  // as in subrun_gather
#pragma unroll
    for (int j = 0; j < (1 << NR); j++) {
        int cj = 0;
#pragma unroll
        for (int k = 0; k < NR; k++)
            if ((j >> k) & 1) cj |= off[k];
        const int l = (sb ^ swz<R>(cj & swz_lo_mask<R>())) + (cj & ~swz_lo_mask<R>());
        c.sphi[l] = a[j];
        if constexpr (REV) c.spsi[l] = b[j];
    }
    __syncthreads();
}

// Z-generator reads of a phase block (reverse): per register bit k the sum of
// Im(conj(Psi) Phi) with sign (-1)^(bit k), and the total.  A halving tree: level k
// holds the sums of v over the lowest k bits, and dk[k] is the alternating sum of level
// k's entries (2^(NR+1) + 2^NR - NR - 3 adds instead of (NR + 1) 2^NR).
template <typename R, int NR>
__device__ __forceinline__ void z_sums(const typename CT<R>::T *a, const typename CT<R>::T *b, R &tot, R (&dk)[NR])
{
    R s[1 << NR];
#pragma unroll
    for (int j = 0; j < (1 << NR); j++) s[j] = b[j].x * a[j].y - b[j].y * a[j].x;  // Im(conj(Psi) Phi)
#pragma unroll
    for (int k = 0; k < NR; k++) {
        const int m = 1 << (NR - k - 1);  // pairs at this level
        R d = s[0] - s[1];
#pragma unroll
        for (int i = 1; i < m; i++) d += s[2 * i] - s[2 * i + 1];
        dk[k] = d;
#pragma unroll
        for (int i = 0; i < m; i++) s[i] = s[2 * i] + s[2 * i + 1];
    }
    tot = s[0];
}

// The record interpreter: gates [g_begin, g_end) of the pass on the register amplitudes.
template <typename R, int NR, bool REV, bool TWOQ>
__device__ __forceinline__ void run_records(const TileCtx<R, NR, REV> &c, int g_begin, int g_end, int base,
                                            typename CT<R>::T *a, typename CT<R>::T *b)
{
    const FGate *sgates = c.sgates;
    const DEnt *sents = c.sents;
    const R *smat = c.smat;
    const int64_t tilebase = c.tilebase;
    const RedCtx<R> &rc = c.rc;
    FGate gn = sgates[g_begin < g_end ? g_begin : 0];
    for (int gi = g_begin; gi < g_end; gi++) {
        const FGate g = gn;
        if (gi + 1 < g_end) gn = sgates[gi + 1];  // prefetch the next record
        if (g.type == FT_LAYER1) {
            apply_layer<R, NR, REV, !TWOQ>(g, sents + g.ent, smat, a, b, rc);
            continue;
        }
        if (g.type == FT_DIAGB) {
            const DEnt *ents = sents + g.ent;
            const R *cst = c.sconst + 4 * g.slot;
            if constexpr (REV) {
                if (g.nz > 0) {  // Z generators on the states after the block
                    R tot, dk[NR];
                    z_sums<R, NR>(a, b, tot, dk);
                    for (int e = 0; e < g.nz; e++) {
                        const DEnt d = ents[e];
                        R part;
                        if (d.ca >= 0 && d.ca < NR) {
                            part = dk[0];
#pragma unroll
                            for (int k = 1; k < NR; k++)
                                if (k == d.ca) part = dk[k];
                        } else {
                            part = const_bit<NR>(d.ca, base, tilebase) ? -tot : tot;
                        }
                        emit_partial<R>(rc, d.slot, part * (R)d.coef);
                    }
                }
                if (g.flags & FLAG_TABLE) {
                    if (g.flags & FLAG_SEPARATE) {
                        phase_table<R, NR>(ents + g.nz, g.perm, smat, g.mat, false, cst[0], cst[1], a, nullptr, base, tilebase);
                        phase_table<R, NR>(ents + g.nz, g.perm, smat, g.mat2, true, cst[2], cst[3], b, nullptr, base, tilebase);
                    } else {
                        phase_table<R, NR>(ents + g.nz, g.perm, smat, g.mat, false, cst[0], cst[1], a, b, base, tilebase);
                    }
                } else if (g.flags & FLAG_SEPARATE) {
                    phase_block<R, NR>(ents + g.nz, g.perm, smat, false, cst[0], cst[1], a, nullptr, base, tilebase);
                    phase_block<R, NR>(ents + g.nz, g.perm, smat, true, cst[2], cst[3], b, nullptr, base, tilebase);
                } else {
                    phase_block<R, NR>(ents + g.nz, g.perm, smat, false, cst[0], cst[1], a, b, base, tilebase);
                }
            } else if (g.flags & FLAG_TABLE) {
                phase_table<R, NR>(ents, g.perm, smat, g.mat, false, cst[0], cst[1], a, nullptr, base, tilebase);
            } else {
                phase_block<R, NR>(ents, g.perm, smat, false, cst[0], cst[1], a, nullptr, base, tilebase);
            }
            continue;
        }
        if constexpr (REV && TWOQ) {
            if (g.type == FT_PROBE2) {  // gradient read only: the states stay as they are
                emit_partial<R>(rc, g.slot, probe2_dispatch<R, NR>(g.a, g.b, a, b, smat + 8 * g.mat) * (R)g.coef);
                continue;
            }
        }
        if constexpr (REV) {
            if (g.gen == GEN_X)
                emit_partial<R>(rc, g.slot, gen_xy_dispatch<R, NR, GEN_X>(g.gpos, a, b) * (R)g.coef);
            else if (g.gen == GEN_Y)
                emit_partial<R>(rc, g.slot, gen_xy_dispatch<R, NR, GEN_Y>(g.gpos, a, b) * (R)g.coef);
        }
        apply_fgate<R, NR, TWOQ>(g.type, g.a, g.b, g.perm, smat + 8 * g.mat, a);
        if constexpr (REV) apply_fgate<R, NR, TWOQ>(g.type, g.a, g.b, g.perm, smat + 8 * g.mat2, b);
    }
}

// Epilogue: the tile back to global memory and (reverse) the tile's FP64 partial of every
// gradient slot of the pass, summed over the warps in fixed order.
template <typename R, int NR, bool REV, class Geom = RuntimeGeom>
__device__ __forceinline__ void tile_end(typename CT<R>::T *__restrict__ phi, typename CT<R>::T *__restrict__ psi,
                                         const FusedArgs &args, const int64_t tile, const TileCtx<R, NR, REV> &c)
{
    typedef typename CT<R>::T T;
    constexpr int CNT = sizeof(T) == 8 ? (1 << (NR - 1)) : (1 << NR);
    if (args.dry) return;  // a code-prefetch launch writes nothing
    tile_store<R, CNT, Geom::kThreads>(phi, c.sphi, c.low, c.tilebase, c.hitab);
    if (REV) {
        tile_store<R, CNT, Geom::kThreads>(psi, c.spsi, c.low, c.tilebase, c.hitab);
        const int nwarps = c.rc.nwarps;
        for (int sl = threadIdx.x; sl < c.n_slots; sl += blockDim.x) {
            double acc = 0.0;
            for (int w = 0; w < nwarps; w++) acc += (double)c.rc.sgrad[sl * nwarps + w];
            args.slot_partials[(int64_t)(c.slot_begin + sl) * args.tiles_stride + tile] = acc;
        }
    }
}

// One tile of one pass: the body shared by the single-circuit kernel (tile = CTA index)
// and the batched kernel (tile looked up from the CTA index).
template <typename R, int NR, bool REV, bool TWOQ>
__device__ __forceinline__ void fused_tile(typename CT<R>::T *__restrict__ phi, typename CT<R>::T *__restrict__ psi,
                                           const FusedArgs &args, const int64_t tile)
{
    typedef typename CT<R>::T T;
    TileCtx<R, NR, REV> c;
    if (!tile_begin<R, NR, REV>(phi, psi, args, tile, c)) return;
    const int n_sub = args.pd->n_sub, sub_begin = args.pd->sub_begin;
    T a[1 << NR], b[REV ? (1 << NR) : 1];
    for (int s = 0; s < n_sub; s++) {
        const SubRun sr = args.subs[sub_begin + s];
        int Rp[NR], off[NR];
#pragma unroll
        for (int k = 0; k < NR; k++) Rp[k] = sr.R[k];
        const int base = subrun_load<R, NR, REV>(c, Rp, off, a, b);
        run_records<R, NR, REV, TWOQ>(c, sr.g_begin, sr.g_end, base, a, b);
        subrun_store<R, NR, REV>(c, base, off, a, b);
    }
    tile_end<R, NR, REV>(phi, psi, args, tile, c);
}

}  // namespace gbvqc
