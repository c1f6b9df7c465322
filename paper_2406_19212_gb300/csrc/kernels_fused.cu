// Fused tile passes: one HBM read and one write of the state apply a whole run of gates.
//
// A pass names a set S of t "tile" qubits (the lowest `low` qubits are always in S, so
// every tile is made of contiguous 2^low-amplitude segments).  CTA i owns the 2^t
// amplitudes whose non-tile bits spell i, stages them in shared memory, applies the
// pass's gates and writes them back.  Inside the tile, gates run in "sub-runs": each
// sub-run names NR tile positions that every thread gathers into registers (2^NR
// amplitudes per thread), applies all of the sub-run's gates on them with no further
// memory traffic, and scatters back.  Diagonal gates need no register position and
// ride along in any sub-run, including diagonal gates on non-tile qubits.
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
// with Q^dag.  Per-thread FP32 partials over 2^NR terms are reduced across the warp in
// FP64 with shuffles and across warps in fixed order, giving one FP64 partial per
// (gradient slot, tile).
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
                R mr = c == 0 ? m[8 * r] : c == 1 ? m[8 * r + 2] : c == 2 ? m[8 * r + 4] : m[8 * r + 6];
                R mi = c == 0 ? m[8 * r + 1] : c == 1 ? m[8 * r + 3] : c == 2 ? m[8 * r + 5] : m[8 * r + 7];
                w[r] = cmul<T, R>(mr, mi, x);
            }
        }
        a[j] = w[0];
        a[i1] = w[1];
        a[i2] = w[2];
        a[i3] = w[3];
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

// Bit of a position code for register amplitude j (j compile-time after unrolling).
template <int NR>
__device__ __forceinline__ int code_bit(int code, int j, int base, int64_t tilebase)
{
    if (code < 0) return (int)((tilebase >> (-1 - code)) & 1);
    if (code >= NR) return (base >> (code - NR)) & 1;
    return (j >> code) & 1;
}

// Diagonal one-qubit gate on a position code.
template <typename R, int NR>
__device__ __forceinline__ void dg1(typename CT<R>::T *a, const R *m, int code, int base,
                                    int64_t tilebase)
{
    typedef typename CT<R>::T T;
    if (code >= 0 && code < NR) {
        rg1_dispatch<R, NR, SH_DIAG1>(code, a, m);
        return;
    }
    const int bit = code_bit<NR>(code, 0, base, tilebase);
    const R pr = bit ? m[6] : m[0], pi = bit ? m[7] : m[1];
#pragma unroll
    for (int j = 0; j < (1 << NR); j++) a[j] = cmul<T, R>(pr, pi, a[j]);
}

// Diagonal two-qubit gate on two position codes (matrix bit 0 = code ca).
template <typename R, int NR>
__device__ __forceinline__ void dg2(typename CT<R>::T *a, const R *m, int ca, int cb, int base,
                                    int64_t tilebase)
{
    typedef typename CT<R>::T T;
    const R p0r = m[0], p0i = m[1], p1r = m[10], p1i = m[11];
    const R p2r = m[20], p2i = m[21], p3r = m[30], p3i = m[31];
#pragma unroll
    for (int j = 0; j < (1 << NR); j++) {
        const int idx = code_bit<NR>(ca, j, base, tilebase) | (code_bit<NR>(cb, j, base, tilebase) << 1);
        const R pr = idx == 0 ? p0r : idx == 1 ? p1r : idx == 2 ? p2r : p3r;
        const R pi = idx == 0 ? p0i : idx == 1 ? p1i : idx == 2 ? p2i : p3i;
        a[j] = cmul<T, R>(pr, pi, a[j]);
    }
}

template <typename R, int NR>
__device__ __forceinline__ void apply_fgate(const FGate &g, const R *m, typename CT<R>::T *a,
                                            int base, int64_t tilebase)
{
    switch (g.type) {
    case FT_DENSE1: rg1_dispatch<R, NR, SH_DENSE1>(g.a, a, m); break;
    case FT_REAL1: rg1_dispatch<R, NR, SH_REAL1>(g.a, a, m); break;
    case FT_ANTI1: rg1_dispatch<R, NR, SH_ANTI1>(g.a, a, m); break;
    case FT_DIAG1: dg1<R, NR>(a, m, g.a, base, tilebase); break;
    case FT_DENSE2: rg2_dispatch<R, NR, SH_DENSE2>(g.a, g.b, a, m, 0); break;
    case FT_DIAG2: dg2<R, NR>(a, m, g.a, g.b, base, tilebase); break;
    case FT_PERM2: rg2_dispatch<R, NR, SH_PERM2>(g.a, g.b, a, m, g.perm); break;
    default: rg2_dispatch<R, NR, SH_CTRL2>(g.a, g.b, a, m, 0); break;
    }
}

// ------------------------------------------------------------ generator inner products

// Im <Psi| P_K |Phi> over the thread's register amplitudes, P = X or Y on slot K.
template <typename R, int NR, int K, int G>
__device__ __forceinline__ R gen_xy(const typename CT<R>::T *f, const typename CT<R>::T *p)
{
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

// Im <Psi| Z |Phi> with the Z bit given by a position code.
template <typename R, int NR>
__device__ __forceinline__ R gen_z(int code, const typename CT<R>::T *f, const typename CT<R>::T *p,
                                   int base, int64_t tilebase)
{
    R s = 0;
#pragma unroll
    for (int j = 0; j < (1 << NR); j++) {
        const R v = p[j].x * f[j].y - p[j].y * f[j].x;
        s += code_bit<NR>(code, j, base, tilebase) ? -v : v;
    }
    return s;
}

// ----------------------------------------------------------------------- the kernel

struct FusedArgs {
    const PassDesc *pd;
    const SubRun *subs;
    const FGate *gates;
    const MatRec *recs;
    double *slot_partials;
    int tiles_stride;
};

template <typename R>
__device__ __forceinline__ void tile_io(typename CT<R>::T *gmem, typename CT<R>::T *sm, int t, int low,
                                        int64_t tilebase, const int64_t *hitab, bool load)
{
    typedef typename CT<R>::T T;
    const int L = 1 << t, lowmask = (1 << low) - 1;
    if (sizeof(T) == 8) {  // complex64: two amplitudes per 16-byte access
        for (int v = threadIdx.x; v < (L >> 1); v += blockDim.x) {
            const int l = v << 1;
            const int64_t g = tilebase | hitab[l >> low] | (l & lowmask);
            float4 *p = reinterpret_cast<float4 *>(gmem + g);
            float2 *s = reinterpret_cast<float2 *>(sm);
            if (load) {
                float4 x = *p;
                s[swz<R>(l)] = make_float2(x.x, x.y);
                s[swz<R>(l + 1)] = make_float2(x.z, x.w);
            } else {
                float2 a = s[swz<R>(l)], b = s[swz<R>(l + 1)];
                *p = make_float4(a.x, a.y, b.x, b.y);
            }
        }
    } else {
        for (int l = threadIdx.x; l < L; l += blockDim.x) {
            const int64_t g = tilebase | hitab[l >> low] | (l & lowmask);
            if (load) sm[swz<R>(l)] = gmem[g];
            else gmem[g] = sm[swz<R>(l)];
        }
    }
}

template <typename R, int NR, bool REV>
__global__ void __launch_bounds__(256) k_fused(typename CT<R>::T *__restrict__ phi,
                                               typename CT<R>::T *__restrict__ psi, FusedArgs args)
{
    typedef typename CT<R>::T T;
    extern __shared__ __align__(16) unsigned char smem[];
    const PassDesc &pd = *args.pd;
    const int t = pd.t, n = pd.n, low = pd.low;
    const int L = 1 << t;
    T *sphi = reinterpret_cast<T *>(smem);
    T *spsi = sphi + (REV ? L : 0);
    int64_t *hitab = reinterpret_cast<int64_t *>(smem + (REV ? 2 : 1) * (size_t)L * sizeof(T));
    const int nhi = 1 << (t - low);
    double *sgrad = reinterpret_cast<double *>(hitab + nhi);
    const int lanes = blockDim.x < 32 ? blockDim.x : 32;
    const int nwarps = (blockDim.x + 31) >> 5, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const unsigned lanemask = lanes == 32 ? 0xffffffffu : ((1u << lanes) - 1u);

    const int64_t tile = blockIdx.x;
    int64_t tilebase = 0;
    for (int i = 0; i < n - t; i++)
        if ((tile >> i) & 1) tilebase |= int64_t(1) << pd.NS[i];
    for (int h = threadIdx.x; h < nhi; h += blockDim.x) {
        int64_t o = 0;
        for (int i = 0; i < t - low; i++)
            if ((h >> i) & 1) o |= int64_t(1) << pd.S[low + i];
        hitab[h] = o;
    }
    if (REV)
        for (int i = threadIdx.x; i < pd.n_slots * nwarps; i += blockDim.x) sgrad[i] = 0.0;
    __syncthreads();
    tile_io<R>(phi, sphi, t, low, tilebase, hitab, true);
    if (REV) tile_io<R>(psi, spsi, t, low, tilebase, hitab, true);
    __syncthreads();

    T a[1 << NR], b[REV ? (1 << NR) : 1];
    for (int s = 0; s < pd.n_sub; s++) {
        const SubRun sr = args.subs[pd.sub_begin + s];
        // thread bits -> tile positions outside R, ascending
        int rmask = 0;
#pragma unroll
        for (int k = 0; k < NR; k++) rmask |= 1 << sr.R[k];
        int base = 0;
        for (int p = 0, i = 0; p < t; p++) {
            if ((rmask >> p) & 1) continue;
            if ((threadIdx.x >> i) & 1) base |= 1 << p;
            i++;
        }
        int off[NR];
#pragma unroll
        for (int k = 0; k < NR; k++) off[k] = 1 << sr.R[k];
#pragma unroll
        for (int j = 0; j < (1 << NR); j++) {
            int l = base;
#pragma unroll
            for (int k = 0; k < NR; k++)
                if ((j >> k) & 1) l |= off[k];
            a[j] = sphi[swz<R>(l)];
            if constexpr (REV) b[j] = spsi[swz<R>(l)];
        }
        for (int gi = sr.g_begin; gi < sr.g_end; gi++) {
            const FGate g = args.gates[gi];
            if constexpr (REV) {
                if (g.gen != GEN_NONE) {
                R part;
                if (g.gen == GEN_Z) part = gen_z<R, NR>(g.gpos, a, b, base, tilebase);
                else if (g.gen == GEN_X) part = gen_xy_dispatch<R, NR, GEN_X>(g.gpos, a, b);
                else part = gen_xy_dispatch<R, NR, GEN_Y>(g.gpos, a, b);
                double v = (double)part * (double)g.coef;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1)
                    if (o < lanes) v += __shfl_xor_sync(lanemask, v, o);
                if (lane == 0) sgrad[(g.slot - pd.slot_begin) * nwarps + warp] = v;
                }
            }
            apply_fgate<R, NR>(g, mat_of<R>(&args.recs[g.rec]), a, base, tilebase);
            if constexpr (REV) apply_fgate<R, NR>(g, mat_of<R>(&args.recs[g.rec2]), b, base, tilebase);
        }
#pragma unroll
        for (int j = 0; j < (1 << NR); j++) {
            int l = base;
#pragma unroll
            for (int k = 0; k < NR; k++)
                if ((j >> k) & 1) l |= off[k];
            sphi[swz<R>(l)] = a[j];
            if constexpr (REV) spsi[swz<R>(l)] = b[j];
        }
        __syncthreads();
    }
    tile_io<R>(phi, sphi, t, low, tilebase, hitab, false);
    if (REV) {
        tile_io<R>(psi, spsi, t, low, tilebase, hitab, false);
        for (int sl = threadIdx.x; sl < pd.n_slots; sl += blockDim.x) {
            double acc = 0.0;
            for (int w = 0; w < nwarps; w++) acc += sgrad[sl * nwarps + w];
            args.slot_partials[(int64_t)(pd.slot_begin + sl) * args.tiles_stride + tile] = acc;
        }
    }
}

// -------------------------------------------------------------------------- launchers

int fused_nr(int dtype, bool reverse)
{
    if (dtype == 0) return reverse ? 4 : 5;
    return reverse ? 3 : 4;
}

size_t fused_smem_bytes(int dtype, int t, bool reverse, int max_slots)
{
    const int nr = fused_nr(dtype, reverse);
    const size_t amp = dtype == 0 ? 8 : 16;
    const int threads = 1 << (t - nr);
    const int nwarps = (threads + 31) / 32;
    size_t b = (reverse ? 2 : 1) * (size_t(1) << t) * amp;
    b += sizeof(int64_t) * (size_t(1) << t);  // upper bound of the hi table
    if (reverse) b += sizeof(double) * (size_t)max_slots * nwarps;
    return b;
}

template <typename R, int NR, bool REV>
static cudaError_t fused_launch(void *phi, void *psi, const PassDesc &ph, FusedArgs args, cudaStream_t s)
{
    typedef typename CT<R>::T T;
    const int threads = 1 << (ph.t - NR);
    const int64_t tiles = int64_t(1) << (ph.n - ph.t);
    const int nwarps = (threads + 31) / 32;
    size_t smem = (REV ? 2 : 1) * (size_t(1) << ph.t) * sizeof(T) +
                  sizeof(int64_t) * (size_t(1) << (ph.t - ph.low)) +
                  (REV ? sizeof(double) * (size_t)ph.n_slots * nwarps : 0);
    k_fused<R, NR, REV><<<(unsigned)tiles, threads, smem, s>>>((T *)phi, (T *)psi, args);
    return cudaGetLastError();
}

// Opt the fused kernels in to large dynamic shared memory (call outside stream capture).
cudaError_t fused_prepare()
{
    const int bytes = 200 * 1024;
    cudaError_t e = cudaFuncSetAttribute(k_fused<float, 5, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_fused<float, 4, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_fused<double, 4, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_fused<double, 3, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    return e;
}

cudaError_t launch_fused_forward(int dtype, void *psi, const PassDesc *pass_dev, const PassDesc &ph,
                                 const SubRun *subs, const FGate *gates, const MatRec *recs,
                                 cudaStream_t s)
{
    FusedArgs args{pass_dev, subs, gates, recs, nullptr, 0};
    if (dtype == 0) return fused_launch<float, 5, false>(psi, nullptr, ph, args, s);
    return fused_launch<double, 4, false>(psi, nullptr, ph, args, s);
}

cudaError_t launch_fused_reverse(int dtype, void *phi, void *psi, const PassDesc *pass_dev,
                                 const PassDesc &ph, const SubRun *subs, const FGate *gates,
                                 const MatRec *recs, double *slot_partials, int n_tiles_stride,
                                 cudaStream_t s)
{
    FusedArgs args{pass_dev, subs, gates, recs, slot_partials, n_tiles_stride};
    if (dtype == 0) return fused_launch<float, 4, true>(phi, psi, ph, args, s);
    return fused_launch<double, 3, true>(phi, psi, ph, args, s);
}

// slot_grad[s] = sum over tiles, in tile order within each thread, then a fixed tree.
__global__ void k_reduce_slots(const double *__restrict__ part, int n_tiles, int stride, double *out)
{
    __shared__ double sh[256];
    const int s = blockIdx.x;
    double acc = 0.0;
    for (int i = threadIdx.x; i < n_tiles; i += blockDim.x) acc += part[(int64_t)s * stride + i];
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[s] = sh[0];
}

cudaError_t launch_reduce_slots(const double *slot_partials, int n_slots, int n_tiles, int stride,
                                double *slot_grad, cudaStream_t s)
{
    if (n_slots == 0) return cudaSuccess;
    k_reduce_slots<<<n_slots, 256, 0, s>>>(slot_partials, n_tiles, stride, slot_grad);
    return cudaGetLastError();
}

}  // namespace gbvqc
