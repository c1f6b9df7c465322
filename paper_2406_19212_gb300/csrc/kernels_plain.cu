// Per-gate kernels: one launch applies one gate to the whole state (Eq. 3 and
// Eq. twoqubitgate of the paper; Algorithm 1 with the three outer loops flattened into
// one grid-stride index).  Each thread owns one amplitude pair (one-qubit gate) or
// quadruple (two-qubit gate): the groups touch disjoint amplitudes, which is the
// paper's non-overlapping-segment parallelisation (Sec. III.B, Fig. 4) mapped to a
// CUDA grid.  Specialised bodies for diagonal, anti-diagonal, real, permutation and
// controlled matrices (Sec. II.B).
#include "devmath.cuh"
#include "kernels.h"

namespace gbvqc {

__device__ __forceinline__ int64_t insert_zero(int64_t g, int q)
{
    int64_t low = g & ((int64_t(1) << q) - 1);
    return ((g >> q) << (q + 1)) | low;
}

static inline int grid_for(int64_t items, int threads)
{
    int64_t b = (items + threads - 1) / threads;
    const int64_t cap = 152 * 16;
    if (b > cap) b = cap;
    if (b < 1) b = 1;
    return (int)b;
}

// ------------------------------------------------------------------ one-qubit gates

template <typename R, int SH>
__global__ void __launch_bounds__(256) k_gate1(typename CT<R>::T *__restrict__ psi, int64_t npairs,
                                               int q, const MatRec *__restrict__ rec)
{
    typedef typename CT<R>::T T;
    R m[8];
    const R *src = mat_of<R>(rec);
#pragma unroll
    for (int i = 0; i < 8; i++) m[i] = src[i];
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < npairs; g += stride) {
        int64_t i0 = insert_zero(g, q), i1 = i0 | (int64_t(1) << q);
        T a = psi[i0], b = psi[i1];
        apply2<R, SH>(m, a, b);
        psi[i0] = a;
        psi[i1] = b;
    }
}

// Gate on qubit 0 of a complex64 state: both amplitudes of a pair in one 16-byte load.
template <int SH>
__global__ void __launch_bounds__(256) k_gate1_q0_c64(float4 *__restrict__ psi, int64_t npairs,
                                                      const MatRec *__restrict__ rec)
{
    float m[8];
#pragma unroll
    for (int i = 0; i < 8; i++) m[i] = rec->f[i];
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < npairs; g += stride) {
        float4 v = psi[g];
        float2 a = make_float2(v.x, v.y), b = make_float2(v.z, v.w);
        apply2<float, SH>(m, a, b);
        psi[g] = make_float4(a.x, a.y, b.x, b.y);
    }
}

// ------------------------------------------------------------------ two-qubit gates

template <typename R, int SH>
__global__ void __launch_bounds__(256) k_gate2(typename CT<R>::T *__restrict__ psi, int64_t nquads,
                                               int q0, int q1, const MatRec *__restrict__ rec)
{
    typedef typename CT<R>::T T;
    const R *src = mat_of<R>(rec);
    R m[32];
#pragma unroll
    for (int i = 0; i < 32; i++) m[i] = src[i];
    int col[4];
    if (SH == SH_PERM2) {
#pragma unroll
        for (int r = 0; r < 4; r++) {
            col[r] = 0;
#pragma unroll
            for (int c = 0; c < 4; c++)
                if (m[2 * (4 * r + c)] != R(0) || m[2 * (4 * r + c) + 1] != R(0)) col[r] = c;
        }
    }
    const int lo = q0 < q1 ? q0 : q1, hi = q0 < q1 ? q1 : q0;
    const int64_t b0 = int64_t(1) << q0, b1 = int64_t(1) << q1;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < nquads; g += stride) {
        int64_t base = insert_zero(insert_zero(g, lo), hi);
        if (SH == SH_CTRL2) {  // control = q0 must be 1; 2x2 block on q1
            int64_t i0 = base | b0, i1 = base | b0 | b1;
            T a = psi[i0], b = psi[i1];
            R u[8] = {m[2 * 5], m[2 * 5 + 1], m[2 * 7], m[2 * 7 + 1],
                      m[2 * 13], m[2 * 13 + 1], m[2 * 15], m[2 * 15 + 1]};
            apply2<R, SH_DENSE1>(u, a, b);
            psi[i0] = a;
            psi[i1] = b;
            continue;
        }
        if (SH == SH_BLOCK2) {  // phases on |00>, |11>; 2x2 on |01>, |10>
            const int64_t i1 = base | b0, i2 = base | b1, i3 = base | b0 | b1;
            T a = psi[i1], b = psi[i2], c = psi[base], d = psi[i3];
            R u[8] = GBVQC_BLOCK2_U(m);
            apply2<R, SH_DENSE1>(u, a, b);
            cmul_ip<T, R>(m[0], m[1], c);
            cmul_ip<T, R>(m[30], m[31], d);
            psi[i1] = a;
            psi[i2] = b;
            psi[base] = c;
            psi[i3] = d;
            continue;
        }
        if (SH == SH_CX) {  // CNOT: the two amplitudes with the control set trade places
            const int64_t i1 = base | b0, i3 = base | b0 | b1;
            const T t = psi[i1];
            psi[i1] = psi[i3];
            psi[i3] = t;
            continue;
        }
        if (SH == SH_CZ) {  // CZ: the |11> amplitude changes sign
            const int64_t i3 = base | b0 | b1;
            T t = psi[i3];
            t.x = -t.x;
            t.y = -t.y;
            psi[i3] = t;
            continue;
        }
        if (SH == SH_PAR2 || SH == SH_RPAR2) {  // 2x2 on |00>, |11>; 2x2 on |01>, |10>
            const int64_t i1 = base | b0, i2 = base | b1, i3 = base | b0 | b1;
            T a = psi[base], d = psi[i3], b = psi[i1], c = psi[i2];
            R o[8] = GBVQC_OUTER_U(m), u[8] = GBVQC_BLOCK2_U(m);
            apply2<R, SH == SH_PAR2 ? SH_DENSE1 : SH_REAL1>(o, a, d);
            apply2<R, SH == SH_PAR2 ? SH_DENSE1 : SH_REAL1>(u, b, c);
            psi[base] = a;
            psi[i1] = b;
            psi[i2] = c;
            psi[i3] = d;
            continue;
        }
        int64_t idx[4] = {base, base | b0, base | b1, base | b0 | b1};
        T v[4], w[4];
#pragma unroll
        for (int l = 0; l < 4; l++) v[l] = psi[idx[l]];
        if (SH == SH_DENSE2) {
#pragma unroll
            for (int r = 0; r < 4; r++) {
                T acc = cmul<T, R>(m[8 * r], m[8 * r + 1], v[0]);
#pragma unroll
                for (int c = 1; c < 4; c++) cfma<T, R>(m[8 * r + 2 * c], m[8 * r + 2 * c + 1], v[c], acc);
                w[r] = acc;
            }
        } else if (SH == SH_DIAG2) {
#pragma unroll
            for (int r = 0; r < 4; r++) w[r] = cmul<T, R>(m[10 * r], m[10 * r + 1], v[r]);
        } else {  // SH_PERM2
#pragma unroll
            for (int r = 0; r < 4; r++) {
                T x = v[0];
#pragma unroll
                for (int c = 1; c < 4; c++)
                    if (col[r] == c) x = v[c];
                w[r] = cmul<T, R>(m[8 * r + 2 * col[r]], m[8 * r + 2 * col[r] + 1], x);
            }
        }
#pragma unroll
        for (int l = 0; l < 4; l++) psi[idx[l]] = w[l];
    }
}

template <typename R>
static cudaError_t gate_dispatch(void *psi_, int n, int shape, int q0, int q1, const MatRec *rec,
                                 cudaStream_t s)
{
    typedef typename CT<R>::T T;
    T *psi = (T *)psi_;
    const int th = 256;
    if (shape_qubits(shape) == 1) {
        int64_t np = int64_t(1) << (n - 1);
        int gr = grid_for(np, th);
        switch (shape) {
        case SH_DENSE1: k_gate1<R, SH_DENSE1><<<gr, th, 0, s>>>(psi, np, q0, rec); break;
        case SH_DIAG1: k_gate1<R, SH_DIAG1><<<gr, th, 0, s>>>(psi, np, q0, rec); break;
        case SH_ANTI1: k_gate1<R, SH_ANTI1><<<gr, th, 0, s>>>(psi, np, q0, rec); break;
        case SH_IMAG1: k_gate1<R, SH_IMAG1><<<gr, th, 0, s>>>(psi, np, q0, rec); break;
        default: k_gate1<R, SH_REAL1><<<gr, th, 0, s>>>(psi, np, q0, rec); break;
        }
    } else {
        int64_t nq = int64_t(1) << (n - 2);
        int gr = grid_for(nq, th);
        switch (shape) {
        case SH_DENSE2: k_gate2<R, SH_DENSE2><<<gr, th, 0, s>>>(psi, nq, q0, q1, rec); break;
        case SH_DIAG2: k_gate2<R, SH_DIAG2><<<gr, th, 0, s>>>(psi, nq, q0, q1, rec); break;
        case SH_PERM2: k_gate2<R, SH_PERM2><<<gr, th, 0, s>>>(psi, nq, q0, q1, rec); break;
        case SH_BLOCK2: k_gate2<R, SH_BLOCK2><<<gr, th, 0, s>>>(psi, nq, q0, q1, rec); break;
        case SH_PAR2: k_gate2<R, SH_PAR2><<<gr, th, 0, s>>>(psi, nq, q0, q1, rec); break;
        case SH_RPAR2: k_gate2<R, SH_RPAR2><<<gr, th, 0, s>>>(psi, nq, q0, q1, rec); break;
        case SH_CX:  // measured: the swap wins in complex128 (no FP64 arithmetic), the
                     // controlled 2x2 in complex64 (87-97% of HBM against 55-60% for the swap)
            if constexpr (sizeof(R) == 8) k_gate2<R, SH_CX><<<gr, th, 0, s>>>(psi, nq, q0, q1, rec);
            else k_gate2<R, SH_CTRL2><<<gr, th, 0, s>>>(psi, nq, q0, q1, rec);
            break;
        case SH_CZ: k_gate2<R, SH_CZ><<<gr, th, 0, s>>>(psi, nq, q0, q1, rec); break;
        default: k_gate2<R, SH_CTRL2><<<gr, th, 0, s>>>(psi, nq, q0, q1, rec); break;
        }
    }
    return cudaGetLastError();
}

cudaError_t launch_gate(int dtype, void *psi, int n, int shape, int q0, int q1, const MatRec *rec,
                        cudaStream_t s)
{
    if (dtype == 0 && shape_qubits(shape) == 1 && q0 == 0) {
        int64_t np = int64_t(1) << (n - 1);
        int gr = grid_for(np, 256);
        float4 *p = (float4 *)psi;
        switch (shape) {
        case SH_DENSE1: k_gate1_q0_c64<SH_DENSE1><<<gr, 256, 0, s>>>(p, np, rec); break;
        case SH_DIAG1: k_gate1_q0_c64<SH_DIAG1><<<gr, 256, 0, s>>>(p, np, rec); break;
        case SH_ANTI1: k_gate1_q0_c64<SH_ANTI1><<<gr, 256, 0, s>>>(p, np, rec); break;
        case SH_IMAG1: k_gate1_q0_c64<SH_IMAG1><<<gr, 256, 0, s>>>(p, np, rec); break;
        default: k_gate1_q0_c64<SH_REAL1><<<gr, 256, 0, s>>>(p, np, rec); break;
        }
        return cudaGetLastError();
    }
    return dtype == 0 ? gate_dispatch<float>(psi, n, shape, q0, q1, rec, s)
                      : gate_dispatch<double>(psi, n, shape, q0, q1, rec, s);
}

// ------------------------------------------------------------------ four-qubit gates

// One thread per group of 16 amplitudes: gather, 16 x 16 complex product from the matrix
// staged in shared memory, scatter (a two-qubit channel's superoperator on (ket q0, ket q1,
// bra q0, bra q1), Eq. channel2).
template <typename R>
__global__ void __launch_bounds__(128) k_gate4(typename CT<R>::T *__restrict__ psi, int64_t ngroups, int4 q,
                                               const MatRec *__restrict__ rows)
{
    typedef typename CT<R>::T T;
    __shared__ R m[512];
    for (int i = threadIdx.x; i < 512; i += blockDim.x) m[i] = mat_of<R>(&rows[i >> 5])[i & 31];
    __syncthreads();
    const int qs[4] = {q.x, q.y, q.z, q.w};
    int srt[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
    for (int a = 0; a < 4; a++)
#pragma unroll
        for (int b = a + 1; b < 4; b++)
            if (srt[b] < srt[a]) {
                const int x = srt[a];
                srt[a] = srt[b];
                srt[b] = x;
            }
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < ngroups; g += stride) {
        int64_t base = g;
#pragma unroll
        for (int u = 0; u < 4; u++) base = insert_zero(base, srt[u]);
        T v[16];
#pragma unroll
        for (int l = 0; l < 16; l++) {
            int64_t ix = base;
#pragma unroll
            for (int u = 0; u < 4; u++)
                if ((l >> u) & 1) ix |= int64_t(1) << qs[u];
            v[l] = psi[ix];
        }
        // the rows in a loop (fully unrolled, the 16 x 16 product put the amplitudes in
        // local memory), each row's index recomputed rather than kept in an array
#pragma unroll 1
        for (int r = 0; r < 16; r++) {
            T acc = cmul<T, R>(m[32 * r], m[32 * r + 1], v[0]);
#pragma unroll
            for (int c = 1; c < 16; c++) cfma<T, R>(m[32 * r + 2 * c], m[32 * r + 2 * c + 1], v[c], acc);
            int64_t ix = base;
#pragma unroll
            for (int u = 0; u < 4; u++)
                if ((r >> u) & 1) ix |= int64_t(1) << qs[u];
            psi[ix] = acc;  // v holds the old values, so rows can be written as they finish
        }
    }
}

cudaError_t launch_gate4(int dtype, void *psi, int n, int q0, int q1, int q2, int q3, const MatRec *rows,
                         cudaStream_t s)
{
    const int64_t ng = int64_t(1) << (n - 4);
    const int gr = grid_for(ng, 128);
    const int4 q = make_int4(q0, q1, q2, q3);
    if (dtype == 0) k_gate4<float><<<gr, 128, 0, s>>>((float2 *)psi, ng, q, rows);
    else k_gate4<double><<<gr, 128, 0, s>>>((double2 *)psi, ng, q, rows);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ small helpers

template <typename T>
__global__ void k_zero_state(T *psi, int64_t len)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < len; i += stride) {
        T z;
        z.x = (i == 0) ? 1 : 0;
        z.y = 0;
        psi[i] = z;
    }
}

cudaError_t launch_zero_state(int dtype, void *psi, int n, cudaStream_t s)
{
    int64_t len = int64_t(1) << n;
    int gr = grid_for(len, 256);
    if (dtype == 0) k_zero_state<float2><<<gr, 256, 0, s>>>((float2 *)psi, len);
    else k_zero_state<double2><<<gr, 256, 0, s>>>((double2 *)psi, len);
    return cudaGetLastError();
}

// Qubit-swap exchange of a sharded state: shard a (global bit j = 0) and shard b (its
// partner, bit j = 1) of 2^L amplitudes each exchange the amplitudes whose local bit l is
// 1 in a with those whose local bit l is 0 in b, at equal other bits; afterwards the
// global qubit and the local qubit have traded positions.  2^(L-1) swaps per pair.
template <typename T>
__global__ void __launch_bounds__(256) k_shard_swap(T *__restrict__ a, T *__restrict__ b, int64_t half, int l)
{
    const int64_t lowmask = (int64_t(1) << l) - 1;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < half; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t x0 = ((i & ~lowmask) << 1) | (i & lowmask);  // local bit l = 0
        const int64_t x1 = x0 | (int64_t(1) << l);
        const T u = a[x1];
        a[x1] = b[x0];
        b[x0] = u;
    }
}

cudaError_t launch_shard_swap(int dtype, void *a, void *b, int local_qubits, int l, cudaStream_t s)
{
    const int64_t half = int64_t(1) << (local_qubits - 1);
    const int gr = grid_for(half, 256);
    if (dtype == 0) k_shard_swap<float2><<<gr, 256, 0, s>>>((float2 *)a, (float2 *)b, half, l);
    else k_shard_swap<double2><<<gr, 256, 0, s>>>((double2 *)a, (double2 *)b, half, l);
    return cudaGetLastError();
}

// Gate materialisation on the device: theta -> rotation matrices (record by record).
__global__ void k_materialize(const DynRec *__restrict__ dyn, int n_dyn,
                              const double *__restrict__ theta, MatRec *recs)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_dyn) return;
    DynRec r = dyn[i];
    materialize(r, theta + r.param, &recs[r.rec]);
}

cudaError_t launch_materialize(const DynRec *dyn, int n_dyn, const double *theta, MatRec *recs,
                               cudaStream_t s)
{
    if (n_dyn == 0) return cudaSuccess;
    k_materialize<<<(n_dyn + 31) / 32, 32, 0, s>>>(dyn, n_dyn, theta, recs);  // spread over SMs
    return cudaGetLastError();
}

// grad[p] = sum of slot_grad over the slots of parameter p, in slot order.
__global__ void k_accumulate(const double *__restrict__ slot_grad, const int *__restrict__ ptr,
                             const int *__restrict__ slots, int n_params, double *grad)
{
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n_params) return;
    double acc = 0.0;
    for (int i = ptr[p]; i < ptr[p + 1]; i++) acc += slot_grad[slots[i]];
    grad[p] = acc;
}

cudaError_t launch_accumulate(const double *slot_grad, const int *csr_ptr, const int *csr_slots,
                              int n_params, double *grad, cudaStream_t s)
{
    if (n_params == 0) return cudaSuccess;
    k_accumulate<<<(n_params + 127) / 128, 128, 0, s>>>(slot_grad, csr_ptr, csr_slots, n_params, grad);
    return cudaGetLastError();
}

}  // namespace gbvqc
