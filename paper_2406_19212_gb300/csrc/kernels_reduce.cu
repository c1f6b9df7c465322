// Reductions over 2^n amplitudes: Pauli-sum expectation (Sec. II.E) fused with the
// adjoint seed lambda = H psi (Algorithm 2 initialisation), the per-gate gradient term
// 2 Re <Psi|dQ|Phi> of Algorithm 2, and the density-matrix trace tr(H rho) / vec(H)
// seed of Sec. III.E.  Complex64 states accumulate in FP32 over runs of 16 terms and
// in FP64 above that; warp shuffles and a last-block-done pass make every sum a
// deterministic FP64 tree.
#include "kernels.h"
#include "pauli.cuh"

namespace gbvqc {

template <typename R> struct CTr;
template <> struct CTr<float> { typedef float2 T; };
template <> struct CTr<double> { typedef double2 T; };

template <typename R> __device__ __forceinline__ const R *mat_r(const MatRec *r);
template <> __device__ __forceinline__ const float *mat_r<float>(const MatRec *r) { return r->f; }
template <> __device__ __forceinline__ const double *mat_r<double>(const MatRec *r) { return r->d; }

// Per-thread accumulator: FP64 directly, or FP32 runs of 16 folded into FP64.
template <typename R> struct Acc;
template <> struct Acc<double> {
    double s = 0.0;
    __device__ __forceinline__ void add(double v) { s += v; }
    __device__ __forceinline__ double get() const { return s; }
};
template <> struct Acc<float> {
    double s = 0.0;
    float run = 0.f;
    int k = 0;
    __device__ __forceinline__ void add(float v)
    {
        run += v;
        if (++k == 16) { s += (double)run; run = 0.f; k = 0; }
    }
    __device__ __forceinline__ double get() const { return s + (double)run; }
};

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Sum over the block (result valid in thread 0); blockDim.x a multiple of 32, <= 1024.
__device__ double block_sum(double v)
{
    __shared__ double sh[32];
    v = warp_sum(v);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
    __syncthreads();
    if (l == 0) sh[w] = v;
    __syncthreads();
    double r = 0.0;
    if (w == 0) {
        r = l < nw ? sh[l] : 0.0;
        r = warp_sum(r);
    }
    return r;
}

// Each block writes its partial; the last block to arrive sums them in index order.
__device__ void grid_finish(double v, RedScratch red, double *out, double scale)
{
    __shared__ bool last;
    double b = block_sum(v);
    if (threadIdx.x == 0) {
        red.partials[blockIdx.x] = b;
        __threadfence();
        unsigned prev = atomicAdd(red.counter, 1u);
        last = (prev == gridDim.x - 1);
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    double s = 0.0;
    for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) s += __ldcg(&red.partials[i]);
    s = block_sum(s);
    if (threadIdx.x == 0) {
        *out = s * scale;
        *red.counter = 0u;
    }
}

static inline int red_grid(int64_t items, int threads)
{
    int64_t b = (items + threads - 1) / threads;
    if (b > 152 * 4) b = 152 * 4;
    if (b < 1) b = 1;
    return (int)b;
}

__device__ __forceinline__ int64_t insert0(int64_t g, int q)
{
    return ((g >> q) << (q + 1)) | (g & ((int64_t(1) << q) - 1));
}

// ---------------------------------------------------------------- 2 Re <Psi|D|Phi>

template <typename R, int K>
__global__ void __launch_bounds__(256) k_dot_matrix(const typename CTr<R>::T *__restrict__ psi,
                                                    const typename CTr<R>::T *__restrict__ phi,
                                                    int64_t ngroups, int q0, int q1,
                                                    const MatRec *__restrict__ rec, double scale,
                                                    RedScratch red, double *out)
{
    typedef typename CTr<R>::T T;
    constexpr int D = 1 << K;
    R m[2 * D * D];
    const R *src = mat_r<R>(rec);
#pragma unroll
    for (int i = 0; i < 2 * D * D; i++) m[i] = src[i];
    const int lo = q0 < q1 ? q0 : q1, hi = q0 < q1 ? q1 : q0;
    Acc<R> acc;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < ngroups; g += stride) {
        int64_t idx[D];
        if (K == 1) {
            idx[0] = insert0(g, q0);
            idx[1] = idx[0] | (int64_t(1) << q0);
        } else {
            int64_t base = insert0(insert0(g, lo), hi);
            idx[0] = base;
            idx[1] = base | (int64_t(1) << q0);
            idx[2] = base | (int64_t(1) << q1);
            idx[3] = idx[1] | (int64_t(1) << q1);
        }
        T f[D];
#pragma unroll
        for (int l = 0; l < D; l++) f[l] = phi[idx[l]];
        R part = 0;
#pragma unroll
        for (int r = 0; r < D; r++) {
            R wr = 0, wi = 0;
#pragma unroll
            for (int c = 0; c < D; c++) {
                R mr = m[2 * (r * D + c)], mi = m[2 * (r * D + c) + 1];
                wr += mr * f[c].x - mi * f[c].y;
                wi += mr * f[c].y + mi * f[c].x;
            }
            T p = psi[idx[r]];
            part += p.x * wr + p.y * wi;   // Re(conj(p) * w)
        }
        acc.add(part);
    }
    grid_finish(acc.get(), red, out, scale);
}

cudaError_t launch_dot_matrix(int dtype, const void *psi, const void *phi, int n, int k, int q0,
                              int q1, const MatRec *rec, double scale, RedScratch red, double *out,
                              cudaStream_t s)
{
    int64_t ng = int64_t(1) << (n - k);
    int gr = red_grid(ng, 256);
    if (dtype == 0) {
        if (k == 1)
            k_dot_matrix<float, 1><<<gr, 256, 0, s>>>((const float2 *)psi, (const float2 *)phi, ng,
                                                      q0, q1, rec, scale, red, out);
        else
            k_dot_matrix<float, 2><<<gr, 256, 0, s>>>((const float2 *)psi, (const float2 *)phi, ng,
                                                      q0, q1, rec, scale, red, out);
    } else {
        if (k == 1)
            k_dot_matrix<double, 1><<<gr, 256, 0, s>>>((const double2 *)psi, (const double2 *)phi,
                                                       ng, q0, q1, rec, scale, red, out);
        else
            k_dot_matrix<double, 2><<<gr, 256, 0, s>>>((const double2 *)psi, (const double2 *)phi,
                                                       ng, q0, q1, rec, scale, red, out);
    }
    return cudaGetLastError();
}

// ------------------------------------------------------------------- Pauli sums

// lambda = H psi (when lam is set) and Re <psi|H psi>.  MODE 0 reads the observable
// from global memory; 1 and 2 stage it in shared memory (2: more than 32 qubits).
template <typename R, int MODE>
__global__ void __launch_bounds__(256) k_pauli_expect(const typename CTr<R>::T *__restrict__ psi,
                                                      typename CTr<R>::T *__restrict__ lam,
                                                      int64_t len, ObsDev obs, RedScratch red,
                                                      double *out)
{
    typedef typename CTr<R>::T T;
    extern __shared__ __align__(16) unsigned char psm[];
    const PGroup *sg = nullptr;
    const PTerm<R> *st = nullptr;
    if (MODE != 0) stage_obs<R>(obs, psm, sg, st);
    Acc<R> acc;
    if (MODE == 0) {
        const int64_t stride = (int64_t)gridDim.x * blockDim.x;
        for (int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; a < len; a += stride) {
            const T pa = psi[a];
            R lr, li;
            pauli_apply_amp<R, T>(psi, (uint64_t)a, pa, obs, lr, li);
            if (lam) {
                T l;
                l.x = lr;
                l.y = li;
                lam[a] = l;
            }
            acc.add(pa.x * lr + pa.y * li);
        }
    } else {
        // V amplitudes per thread, blockDim apart (coalesced), per outer iteration
        constexpr int V = 4;
        const int64_t stride = (int64_t)gridDim.x * blockDim.x * V;
        for (int64_t base = (int64_t)blockIdx.x * blockDim.x * V + threadIdx.x; base < len; base += stride) {
            uint64_t a[V];
            bool ok[V];
            T pa[V];
            R lr[V], li[V];
#pragma unroll
            for (int j = 0; j < V; j++) {
                a[j] = (uint64_t)(base + (int64_t)j * blockDim.x);
                ok[j] = (int64_t)a[j] < len;
                pa[j] = ok[j] ? psi[a[j]] : T{};
            }
            pauli_apply_staged<R, MODE == 2, V, T>(psi, a, ok, pa, sg, st, obs.n_groups, lr, li);
#pragma unroll
            for (int j = 0; j < V; j++) {
                if (!ok[j]) continue;
                if (lam) {
                    T l;
                    l.x = lr[j];
                    l.y = li[j];
                    lam[a[j]] = l;
                }
                acc.add(pa[j].x * lr[j] + pa[j].y * li[j]);
            }
        }
    }
    grid_finish(acc.get(), red, out, 1.0);
}

// ----------------------------------------------------- chunked Pauli sums (n >= 10)
//
// The same lambda = H psi and Re <psi|H psi> with the state read in chunks of 2^kPauliC
// amplitudes: a CTA stages its chunk in shared memory, so the partner psi_{a ^ x_g} of a
// group whose X mask stays inside the chunk's bits is a shared-memory read (only groups
// that flip a higher bit read the partner chunk from global memory / L2).  A thread owns
// the kPauliPV amplitudes a = hi | r << kPauliTB | tid.  Since popcount((a ^ x) & z) =
// popcount(a & z) + popcount(x & z) mod 2, each term's group sign (-1)^{x_g . z} is folded
// into its staged coefficient, and the sign of amplitude r is the thread's parity of
// (hi | tid) & z flipped by bit r of the term's rpat: terms with rpat 0 add one per-thread
// constant, groups whose every Z mask is empty take one constant coefficient.
template <typename R> struct ChunkTerm;
template <> struct ChunkTerm<float> { typedef ChunkTermF T; };
template <> struct ChunkTerm<double> { typedef ChunkTermD T; };

inline size_t chunk_smem_bytes(const ObsDev &obs, int dtype)
{
    const size_t amp = dtype == 0 ? 8 : 16, term = dtype == 0 ? sizeof(ChunkTermF) : sizeof(ChunkTermD);
    return (amp << kPauliC) + chunk_terms_f_offset(obs.n_groups) + ((term * (size_t)obs.n_terms + 15) & ~size_t(15));
}

template <typename R>
__global__ void __launch_bounds__(1 << kPauliTB) k_pauli_chunk(const typename CTr<R>::T *__restrict__ psi,
                                                               typename CTr<R>::T *__restrict__ lam,
                                                               int64_t n_chunks, ObsDev obs, RedScratch red,
                                                               double *out)
{
    typedef typename CTr<R>::T T;
    typedef typename ChunkTerm<R>::T CT_;
    constexpr int PV = kPauliPV, TB = kPauliTB, PC = kPauliC;
    extern __shared__ __align__(16) unsigned char psm[];
    T *sx = reinterpret_cast<T *>(psm);
    unsigned char *sobs = psm + (sizeof(T) << PC);
    const int tid = threadIdx.x, G = obs.n_groups;
    const size_t goff = chunk_terms_f_offset(G);
    const ChunkGroup *sg = reinterpret_cast<const ChunkGroup *>(sobs);
    const CT_ *st = reinterpret_cast<const CT_ *>(sobs + goff);

    // the first chunk's own amplitudes are requested before the observable is staged
    int64_t chunk = blockIdx.x;
    T pa[PV];
#pragma unroll
    for (int r = 0; r < PV; r++) pa[r] = psi[(chunk << PC) | (r << TB) | tid];
    {
        const int4 *src = reinterpret_cast<const int4 *>(obs.chunk);
        int4 *dst = reinterpret_cast<int4 *>(sobs);
        for (int i = tid; i < (int)(goff / 16); i += blockDim.x) dst[i] = src[i];
        const size_t toff = sizeof(R) == 4 ? goff : chunk_terms_d_offset(G, obs.n_terms);
        const int tw = (int)((sizeof(CT_) * (size_t)obs.n_terms + 15) / 16);
        const int4 *tsrc = reinterpret_cast<const int4 *>(obs.chunk + toff);
        int4 *tdst = reinterpret_cast<int4 *>(sobs + goff);
        for (int i = tid; i < tw; i += blockDim.x) tdst[i] = tsrc[i];
    }
    double acc = 0.0;
    for (; chunk < n_chunks; chunk += gridDim.x) {
        const int64_t hi = chunk << PC;
        if (chunk != (int64_t)blockIdx.x) {
#pragma unroll
            for (int r = 0; r < PV; r++) pa[r] = psi[hi | (r << TB) | tid];
        }
#pragma unroll
        for (int r = 0; r < PV; r++) sx[(r << TB) | tid] = pa[r];
        __syncthreads();
        const uint64_t a0 = (uint64_t)(hi | tid);
        const uint32_t a0lo = (uint32_t)a0, a0hi = (uint32_t)(a0 >> 32);
        R lr[PV], li[PV];
#pragma unroll
        for (int r = 0; r < PV; r++) lr[r] = li[r] = R(0);
        for (int g = 0; g < G; g++) {
            const ChunkGroup gr = sg[g];
            T pb[PV];
            if (gr.flags & CG_SELF) {
#pragma unroll
                for (int r = 0; r < PV; r++) pb[r] = pa[r];
            } else {
                const uint32_t xl = gr.xlo & ((1u << PC) - 1);
                if (gr.flags & CG_CHUNK) {
#pragma unroll
                    for (int r = 0; r < PV; r++) pb[r] = sx[((uint32_t)(r << TB) | tid) ^ xl];
                } else {
                    const uint64_t x = (uint64_t)gr.xlo | ((uint64_t)gr.xhi << 32);
                    const int64_t ph = hi ^ (int64_t)(x & ~uint64_t((1u << PC) - 1));
#pragma unroll
                    for (int r = 0; r < PV; r++) pb[r] = psi[ph | (int64_t)(((uint32_t)(r << TB) | tid) ^ xl)];
                }
            }
            // per-amplitude coefficient: a per-thread constant part (c0) plus the terms
            // whose sign depends on the register index (cr / ci)
            R c0r = 0, c0i = 0, cr[PV], ci[PV];
#pragma unroll
            for (int r = 0; r < PV; r++) cr[r] = ci[r] = R(0);
            const bool real = (gr.flags & CG_REAL) != 0;
            if (gr.flags & CG_CONST) {
                for (int k = gr.t_begin; k < gr.t_end; k++) {
                    c0r += st[k].cr;
                    c0i += st[k].ci;
                }
            } else {
                for (int k = gr.t_begin; k < gr.t_end; k++) {
                    const CT_ t = st[k];
                    const uint32_t par = (__popc(a0lo & t.zlo) ^ __popc(a0hi & t.zhi)) & 1;
                    const R sr = sign_flip(t.cr, par), si = sign_flip(t.ci, par);
                    if (t.rpat == 0) {
                        c0r += sr;
                        c0i += si;
                    } else {
#pragma unroll
                        for (int r = 0; r < PV; r++) {
                            const uint32_t f = (t.rpat >> r) & 1;
                            cr[r] += sign_flip(sr, f);
                            if (!real) ci[r] += sign_flip(si, f);
                        }
                    }
                }
            }
            if (real) {
#pragma unroll
                for (int r = 0; r < PV; r++) {
                    const R c = cr[r] + c0r;
                    lr[r] = fma(c, pb[r].x, lr[r]);
                    li[r] = fma(c, pb[r].y, li[r]);
                }
            } else {
#pragma unroll
                for (int r = 0; r < PV; r++) {
                    const R c = cr[r] + c0r, d = ci[r] + c0i;
                    lr[r] = fma(c, pb[r].x, fma(-d, pb[r].y, lr[r]));
                    li[r] = fma(c, pb[r].y, fma(d, pb[r].x, li[r]));
                }
            }
        }
        R e = 0;
#pragma unroll
        for (int r = 0; r < PV; r++) {
            if (lam) {
                T l;
                l.x = lr[r];
                l.y = li[r];
                lam[hi | (r << TB) | tid] = l;
            }
            e += pa[r].x * lr[r] + pa[r].y * li[r];
        }
        acc += (double)e;
        __syncthreads();  // the next chunk overwrites sx
    }
    grid_finish(acc, red, out, 1.0);
}

cudaError_t pauli_prepare()
{
    const int bytes = (int)kObsStageMax;
    cudaError_t e = cudaFuncSetAttribute(k_pauli_expect<float, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_pauli_expect<float, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_pauli_expect<double, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_pauli_expect<double, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_pauli_chunk<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_pauli_chunk<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess) e = pauli_batch_prepare();
    return e;
}

cudaError_t launch_pauli_expect(int dtype, const void *psi, void *lam, int n, ObsDev obs,
                                RedScratch red, double *out, cudaStream_t s)
{
    int64_t len = int64_t(1) << n;
    if (n >= kPauliC && obs.chunk && obs.n_groups > 0 && obs.n_terms < 65536 &&
        chunk_smem_bytes(obs, dtype) <= kObsStageMax) {
        const int64_t chunks = int64_t(1) << (n - kPauliC);
        const int gr = (int)(chunks > kMaxRedBlocks ? kMaxRedBlocks : chunks);
        const size_t smem = chunk_smem_bytes(obs, dtype);
        if (dtype == 0)
            k_pauli_chunk<float><<<gr, 1 << kPauliTB, smem, s>>>((const float2 *)psi, (float2 *)lam, chunks, obs, red,
                                                                 out);
        else
            k_pauli_chunk<double><<<gr, 1 << kPauliTB, smem, s>>>((const double2 *)psi, (double2 *)lam, chunks, obs,
                                                                  red, out);
        return cudaGetLastError();
    }
    // up to the reduction scratch's 1024 blocks: about 54 warps per SM at 2^20 amplitudes
    const int mode = obs_stageable(obs, dtype) ? (n > 32 ? 2 : 1) : 0;
    const int64_t per_block = mode ? 1024 : 256;  // staged kernels take 4 amplitudes per thread
    int64_t gb = (len + per_block - 1) / per_block;
    const int gr = (int)(gb > kMaxRedBlocks ? kMaxRedBlocks : (gb < 1 ? 1 : gb));
    const size_t smem = mode ? obs_smem_bytes(obs, dtype) : 0;
#define GBVQC_PE(R, T, M) \
    k_pauli_expect<R, M><<<gr, 256, smem, s>>>((const T *)psi, (T *)lam, len, obs, red, out)
    if (dtype == 0) {
        if (mode == 0) GBVQC_PE(float, float2, 0);
        else if (mode == 1) GBVQC_PE(float, float2, 1);
        else GBVQC_PE(float, float2, 2);
    } else {
        if (mode == 0) GBVQC_PE(double, double2, 0);
        else if (mode == 1) GBVQC_PE(double, double2, 1);
        else GBVQC_PE(double, double2, 2);
    }
#undef GBVQC_PE
    return cudaGetLastError();
}

// ------------------------------------------------------------------ density path

__device__ __forceinline__ uint64_t deposit(uint64_t v, const int8_t *pos, int n)
{
    uint64_t r = 0;
    for (int q = 0; q < n; q++)
        if ((v >> q) & 1) r |= uint64_t(1) << pos[q];
    return r;
}

// tr(P rho) = sum_a ph(a) rho_{a, a ^ x}: E = Re sum_a sum_g c_g(a) rho[a, a ^ x_g].
template <typename R>
__global__ void __launch_bounds__(256) k_density_expect(const typename CTr<R>::T *__restrict__ rho,
                                                        int n, DensMap map, ObsDev obs,
                                                        RedScratch red, double *out)
{
    typedef typename CTr<R>::T T;
    const int64_t dim = int64_t(1) << n;
    double acc = 0.0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; a < dim; a += stride) {
        uint64_t ka = deposit((uint64_t)a, map.ket, n);
        for (int g = 0; g < obs.n_groups; g++) {
            ObsGroup gr = obs.groups[g];
            uint64_t b = (uint64_t)a ^ gr.x;
            T v = rho[ka | deposit(b, map.bra, n)];
            R cr, ci;
            group_coeff<R>(obs.terms, gr.t_begin, gr.t_end, (uint64_t)a, cr, ci);
            acc += (double)(cr * v.x - ci * v.y);
        }
    }
    grid_finish(acc, red, out, 1.0);
}

cudaError_t launch_density_expect(int dtype, const void *rho, int n, DensMap map, ObsDev obs,
                                  RedScratch red, double *out, cudaStream_t s)
{
    int gr = red_grid(int64_t(1) << n, 256);
    if (dtype == 0)
        k_density_expect<float><<<gr, 256, 0, s>>>((const float2 *)rho, n, map, obs, red, out);
    else
        k_density_expect<double><<<gr, 256, 0, s>>>((const double2 *)rho, n, map, obs, red, out);
    return cudaGetLastError();
}

// psi_ab = H_ab = sum_k coeff_k ph_k(b) [a == b ^ x_k]
template <typename R>
__global__ void k_density_seed(typename CTr<R>::T *__restrict__ psi, int n, DensMap map, ObsDev obs)
{
    typedef typename CTr<R>::T T;
    const int64_t dim = int64_t(1) << n;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < dim; b += stride) {
        uint64_t kb = deposit((uint64_t)b, map.bra, n);
        for (int g = 0; g < obs.n_groups; g++) {
            ObsGroup gr = obs.groups[g];
            uint64_t a = (uint64_t)b ^ gr.x;
            R cr, ci;
            group_coeff<R>(obs.terms, gr.t_begin, gr.t_end, (uint64_t)b, cr, ci);
            T v;
            v.x = cr;
            v.y = ci;
            psi[deposit(a, map.ket, n) | kb] = v;
        }
    }
}

cudaError_t launch_density_seed(int dtype, void *psi, int n, DensMap map, ObsDev obs, cudaStream_t s)
{
    size_t bytes = (size_t(1) << (2 * n)) * (dtype == 0 ? 8 : 16);
    cudaError_t e = cudaMemsetAsync(psi, 0, bytes, s);
    if (e != cudaSuccess) return e;
    int gr = red_grid(int64_t(1) << n, 256);
    if (dtype == 0) k_density_seed<float><<<gr, 256, 0, s>>>((float2 *)psi, n, map, obs);
    else k_density_seed<double><<<gr, 256, 0, s>>>((double2 *)psi, n, map, obs);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- measurement

// Per-block partial sums of the outcome weights of qubit q (Sec. II.D measure!):
// part[2 blk + k] = sum over this block's indices a with bit q of a equal to k of
// |psi_a|^2 (pure) or Re rho_aa (density, rho_ab at a + 2^n b), in FP64.
template <typename R>
__global__ void __launch_bounds__(256) k_measure_sums(const typename CTr<R>::T *__restrict__ st, int n,
                                                      int density, int q, double *part)
{
    __shared__ double sh[2][256];
    const int64_t dim = int64_t(1) << n;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    double acc[2] = {0.0, 0.0};
    for (int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; a < dim; a += stride) {
        double v;
        if (density) {
            v = (double)st[a + dim * a].x;
        } else {
            const double x = (double)st[a].x, y = (double)st[a].y;
            v = x * x + y * y;
        }
        acc[(a >> q) & 1] += v;
    }
    sh[0][threadIdx.x] = acc[0];
    sh[1][threadIdx.x] = acc[1];
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) {
            sh[0][threadIdx.x] += sh[0][threadIdx.x + w];
            sh[1][threadIdx.x] += sh[1][threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = sh[0][0];
        part[2 * blockIdx.x + 1] = sh[1][0];
    }
}

// out[k] = sum over blocks of part[2 blk + k], in block order.
__global__ void k_measure_finish(const double *__restrict__ part, int nblk, double *out)
{
    if (threadIdx.x < 2) {
        double t = 0.0;
        for (int b = 0; b < nblk; b++) t += part[2 * b + threadIdx.x];
        out[threadIdx.x] = t;
    }
}

cudaError_t launch_measure_sums(int dtype, const void *st, int n, int density, int q, double *scratch,
                                int max_blocks, double *out, cudaStream_t s)
{
    int64_t gb = ((int64_t(1) << n) + 255) / 256;
    const int gr = (int)(gb > max_blocks ? max_blocks : gb);
    if (dtype == 0) k_measure_sums<float><<<gr, 256, 0, s>>>((const float2 *)st, n, density, q, scratch);
    else k_measure_sums<double><<<gr, 256, 0, s>>>((const double2 *)st, n, density, q, scratch);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_measure_finish<<<1, 32, 0, s>>>(scratch, gr, out);
    return cudaGetLastError();
}

// Projection on outcome k of qubit q and renormalisation: pure psi_a -> psi_a * scale if
// bit q of a is k, else 0; density rho_ab -> rho_ab * scale if bit q of a and of b are
// both k, else 0.
template <typename R>
__global__ void k_collapse(typename CTr<R>::T *__restrict__ st, int n, int density, int q, int k, R scale)
{
    typedef typename CTr<R>::T T;
    const int64_t len = int64_t(1) << (density ? 2 * n : n);
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < len; i += stride) {
        const bool keep = density ? (((i >> q) & 1) == k && ((i >> (q + n)) & 1) == k) : ((i >> q) & 1) == k;
        T v = st[i];
        if (keep) {
            v.x *= scale;
            v.y *= scale;
        } else {
            v.x = 0;
            v.y = 0;
        }
        st[i] = v;
    }
}

cudaError_t launch_collapse(int dtype, void *st, int n, int density, int q, int k, double scale, cudaStream_t s)
{
    const int64_t len = int64_t(1) << (density ? 2 * n : n);
    const int gr = red_grid(len, 256);
    if (dtype == 0) k_collapse<float><<<gr, 256, 0, s>>>((float2 *)st, n, density, q, k, (float)scale);
    else k_collapse<double><<<gr, 256, 0, s>>>((double2 *)st, n, density, q, k, scale);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ sampling

template <typename R>
__device__ __forceinline__ double sample_weight(const typename CTr<R>::T *st, int64_t dim, int density, int64_t a)
{
    if (density) return (double)st[a + dim * a].x;
    const double x = (double)st[a].x, y = (double)st[a].y;
    return x * x + y * y;
}

// chunk_sum[m] = sum of the weights of indices [m C, (m+1) C), C = 2^cbits, in FP64 (a
// fixed tree per block).
template <typename R>
__global__ void __launch_bounds__(256) k_chunk_sums(const typename CTr<R>::T *__restrict__ st, int n, int density,
                                                    int cbits, double *chunk_sum)
{
    __shared__ double sh[256];
    const int64_t dim = int64_t(1) << n, a0 = (int64_t)blockIdx.x << cbits, C = int64_t(1) << cbits;
    double acc = 0.0;
    for (int64_t a = a0 + threadIdx.x; a < a0 + C; a += blockDim.x) acc += sample_weight<R>(st, dim, density, a);
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) chunk_sum[blockIdx.x] = sh[0];
}

// incl[m] = chunk_sum[0] + ... + chunk_sum[m] (one block: per-thread runs, then a scan of
// the run totals in thread order).
__global__ void __launch_bounds__(1024) k_chunk_prefix(const double *__restrict__ chunk_sum, int m_chunks, double *incl)
{
    __shared__ double run[1024];
    const int per = (m_chunks + blockDim.x - 1) / blockDim.x;
    const int b = threadIdx.x * per, e = min(m_chunks, b + per);
    double t = 0.0;
    for (int m = b; m < e; m++) t += chunk_sum[m];
    run[threadIdx.x] = t;
    __syncthreads();
    if (threadIdx.x == 0)
        for (int i = 1; i < (int)blockDim.x; i++) run[i] += run[i - 1];
    __syncthreads();
    double acc = threadIdx.x ? run[threadIdx.x - 1] : 0.0;
    for (int m = b; m < e; m++) {
        acc += chunk_sum[m];
        incl[m] = acc;
    }
}

// One warp per shot: the chunk holding u*total by binary search of incl, then the index
// inside it by a warp scan of the chunk's weights in steps of 32.
template <typename R>
__global__ void __launch_bounds__(256) k_sample_shots(const typename CTr<R>::T *__restrict__ st, int n, int density,
                                                      int cbits, const double *__restrict__ incl, int m_chunks,
                                                      const double *__restrict__ u, int n_shots, int64_t *out)
{
    const int lane = threadIdx.x & 31;
    const int shot = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
    if (shot >= n_shots) return;  // whole warps leave together
    const int64_t dim = int64_t(1) << n, C = int64_t(1) << cbits;
    const double total = incl[m_chunks - 1];
    // u < 1 makes target < total in round-to-nearest (u <= 1 - 2^-53, and the rounding error
    // of the product is below half an ulp of total), so the search below always finds a
    // chunk with target < incl[m]; that chunk has non-zero weight (a zero-weight chunk
    // repeats incl[m - 1], which would then have satisfied the test already).
    const double target = u[shot] * total;
    int lo = 0, hi = m_chunks - 1;  // least chunk with target < incl[m]
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (target < incl[mid]) hi = mid;
        else lo = mid + 1;
    }
    double run = lo ? incl[lo - 1] : 0.0;
    const int64_t a0 = (int64_t)lo << cbits;
    int64_t found = a0 + C - 1, last_nz = -1;
    for (int64_t base = a0; base < a0 + C; base += 32) {
        const double w = base + lane < a0 + C ? sample_weight<R>(st, dim, density, base + lane) : 0.0;
        double x = w;  // inclusive warp scan
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const double y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        const unsigned hit = __ballot_sync(0xffffffffu, target < run + x && w > 0.0);
        const unsigned nzm = __ballot_sync(0xffffffffu, w > 0.0);
        if (nzm) last_nz = base + 31 - __clz(nzm);
        if (hit) {
            found = base + __ffs(hit) - 1;
            last_nz = -2;
            break;
        }
        run += __shfl_sync(0xffffffffu, x, 31);
    }
    if (last_nz >= 0) found = last_nz;  // rounding pushed u*total past the chunk's end
    if (lane == 0) out[shot] = found;
}

cudaError_t launch_sample(int dtype, const void *st, int n, int density, int cbits, double *chunk_sum, double *incl,
                          const double *u, int n_shots, int64_t *out, cudaStream_t s)
{
    const int m = 1 << (n - cbits);
    if (dtype == 0) k_chunk_sums<float><<<m, 256, 0, s>>>((const float2 *)st, n, density, cbits, chunk_sum);
    else k_chunk_sums<double><<<m, 256, 0, s>>>((const double2 *)st, n, density, cbits, chunk_sum);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_chunk_prefix<<<1, 1024, 0, s>>>(chunk_sum, m, incl);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const int blocks = (int)((32 * (int64_t)n_shots + 255) / 256);
    if (dtype == 0)
        k_sample_shots<float><<<blocks, 256, 0, s>>>((const float2 *)st, n, density, cbits, incl, m, u, n_shots, out);
    else
        k_sample_shots<double><<<blocks, 256, 0, s>>>((const double2 *)st, n, density, cbits, incl, m, u, n_shots, out);
    return cudaGetLastError();
}

}  // namespace gbvqc
