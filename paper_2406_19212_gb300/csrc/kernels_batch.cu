// Batched kernels: many independent circuits (each with its own qubit count, gates,
// parameters and observable) in one launch per step of the gradient sequence.  Every
// CTA finds its (instance, tile) or (instance, chunk) by binary search over the
// launch's prefix table, so one launch covers pass p of every instance that has one.
#include "fused_tile.cuh"
#include "pauli.cuh"

namespace gbvqc {

template <typename E>
__device__ __forceinline__ int find_entry(const E *entries, int n, int64_t cta)
{
    int lo = 0, hi = n - 1;
    while (lo < hi) {  // last entry with begin <= cta
        const int mid = (lo + hi + 1) >> 1;
        if (entries[mid].begin <= cta) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// ------------------------------------------------------------------- fused passes

template <typename R, int NR, bool REV, bool TWOQ>
__global__ void __launch_bounds__(fused_max_threads(NR, REV), fused_min_blocks(REV))
    k_fused_batch(const FusedBatchEntry *__restrict__ entries, int n_entries)
{
    typedef typename CT<R>::T T;
    __shared__ int s_e;
    if (threadIdx.x == 0) s_e = find_entry(entries, n_entries, blockIdx.x);
    __syncthreads();
    const FusedBatchEntry &e = entries[s_e];
    fused_tile<R, NR, REV, TWOQ>((T *)e.phi, (T *)e.psi, e.args, (int64_t)blockIdx.x - e.begin);
}

// Per-instance launch and shared-memory opt-in, compiled in separate objects like the
// single-circuit kernels (GBVQC_PART 0..7; 8 = everything else).
template <typename R, int NR, bool REV, bool TWOQ>
cudaError_t fused_batch_launch_t(unsigned grid, int threads, size_t smem, const FusedBatchEntry *entries,
                                 int n_entries, cudaStream_t s)
{
    k_fused_batch<R, NR, REV, TWOQ><<<grid, threads, smem, s>>>(entries, n_entries);
    return cudaGetLastError();
}

template <typename R, int NR, bool REV, bool TWOQ>
cudaError_t fused_batch_prepare_t()
{
    return cudaFuncSetAttribute(k_fused_batch<R, NR, REV, TWOQ>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                200 * 1024);
}

#define GBVQC_BATCH_INST(EXT, R, NR, REV, TQ)                                                                \
    EXT template cudaError_t fused_batch_launch_t<R, NR, REV, TQ>(unsigned, int, size_t, const FusedBatchEntry *, \
                                                                  int, cudaStream_t);                       \
    EXT template cudaError_t fused_batch_prepare_t<R, NR, REV, TQ>();

#if !defined(GBVQC_PART) || GBVQC_PART == 0
GBVQC_BATCH_INST(, float, 5, false, false)
#endif
#if !defined(GBVQC_PART) || GBVQC_PART == 1
GBVQC_BATCH_INST(, float, 5, false, true)
#endif
#if !defined(GBVQC_PART) || GBVQC_PART == 2
GBVQC_BATCH_INST(, float, 4, true, false)
#endif
#if !defined(GBVQC_PART) || GBVQC_PART == 3
GBVQC_BATCH_INST(, float, 4, true, true)
#endif
#if !defined(GBVQC_PART) || GBVQC_PART == 4
GBVQC_BATCH_INST(, double, 4, false, false)
#endif
#if !defined(GBVQC_PART) || GBVQC_PART == 5
GBVQC_BATCH_INST(, double, 4, false, true)
#endif
#if !defined(GBVQC_PART) || GBVQC_PART == 6
GBVQC_BATCH_INST(, double, 3, true, false)
#endif
#if !defined(GBVQC_PART) || GBVQC_PART == 7
GBVQC_BATCH_INST(, double, 3, true, true)
#endif

#if !defined(GBVQC_PART) || GBVQC_PART == 8
#if defined(GBVQC_PART)
GBVQC_BATCH_INST(extern, float, 5, false, false)
GBVQC_BATCH_INST(extern, float, 5, false, true)
GBVQC_BATCH_INST(extern, float, 4, true, false)
GBVQC_BATCH_INST(extern, float, 4, true, true)
GBVQC_BATCH_INST(extern, double, 4, false, false)
GBVQC_BATCH_INST(extern, double, 4, false, true)
GBVQC_BATCH_INST(extern, double, 3, true, false)
GBVQC_BATCH_INST(extern, double, 3, true, true)
#endif

cudaError_t fused_batch_prepare()
{
    cudaError_t e = fused_batch_prepare_t<float, 5, false, false>();
    if (e == cudaSuccess) e = fused_batch_prepare_t<float, 5, false, true>();
    if (e == cudaSuccess) e = fused_batch_prepare_t<float, 4, true, false>();
    if (e == cudaSuccess) e = fused_batch_prepare_t<float, 4, true, true>();
    if (e == cudaSuccess) e = fused_batch_prepare_t<double, 4, false, false>();
    if (e == cudaSuccess) e = fused_batch_prepare_t<double, 4, false, true>();
    if (e == cudaSuccess) e = fused_batch_prepare_t<double, 3, true, false>();
    if (e == cudaSuccess) e = fused_batch_prepare_t<double, 3, true, true>();
    return e;
}

cudaError_t launch_fused_batch(int dtype, bool reverse, bool two_q, int t, const FusedBatchEntry *entries,
                               int n_entries, int64_t total_tiles, size_t smem, cudaStream_t s)
{
    const int nr = fused_nr(dtype, reverse);
    const int threads = 1 << (t - nr);
    const unsigned g = (unsigned)total_tiles;
#define GBVQC_LB(R, NR, REV)                                                                          \
    return two_q ? fused_batch_launch_t<R, NR, REV, true>(g, threads, smem, entries, n_entries, s)    \
                 : fused_batch_launch_t<R, NR, REV, false>(g, threads, smem, entries, n_entries, s);
    if (dtype == 0) {
        if (reverse) GBVQC_LB(float, 4, true)
        GBVQC_LB(float, 5, false)
    }
    if (reverse) GBVQC_LB(double, 3, true)
    GBVQC_LB(double, 4, false)
#undef GBVQC_LB
}

// ------------------------------------------------------------- Pauli expectation

template <typename R> struct CTb;
template <> struct CTb<float> { typedef float2 T; };
template <> struct CTb<double> { typedef double2 T; };

__device__ __forceinline__ double bwarp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// lambda = H psi on one chunk of one instance and the chunk's partial of Re <psi|lambda>.
// STAGED: every CTA stages its instance's observable in shared memory first.
template <typename R, bool STAGED>
__global__ void __launch_bounds__(256) k_pauli_batch(const PauliBatchEntry *__restrict__ entries, int n_entries)
{
    typedef typename CTb<R>::T T;
    extern __shared__ __align__(16) unsigned char psm[];
    __shared__ int s_e;
    __shared__ double s_w[8];
    if (threadIdx.x == 0) s_e = find_entry(entries, n_entries, blockIdx.x);
    __syncthreads();
    const PauliBatchEntry &e = entries[s_e];
    const int64_t chunk = (int64_t)blockIdx.x - e.begin;
    const int64_t len = int64_t(1) << e.n;
    const int64_t a0 = chunk << kPauliChunkBits;
    const int64_t a1 = a0 + (int64_t(1) << kPauliChunkBits) < len ? a0 + (int64_t(1) << kPauliChunkBits) : len;
    const T *psi = (const T *)e.psi;
    T *lam = (T *)e.lam;
    const PGroup *sg = nullptr;
    const PTerm<R> *st = nullptr;
    if (STAGED) stage_obs<R>(e.obs, psm, sg, st);
    const bool wide = e.n > 32;
    double acc = 0.0;
    if (!STAGED) {
        for (int64_t a = a0 + threadIdx.x; a < a1; a += blockDim.x) {
            const T pa = psi[a];
            R lr, li;
            pauli_apply_amp<R, T>(psi, (uint64_t)a, pa, e.obs, lr, li);
            T l;
            l.x = lr;
            l.y = li;
            lam[a] = l;
            acc += (double)(pa.x * lr + pa.y * li);
        }
    } else {
        constexpr int V = 4;
        for (int64_t base = a0 + threadIdx.x; base < a1; base += (int64_t)blockDim.x * V) {
            uint64_t a[V];
            bool ok[V];
            T pa[V];
            R lr[V], li[V];
#pragma unroll
            for (int j = 0; j < V; j++) {
                a[j] = (uint64_t)(base + (int64_t)j * blockDim.x);
                ok[j] = (int64_t)a[j] < a1;
                pa[j] = ok[j] ? psi[a[j]] : T{};
            }
            if (wide) pauli_apply_staged<R, true, V, T>(psi, a, ok, pa, sg, st, e.obs.n_groups, lr, li);
            else pauli_apply_staged<R, false, V, T>(psi, a, ok, pa, sg, st, e.obs.n_groups, lr, li);
#pragma unroll
            for (int j = 0; j < V; j++) {
                if (!ok[j]) continue;
                T l;
                l.x = lr[j];
                l.y = li[j];
                lam[a[j]] = l;
                acc += (double)(pa[j].x * lr[j] + pa[j].y * li[j]);
            }
        }
    }
    acc = bwarp_sum(acc);
    if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) t += s_w[w];
        e.partials[chunk] = t;
    }
}

cudaError_t pauli_batch_prepare()
{
    const int bytes = (int)kObsStageMax;
    cudaError_t e = cudaFuncSetAttribute(k_pauli_batch<float, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_pauli_batch<double, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    return e;
}

// energy[i] = sum of instance i's chunk partials, in chunk order.
__global__ void k_energy_batch(const PauliBatchEntry *__restrict__ entries, int n_entries, double *energies)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_entries) return;
    const PauliBatchEntry &e = entries[i];
    const int64_t chunks = ((int64_t(1) << e.n) + (int64_t(1) << kPauliChunkBits) - 1) >> kPauliChunkBits;
    double t = 0.0;
    for (int64_t c = 0; c < chunks; c++) t += e.partials[c];
    energies[i] = t;
}

cudaError_t launch_pauli_batch(int dtype, const PauliBatchEntry *entries, int n_entries, int64_t total_chunks,
                               size_t smem, double *energies, cudaStream_t s)
{
    const unsigned g = (unsigned)total_chunks;
    if (dtype == 0) {
        if (smem) k_pauli_batch<float, true><<<g, 256, smem, s>>>(entries, n_entries);
        else k_pauli_batch<float, false><<<g, 256, 0, s>>>(entries, n_entries);
    } else {
        if (smem) k_pauli_batch<double, true><<<g, 256, smem, s>>>(entries, n_entries);
        else k_pauli_batch<double, false><<<g, 256, 0, s>>>(entries, n_entries);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_energy_batch<<<(n_entries + 127) / 128, 128, 0, s>>>(entries, n_entries, energies);
    return cudaGetLastError();
}

// ------------------------------------------------------------- gradient slots

// slot_grad[global slot] = sum over the instance's tiles of its per-(slot, tile) partials.
__global__ void k_slots_batch(const SlotBatchEntry *__restrict__ entries, int n_entries, double *slot_grad)
{
    __shared__ double sh[256];
    __shared__ int s_e;
    if (threadIdx.x == 0) s_e = find_entry(entries, n_entries, blockIdx.x);
    __syncthreads();
    const SlotBatchEntry &e = entries[s_e];
    const int64_t slot = (int64_t)blockIdx.x - e.begin;
    double acc = 0.0;
    for (int i = threadIdx.x; i < e.n_tiles; i += blockDim.x) acc += e.partials[slot * e.n_tiles + i];
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) slot_grad[blockIdx.x] = sh[0];
}

cudaError_t launch_slots_batch(const SlotBatchEntry *entries, int n_entries, int64_t total_slots, double *slot_grad,
                               cudaStream_t s)
{
    if (total_slots == 0) return cudaSuccess;
    k_slots_batch<<<(unsigned)total_slots, 256, 0, s>>>(entries, n_entries, slot_grad);
    return cudaGetLastError();
}

// ------------------------------------------------------------- materialisation

__global__ void k_materialize_batch(const BatchDyn *__restrict__ dyn, int n_dyn, const double *__restrict__ theta)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_dyn) return;
    const BatchDyn d = dyn[i];
    materialize(d.r, theta + d.theta_index, d.rec);
}

// psi_i = |0...0> for every instance of a contiguous batch buffer.
__global__ void k_zero_ones(void *base, const int64_t *offsets, int n, int dtype)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (dtype == 0) ((float2 *)base)[offsets[i]] = make_float2(1.f, 0.f);
    else ((double2 *)base)[offsets[i]] = make_double2(1.0, 0.0);
}

cudaError_t launch_batch_init(const BatchDyn *dyn, int n_dyn, const double *theta, int dtype, void *phi_all,
                              size_t phi_bytes, const int64_t *offsets, int n_inst, cudaStream_t s, bool zero_states)
{
    if (n_dyn > 0) {
        k_materialize_batch<<<(n_dyn + 127) / 128, 128, 0, s>>>(dyn, n_dyn, theta);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    if (!zero_states) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(phi_all, 0, phi_bytes, s);
    if (e != cudaSuccess) return e;
    k_zero_ones<<<(n_inst + 127) / 128, 128, 0, s>>>(phi_all, offsets, n_inst, dtype);
    return cudaGetLastError();
}

#endif  // part 8

}  // namespace gbvqc
