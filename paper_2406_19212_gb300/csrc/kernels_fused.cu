// Fused tile-pass kernels of one circuit (one CTA per tile) and their launchers.  The
// tile-pass body lives in fused_tile.cuh.
#include "fused_tile.cuh"

namespace gbvqc {

// Launch bounds from fused_max_threads / fused_min_blocks.
template <typename R, int NR, bool REV, bool TWOQ>
__global__ void __launch_bounds__(fused_max_threads(NR, REV), fused_min_blocks(REV))
    k_fused(typename CT<R>::T *__restrict__ phi, typename CT<R>::T *__restrict__ psi, FusedArgs args)
{
    fused_tile<R, NR, REV, TWOQ>(phi, psi, args, blockIdx.x);
}

// One launch / shared-memory opt-in per kernel instance.  The instances are compiled in
// separate objects (GBVQC_PART 0..7, one per precision x direction x two-qubit flavour;
// 8 = the dispatchers and small kernels) so the build runs them in parallel; without
// GBVQC_PART everything is compiled in one object.
template <typename R, int NR, bool REV, bool TWOQ>
cudaError_t fused_launch_t(void *phi, void *psi, unsigned tiles, int threads, size_t smem, FusedArgs args,
                           cudaStream_t s)
{
    typedef typename CT<R>::T T;
    k_fused<R, NR, REV, TWOQ><<<tiles, threads, smem, s>>>((T *)phi, (T *)psi, args);
    return cudaGetLastError();
}

template <typename R, int NR, bool REV, bool TWOQ>
cudaError_t fused_prepare_t()  // large dynamic shared memory (call outside stream capture)
{
    return cudaFuncSetAttribute(k_fused<R, NR, REV, TWOQ>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
}

#define GBVQC_FUSED_INST(EXT, R, NR, REV, TQ)                                                           \
    EXT template cudaError_t fused_launch_t<R, NR, REV, TQ>(void *, void *, unsigned, int, size_t, FusedArgs, \
                                                            cudaStream_t);                              \
    EXT template cudaError_t fused_prepare_t<R, NR, REV, TQ>();

#if !defined(GBVQC_PART) || GBVQC_PART == 0
GBVQC_FUSED_INST(, float, 5, false, false)
#endif
#if !defined(GBVQC_PART) || GBVQC_PART == 1
GBVQC_FUSED_INST(, float, 5, false, true)
#endif
#if !defined(GBVQC_PART) || GBVQC_PART == 2
GBVQC_FUSED_INST(, float, 4, true, false)
#endif
#if !defined(GBVQC_PART) || GBVQC_PART == 3
GBVQC_FUSED_INST(, float, 4, true, true)
#endif
#if !defined(GBVQC_PART) || GBVQC_PART == 4
GBVQC_FUSED_INST(, double, 4, false, false)
#endif
#if !defined(GBVQC_PART) || GBVQC_PART == 5
GBVQC_FUSED_INST(, double, 4, false, true)
#endif
#if !defined(GBVQC_PART) || GBVQC_PART == 6
GBVQC_FUSED_INST(, double, 3, true, false)
#endif
#if !defined(GBVQC_PART) || GBVQC_PART == 7
GBVQC_FUSED_INST(, double, 3, true, true)
#endif

#if !defined(GBVQC_PART) || GBVQC_PART == 8
#if defined(GBVQC_PART)
GBVQC_FUSED_INST(extern, float, 5, false, false)
GBVQC_FUSED_INST(extern, float, 5, false, true)
GBVQC_FUSED_INST(extern, float, 4, true, false)
GBVQC_FUSED_INST(extern, float, 4, true, true)
GBVQC_FUSED_INST(extern, double, 4, false, false)
GBVQC_FUSED_INST(extern, double, 4, false, true)
GBVQC_FUSED_INST(extern, double, 3, true, false)
GBVQC_FUSED_INST(extern, double, 3, true, true)
#endif

// -------------------------------------------------------------------------- launchers

int fused_nr(int dtype, bool reverse)
{
    if (dtype == 0) return reverse ? 4 : 5;
    return reverse ? 3 : 4;
}

cudaError_t fused_prepare()
{
    cudaError_t e = fused_prepare_t<float, 5, false, false>();
    if (e == cudaSuccess) e = fused_prepare_t<float, 5, false, true>();
    if (e == cudaSuccess) e = fused_prepare_t<float, 4, true, false>();
    if (e == cudaSuccess) e = fused_prepare_t<float, 4, true, true>();
    if (e == cudaSuccess) e = fused_prepare_t<double, 4, false, false>();
    if (e == cudaSuccess) e = fused_prepare_t<double, 4, false, true>();
    if (e == cudaSuccess) e = fused_prepare_t<double, 3, true, false>();
    if (e == cudaSuccess) e = fused_prepare_t<double, 3, true, true>();
    return e;
}

template <typename R, int NR, bool REV>
static cudaError_t fused_launch(void *phi, void *psi, const PassDesc &ph, size_t smem, FusedArgs args,
                                cudaStream_t s)
{
    const int threads = 1 << (ph.t - NR);
    const unsigned tiles = (unsigned)(int64_t(1) << (ph.n - ph.t));
    if (ph.has_2q) return fused_launch_t<R, NR, REV, true>(phi, psi, tiles, threads, smem, args, s);
    return fused_launch_t<R, NR, REV, false>(phi, psi, tiles, threads, smem, args, s);
}

cudaError_t launch_fused_forward(int dtype, void *psi, const FusedDev &fd, int pass, const PassDesc &ph,
                                 size_t smem, cudaStream_t s, bool init)
{
    FusedArgs args{fd.passes + pass, fd.subs, fd.gates, fd.ents, fd.units, fd.recs, fd.img, nullptr, 0};
    args.init = init ? 1 : 0;
    if (dtype == 0) return fused_launch<float, 5, false>(psi, nullptr, ph, smem, args, s);
    return fused_launch<double, 4, false>(psi, nullptr, ph, smem, args, s);
}

cudaError_t launch_fused_reverse(int dtype, void *phi, void *psi, const FusedDev &fd, int pass,
                                 const PassDesc &ph, size_t smem, double *slot_partials, int n_tiles_stride,
                                 cudaStream_t s)
{
    FusedArgs args{fd.passes + pass, fd.subs, fd.gates, fd.ents, fd.units, fd.recs, fd.img, slot_partials,
                   n_tiles_stride};
    if (dtype == 0) return fused_launch<float, 4, true>(phi, psi, ph, smem, args, s);
    return fused_launch<double, 3, true>(phi, psi, ph, smem, args, s);
}

// Register phase table entry j of tab: the FP64 product of its entries' diagonal elements
// at the register bits of j, rounded once to R.
template <typename R>
__device__ __forceinline__ void phase_table_entry(const TabDesc &tab, int j, const TabEnt *__restrict__ ents,
                                                  const MatRec *__restrict__ recs, R *img)
{
    double pr = 1.0, pi = 0.0;
    for (int i = 0; i < tab.n_ent; i++) {
        const TabEnt e = ents[tab.ent_begin + i];
        const int r = e.k == 1 ? (j >> e.ca) & 1 : ((j >> e.ca) & 1) | (((j >> e.cb) & 1) << 1);
        const double *m = recs[e.rec].d + (e.k == 1 ? 6 * r : 10 * r);
        const double x = pr * m[0] - pi * m[1];
        pi = pr * m[1] + pi * m[0];
        pr = x;
    }
    img[tab.off + 2 * j] = (R)pr;
    img[tab.off + 2 * j + 1] = (R)pi;
}

// Item i of a plan's per-step image: element i & 7 of unit i >> 3 (forward units, then
// reverse units), then the entries of the forward and reverse phase tables.
template <typename R>
__device__ __forceinline__ void gather_item(const GatherArgs &g, int i)
{
    const int u = i >> 3, e = i & 7;
    R *img_f = (R *)g.img_f, *img_r = (R *)g.img_r;
    if (u < g.nf) {
        const MatUnit m = g.fu[u];
        if (m.rec >= 0) img_f[i] = unit_elem<R>(m, e, g.recs);  // rec < 0: a table's units
    } else if (u < g.nf + g.nr) {
        const MatUnit m = g.ru[u - g.nf];
        if (m.rec >= 0) img_r[i - 8 * g.nf] = unit_elem<R>(m, e, g.recs);
    } else {
        const int k = i - 8 * (g.nf + g.nr);
        const int nfe = g.n_ftabs << g.fbits;
        if (k < nfe) phase_table_entry<R>(g.ftabs[k >> g.fbits], k & ((1 << g.fbits) - 1), g.ftabents, g.recs, img_f);
        else if (k - nfe < (g.n_rtabs << g.rbits)) {
            const int kr = k - nfe;
            phase_table_entry<R>(g.rtabs[kr >> g.rbits], kr & ((1 << g.rbits) - 1), g.rtabents, g.recs, img_r);
        }
    }
}

template <typename R>
__global__ void k_gather_units(GatherArgs g)
{
    gather_item<R>(g, blockIdx.x * blockDim.x + threadIdx.x);
}

// The images of many plans in one launch: item i belongs to the plan k with
// item_off[k] <= i < item_off[k + 1] (binary search; item_off[n] = total).
template <typename R>
__global__ void k_gather_batch(const GatherArgs *__restrict__ args, const int64_t *__restrict__ item_off, int n)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= item_off[n]) return;
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (item_off[mid] <= i) lo = mid;
        else hi = mid - 1;
    }
    gather_item<R>(args[lo], (int)(i - item_off[lo]));
}

cudaError_t launch_gather_batch(int dtype, const GatherArgs *args, const int64_t *item_off, int n, int64_t total,
                                cudaStream_t s)
{
    if (total == 0) return cudaSuccess;
    const unsigned blocks = (unsigned)((total + 255) / 256);
    if (dtype == 0) k_gather_batch<float><<<blocks, 256, 0, s>>>(args, item_off, n);
    else k_gather_batch<double><<<blocks, 256, 0, s>>>(args, item_off, n);
    return cudaGetLastError();
}

cudaError_t launch_gather_units(int dtype, const GatherArgs &g, cudaStream_t s)
{
    const int64_t total = gather_items(g);
    if (total == 0) return cudaSuccess;
    const int blocks = (int)((total + 255) / 256);
    if (dtype == 0) k_gather_units<float><<<blocks, 256, 0, s>>>(g);
    else k_gather_units<double><<<blocks, 256, 0, s>>>(g);
    return cudaGetLastError();
}

// grad[p] = sum over the slots of parameter p (slot order) of the slot's sum over tiles;
// a slot's sum takes the tiles in order within each thread, then a fixed tree, so the
// result does not depend on timing.
__global__ void k_reduce_grad(const double *__restrict__ part, int n_tiles, int stride, const int *__restrict__ ptr,
                              const int *__restrict__ slots, double *grad)
{
    __shared__ double sh[256];
    const int p = blockIdx.x;
    double total = 0.0;
    for (int i = ptr[p]; i < ptr[p + 1]; i++) {
        const int64_t s = slots[i];
        double acc = 0.0;
        for (int k = threadIdx.x; k < n_tiles; k += blockDim.x) acc += part[s * stride + k];
        sh[threadIdx.x] = acc;
        __syncthreads();
        for (int w = blockDim.x / 2; w > 0; w >>= 1) {
            if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
            __syncthreads();
        }
        total += sh[0];
        __syncthreads();
    }
    if (threadIdx.x == 0) grad[p] = total;
}

cudaError_t launch_reduce_grad(const double *slot_partials, int n_tiles, int stride, const int *csr_ptr,
                               const int *csr_slots, int n_params, double *grad, cudaStream_t s)
{
    if (n_params == 0) return cudaSuccess;
    k_reduce_grad<<<n_params, 256, 0, s>>>(slot_partials, n_tiles, stride, csr_ptr, csr_slots, grad);
    return cudaGetLastError();
}

#endif  // part 8

}  // namespace gbvqc
