// Fused tile-pass kernels of one circuit (one CTA per tile) and their launchers.  The
// tile-pass body lives in fused_tile.cuh.
#include "fused_tile.cuh"

namespace gbvqc {

// Forward kernels run 2^(t-NR) <= 128 threads (three CTAs per SM), reverse kernels
// <= 256 threads (two CTAs per SM).
template <typename R, int NR, bool REV, bool TWOQ>
__global__ void __launch_bounds__(REV ? 256 : 128, REV ? 2 : 3) k_fused(typename CT<R>::T *__restrict__ phi,
                                                                        typename CT<R>::T *__restrict__ psi,
                                                                        FusedArgs args)
{
    fused_tile<R, NR, REV, TWOQ>(phi, psi, args, blockIdx.x);
}

// -------------------------------------------------------------------------- launchers

int fused_nr(int dtype, bool reverse)
{
    if (dtype == 0) return reverse ? 4 : 5;
    return reverse ? 3 : 4;
}

// Opt the fused kernels in to large dynamic shared memory (call outside stream capture).
template <typename R, int NR, bool REV>
static cudaError_t prepare_pair()
{
    const int bytes = 200 * 1024;
    cudaError_t e = cudaFuncSetAttribute(k_fused<R, NR, REV, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_fused<R, NR, REV, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    return e;
}

cudaError_t fused_prepare()
{
    cudaError_t e = prepare_pair<float, 5, false>();
    if (e == cudaSuccess) e = prepare_pair<float, 4, true>();
    if (e == cudaSuccess) e = prepare_pair<double, 4, false>();
    if (e == cudaSuccess) e = prepare_pair<double, 3, true>();
    return e;
}

template <typename R, int NR, bool REV>
static cudaError_t fused_launch(void *phi, void *psi, const PassDesc &ph, size_t smem, FusedArgs args,
                                cudaStream_t s)
{
    typedef typename CT<R>::T T;
    const int threads = 1 << (ph.t - NR);
    const int64_t tiles = int64_t(1) << (ph.n - ph.t);
    if (ph.has_2q)
        k_fused<R, NR, REV, true><<<(unsigned)tiles, threads, smem, s>>>((T *)phi, (T *)psi, args);
    else
        k_fused<R, NR, REV, false><<<(unsigned)tiles, threads, smem, s>>>((T *)phi, (T *)psi, args);
    return cudaGetLastError();
}

cudaError_t launch_fused_forward(int dtype, void *psi, const FusedDev &fd, int pass, const PassDesc &ph,
                                 size_t smem, cudaStream_t s)
{
    FusedArgs args{fd.passes + pass, fd.subs, fd.gates, fd.ents, fd.units, fd.recs, fd.img, nullptr, 0};
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

template <typename R>
__global__ void k_gather_units(const MatUnit *__restrict__ fu, int nf, R *img_f, const MatUnit *__restrict__ ru,
                               int nr, R *img_r, const MatRec *__restrict__ recs)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int u = i >> 3, e = i & 7;
    if (u < nf) {
        const MatUnit m = fu[u];
        img_f[i] = mat_of<R>(&recs[m.rec])[8 * m.part + e];
    } else if (u < nf + nr) {
        const MatUnit m = ru[u - nf];
        img_r[i - 8 * nf] = mat_of<R>(&recs[m.rec])[8 * m.part + e];
    }
}

cudaError_t launch_gather_units(int dtype, const MatUnit *fu, int nf, void *img_f, const MatUnit *ru, int nr,
                                void *img_r, const MatRec *recs, cudaStream_t s)
{
    const int total = 8 * (nf + nr);
    if (total == 0) return cudaSuccess;
    const int blocks = (total + 255) / 256;
    if (dtype == 0) k_gather_units<float><<<blocks, 256, 0, s>>>(fu, nf, (float *)img_f, ru, nr, (float *)img_r, recs);
    else k_gather_units<double><<<blocks, 256, 0, s>>>(fu, nf, (double *)img_f, ru, nr, (double *)img_r, recs);
    return cudaGetLastError();
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
