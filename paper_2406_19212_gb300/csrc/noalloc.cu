// expect_noalloc: the Pauli-sum expectation value of a pure state for callers that must
// not allocate device memory.
//
// Some callers cannot call cudaMalloc: code running while a stream is being captured
// into a CUDA graph (allocation is not a stream operation and is refused or unsafe
// during global-mode capture), applications whose framework owns the whole device
// memory budget through its own pool and forbids allocations from libraries, and
// latency-critical loops that cannot absorb an allocation's implicit synchronisation.
// This entry point serves them: the caller passes the state and the output, the Pauli
// terms travel as kernel parameters, and the only scratch (per-block partial sums and an
// arrival counter) lives in a file-scope __device__ array of fixed size that every GPU
// loading the library keeps until the process exits.
//
// The array is shared by every call: calls whose kernels overlap on the GPU race on it,
// so callers must order them (one stream, or events).  The arrival counter is cleared
// on the stream before every launch; the partial sums are overwritten before use.
#include <cuda_runtime.h>

#include <cstdint>
#include <algorithm>
#include <cstdio>
#include <map>
#include <mutex>

#include "gbvqc.h"

// Sets the thread's gbvqc_last_error() message (defined with the other entry points).
void gbvqc_internal_set_error(const char *msg);

namespace {

constexpr int kNaMaxTerms = 64;      // Pauli terms accepted (kernel-parameter space)
constexpr int kNaMaxBlocks = 608;    // reduction blocks at most: 4 per SM up to 152 SMs (the launch
                                     // takes 4 per SM of the device, capped here)
constexpr int kNaThreads = 256;

// Scratch: [0, 256) arrival counter, [256, 256 + 8 * kNaMaxBlocks) block partials.
constexpr size_t kNaScratchBytes = 256 + sizeof(double) * kNaMaxBlocks;
static __device__ __align__(256) unsigned char g_na_scratch[kNaScratchBytes];

struct NaTerm {
    double coeff;
    uint64_t z;
    int32_t ph;
    int32_t pad;
};
struct NaGroup {
    uint64_t x;
    int32_t t_begin, t_end;
};
struct NaObs {  // passed by value: 64 * (24 + 16) + 8 bytes
    NaGroup groups[kNaMaxTerms];
    NaTerm terms[kNaMaxTerms];
    int n_groups;
    int pad;
};

template <typename R> struct NaC;
template <> struct NaC<float> { typedef float2 T; };
template <> struct NaC<double> { typedef double2 T; };

__device__ __forceinline__ double na_warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ double na_block_sum(double v)
{
    __shared__ double sh[32];
    v = na_warp_sum(v);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
    __syncthreads();
    if (l == 0) sh[w] = v;
    __syncthreads();
    double r = 0.0;
    if (w == 0) {
        r = l < nw ? sh[l] : 0.0;
        r = na_warp_sum(r);
    }
    return r;
}

// E = Re sum_a conj(psi_a) (H psi)_a with (H psi)_a = sum_g c_g(a ^ x_g) psi_{a ^ x_g}.
template <typename R>
__global__ void __launch_bounds__(kNaThreads) k_expect_noalloc(const typename NaC<R>::T *__restrict__ psi,
                                                               int64_t len, const __grid_constant__ NaObs obs,
                                                               unsigned char *scratch, double *out)
{
    typedef typename NaC<R>::T T;
    unsigned *counter = reinterpret_cast<unsigned *>(scratch);
    double *partials = reinterpret_cast<double *>(scratch + 256);
    double acc = 0.0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; a < len; a += stride) {
        const T pa = psi[a];
        R lr = 0, li = 0;
        for (int g = 0; g < obs.n_groups; g++) {
            const uint64_t b = (uint64_t)a ^ obs.groups[g].x;
            const T pb = obs.groups[g].x ? psi[b] : pa;
            R cr = 0, ci = 0;
            for (int k = obs.groups[g].t_begin; k < obs.groups[g].t_end; k++) {
                R c = (R)obs.terms[k].coeff;
                if (__popcll(b & obs.terms[k].z) & 1) c = -c;
                switch (obs.terms[k].ph & 3) {
                case 0: cr += c; break;
                case 1: ci += c; break;
                case 2: cr -= c; break;
                default: ci -= c; break;
                }
            }
            lr += cr * pb.x - ci * pb.y;
            li += cr * pb.y + ci * pb.x;
        }
        acc += (double)(pa.x * lr + pa.y * li);
    }
    __shared__ bool last;
    const double bsum = na_block_sum(acc);
    if (threadIdx.x == 0) {
        partials[blockIdx.x] = bsum;
        __threadfence();
        last = atomicAdd(counter, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    double s = 0.0;
    for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) s += __ldcg(&partials[i]);
    s = na_block_sum(s);
    if (threadIdx.x == 0) {
        *out = s;
        *counter = 0u;
    }
}

gbvqc_status na_fail(gbvqc_status st, const char *msg)
{
    gbvqc_internal_set_error(msg);
    return st;
}

// Device address of the scratch array and the device's SM count, looked up once per
// device with that device current (the host-side symbol is only a stand-in, not a device
// address).
gbvqc_status na_scratch_address(unsigned char **ptr, int *sms)
{
    static std::mutex mu;
    static std::map<int, std::pair<unsigned char *, int>> addr;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return na_fail(GBVQC_ERR_CUDA, "expect_noalloc: no CUDA device");
    std::lock_guard<std::mutex> lk(mu);
    auto it = addr.find(dev);
    if (it == addr.end()) {
        void *p = nullptr;
        int n_sm = 0;
        cudaError_t e = cudaGetSymbolAddress(&p, g_na_scratch);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess || !p) {
            char msg[200];
            snprintf(msg, sizeof msg, "expect_noalloc: device set-up failed: %s", cudaGetErrorString(e));
            return na_fail(GBVQC_ERR_CUDA, msg);
        }
        it = addr.emplace(dev, std::make_pair(static_cast<unsigned char *>(p), n_sm)).first;
    }
    *ptr = it->second.first;
    *sms = it->second.second;
    return GBVQC_OK;
}

}  // namespace

extern "C" gbvqc_status expect_noalloc(const void *psi_device, int n_qubits, int dtype, const gbvqc_pauli *terms,
                                       int n_terms, void *stream, double *energy_device)
{
    if (!psi_device || !energy_device || (!terms && n_terms > 0))
        return na_fail(GBVQC_ERR_ARG, "expect_noalloc: NULL argument");
    if (dtype != GBVQC_C64 && dtype != GBVQC_C128) return na_fail(GBVQC_ERR_ARG, "expect_noalloc: bad dtype");
    if (n_qubits < 1 || n_qubits > 34) return na_fail(GBVQC_ERR_ARG, "expect_noalloc: qubit count out of range");
    if (n_terms < 0 || n_terms > kNaMaxTerms)
        return na_fail(GBVQC_ERR_ARG, "expect_noalloc: more than 64 Pauli terms (the no-allocation maximum)");
    if (((uintptr_t)psi_device) & 15) return na_fail(GBVQC_ERR_ARG, "expect_noalloc: state not 16-byte aligned");
    const uint64_t valid = (uint64_t(1) << n_qubits) - 1;
    NaObs obs{};
    // group the terms by X mask (fixed-size arrays on the host stack)
    int used[kNaMaxTerms] = {0};
    int nt = 0;
    for (int i = 0; i < n_terms; i++) {
        if ((terms[i].x_mask | terms[i].z_mask) & ~valid)
            return na_fail(GBVQC_ERR_ARG, "expect_noalloc: a term touches a qubit >= n_qubits");
        if (used[i]) continue;
        NaGroup &g = obs.groups[obs.n_groups++];
        g.x = terms[i].x_mask;
        g.t_begin = nt;
        for (int j = i; j < n_terms; j++)
            if (!used[j] && terms[j].x_mask == g.x) {
                used[j] = 1;
                NaTerm &t = obs.terms[nt++];
                t.coeff = terms[j].coeff;
                t.z = terms[j].z_mask;
                t.ph = __builtin_popcountll(terms[j].x_mask & terms[j].z_mask) & 3;
            }
        g.t_end = nt;
    }
    unsigned char *scratch = nullptr;
    int sms = 0;
    gbvqc_status st = na_scratch_address(&scratch, &sms);
    if (st != GBVQC_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaMemsetAsync(scratch, 0, sizeof(unsigned), s);  // arrival counter starts at zero
    if (e != cudaSuccess) return na_fail(GBVQC_ERR_CUDA, cudaGetErrorString(e));
    const int64_t len = int64_t(1) << n_qubits;
    int64_t blocks = (len + kNaThreads - 1) / kNaThreads;
    const int max_blocks = std::max(1, std::min(kNaMaxBlocks, 4 * sms));
    if (blocks > max_blocks) blocks = max_blocks;
    if (dtype == GBVQC_C64)
        k_expect_noalloc<float><<<(int)blocks, kNaThreads, 0, s>>>((const float2 *)psi_device, len, obs, scratch,
                                                                   energy_device);
    else
        k_expect_noalloc<double><<<(int)blocks, kNaThreads, 0, s>>>((const double2 *)psi_device, len, obs, scratch,
                                                                    energy_device);
    e = cudaGetLastError();
    if (e != cudaSuccess) return na_fail(GBVQC_ERR_CUDA, cudaGetErrorString(e));
    return GBVQC_OK;
}
