// Declarations shared by the translation units of the C ABI (api_*.cu): error reporting,
// the device allocator, profiling hooks, host-side matrices and the handle types.
#pragma once

#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "gbvqc.h"
#include "kernels.h"
#include "jit.h"
#include "planner.h"

using namespace gbvqc;
typedef std::complex<double> cd;
typedef std::vector<cd> Mat;  // row-major d x d

// ------------------------------------------------------------------------ errors

// Sets the calling thread's message (gbvqc_last_error) and returns st.
gbvqc_status fail(gbvqc_status st, const char *fmt, ...);

#define CUDA_TRY(expr)                                                                       \
    do {                                                                                     \
        cudaError_t e_ = (expr);                                                             \
        if (e_ != cudaSuccess)                                                               \
            return fail(e_ == cudaErrorMemoryAllocation ? GBVQC_ERR_OOM : GBVQC_ERR_CUDA,   \
                        "%s: %s (%s:%d)", #expr, cudaGetErrorString(e_), __FILE__, __LINE__); \
    } while (0)

#define ST_TRY(expr)                      \
    do {                                  \
        gbvqc_status s_ = (expr);         \
        if (s_ != GBVQC_OK) return s_;    \
    } while (0)

// ----------------------------------------------------------------- device memory

// Every device allocation of the library goes through dev_alloc.  The environment
// variable GBVQC_DEVICE_ALLOC_LIMIT (bytes; unset = no limit) caps the library's live
// allocations: a request that would exceed it fails with GBVQC_ERR_OOM exactly like a
// failed cudaMalloc (host-side fault injection for the out-of-memory paths).
gbvqc_status dev_alloc_bytes(void **p, size_t bytes);
void dev_free(void *p);

template <typename T>
gbvqc_status dev_alloc(T **p, size_t count)
{
    void *v = nullptr;
    gbvqc_status st = dev_alloc_bytes(&v, sizeof(T) * (count == 0 ? 1 : count));
    *p = static_cast<T *>(v);
    return st;
}

template <typename T>
gbvqc_status upload(T **p, const std::vector<T> &v)
{
    ST_TRY(dev_alloc(p, v.size()));
    if (!v.empty()) CUDA_TRY(cudaMemcpy(*p, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice));
    return GBVQC_OK;
}

inline size_t amp_size(int dtype) { return dtype == GBVQC_C64 ? 8 : 16; }

// ----------------------------------------------------------------- profiling hooks

// When grad_profile is active, every launch of the gradient sequence is bracketed by
// CUDA events and tagged with its algorithmic flops and bytes.
struct ProfRec {
    std::string name;
    cudaEvent_t a, b;
    double flops, bytes;
};
extern thread_local std::vector<ProfRec> *g_prof;

template <typename F>
gbvqc_status run_k(const char *name, double flops, double bytes, cudaStream_t s, F &&launch)
{
    if (!g_prof) {
        CUDA_TRY(launch());
        return GBVQC_OK;
    }
    ProfRec r{name, nullptr, nullptr, flops, bytes};
    CUDA_TRY(cudaEventCreate(&r.a));
    CUDA_TRY(cudaEventCreate(&r.b));
    CUDA_TRY(cudaEventRecord(r.a, s));
    CUDA_TRY(launch());
    CUDA_TRY(cudaEventRecord(r.b, s));
    g_prof->push_back(r);
    return GBVQC_OK;
}

// Real floating-point operations per amplitude of one matrix application.
double shape_flops(int sh);

// ------------------------------------------------------------------ host matrices

Mat mat_from(const double *m, int d);
void mat_to(const Mat &M, double *m);
Mat mat_dagger(const Mat &M, int d);
Mat mat_conj(const Mat &M);
bool mat_inverse(const Mat &A, int d, Mat &out);
bool is_channel(int kind);
bool is_channel2(int kind);
bool is_rotation(int kind);
int kind_qubits(int kind);
Mat gate_matrix(const gbvqc_op &op);
std::vector<Mat> channel_kraus(int kind, double g, const double *kraus, int n_kraus);
std::vector<Mat> channel_kraus2(int kind, double g, const double *kraus, int n_kraus);
Mat superop2(const std::vector<Mat> &ks);
Mat superop(const std::vector<Mat> &ks);
int classify(const Mat &M);
int perm_bits(const Mat &M);
int join_shape(int a, int b);
int ftype_of(int sh);

// ------------------------------------------------------------------- handle types

struct gbvqc_sv {
    int n_log = 0, n_phys = 0, dtype = 0, density = 0;
    void *data = nullptr;
    bool owned = false;
    cudaStream_t stream = nullptr;
    double *d_scratch = nullptr;   // kMaxRedBlocks partials + result
    unsigned *d_counter = nullptr;
    MatRec *d_rec = nullptr;       // matrix of apply_channel
    size_t amps() const { return size_t(1) << n_phys; }
    size_t bytes() const { return amps() * (dtype == GBVQC_C64 ? 8 : 16); }
};

struct gbvqc_obs {
    int n_qubits = 0;
    std::vector<ObsGroup> groups;
    std::vector<ObsTerm> terms;
    ObsGroup *d_groups = nullptr;
    ObsTerm *d_terms = nullptr;
    unsigned char *d_chunk = nullptr;  // chunked kernels' staging image (chunk_image)
    ObsDev dev() const { return ObsDev{d_groups, d_terms, (int)groups.size(), (int)terms.size(), d_chunk}; }
    // device copies with the X/Z masks permuted to a gradient layout (key: the layout)
    struct PermDev {
        ObsGroup *groups;
        ObsTerm *terms;
        unsigned char *chunk;
    };
    std::map<std::vector<int8_t>, PermDev> perm_dev;
};
// Staging image of the chunked Pauli kernels for a grouped observable (layout in kernels.h).
std::vector<unsigned char> chunk_image(const std::vector<ObsGroup> &groups, const std::vector<ObsTerm> &terms);

// One gate of the per-gate schedule.
struct PlainGate {
    int shape, q0, q1;
    int rec_f, rec_i, rec_a;
    int der_k, dq0, dq1, rec_d;  // derivative operator (rec_d = -1 if none)
    int param;
    double gscale;
    int slot;
    // SH_DENSE4 (two-qubit channel superoperator): qubits 3 and 4 of the matrix
    int q2 = 0, q3 = 0;
    // further derivatives of the same gate (variational FSIM parameters after the first)
    int n_extra = 0;
    int ex_rec[4] = {-1, -1, -1, -1}, ex_param[4] = {-1, -1, -1, -1}, ex_slot[4] = {-1, -1, -1, -1};
};

struct Workspace {
    int dtype = -1;
    void *phi = nullptr, *psi = nullptr;
    double *d_theta = nullptr, *d_energy = nullptr, *d_grad = nullptr, *d_slot_grad = nullptr;
    double *d_slot_partials = nullptr;
    double *d_red = nullptr;
    unsigned *d_counter = nullptr;
};

struct DevPlan {  // a FusedPlan and its device copies (uploaded on first launch)
    FusedPlan p;
    std::vector<int8_t> perm;  // pure gradient plans: physical qubit of logical q (empty: identity)
    bool uploaded = false;
    int elem = 4;
    std::vector<size_t> fwd_smem, rev_smem;
    PassDesc *d_fwd = nullptr, *d_rev = nullptr;
    SubRun *d_fsubs = nullptr, *d_rsubs = nullptr;
    FGate *d_fgates = nullptr, *d_rgates = nullptr;
    DEnt *d_fents = nullptr, *d_rents = nullptr;
    MatUnit *d_funits = nullptr, *d_runits = nullptr;
    void *d_fimg = nullptr, *d_rimg = nullptr;  // per-step matrix images of the unit lists
    TabDesc *d_ftabs = nullptr, *d_rtabs = nullptr;     // register phase tables (table-mode blocks)
    TabEnt *d_ftabents = nullptr, *d_rtabents = nullptr;
    int *d_csr_ptr = nullptr, *d_csr_slots = nullptr;
    std::unique_ptr<JitPlan> jit;  // specialised passes (GBVQC_MODE_JIT), built on first use
    // code prefetch of the specialised passes: one side stream and completion event per
    // kernel, forked from the gradient sequence's stream at its start and joined at its end
    std::vector<cudaStream_t> pf_streams;
    std::vector<cudaEvent_t> pf_done;
    cudaEvent_t pf_fork = nullptr;
};

struct gbvqc_circuit {
    int n_log = 0, n_phys = 0, n_params = 0, density = 0;
    std::vector<gbvqc_op> ops;
    std::vector<std::vector<double>> kraus_store;  // copies of the KRAUS2 operator lists
    std::vector<MatRec> recs;
    std::vector<DynRec> dyn;
    MatRec *d_recs = nullptr;
    DynRec *d_dyn = nullptr;
    // per-gate schedule (standard layout)
    std::vector<PlainGate> plain;
    int plain_slots = 0;
    int *d_plain_ptr = nullptr, *d_plain_slots = nullptr;
    // fused: physical gate lists for the standard and the grad layout
    std::vector<PGate> pg_std, pg_grad;
    DensMap map_std{}, map_grad{};
    int tile_qubits = 0, low_qubits = 0;
    std::map<int, std::unique_ptr<DevPlan>> plans;  // key: dtype*2 + (grad layout)
    Workspace ws;
    cudaStream_t cap_stream = nullptr;
    std::map<int, cudaGraphExec_t> graphs;           // key: dtype*4 + mode
    const void *graph_obs = nullptr;                 // observable the graphs were captured with
    int n_param_ops = 0;                             // ops driven by a parameter
    size_t partials_cap = 0;                         // doubles in ws.d_slot_partials
    bool dev_ready = false;                          // records, CSR and stream on the device
    std::vector<int> plain_slot_param;
    std::mutex mu;
};

// ------------------------------------------------------------- states, observables

gbvqc_status ensure_obs(gbvqc_obs *h);
// The observable in a permuted qubit layout (device copies made once per layout; call
// outside stream capture).
gbvqc_status obs_dev_perm(gbvqc_obs *h, const std::vector<int8_t> &perm, ObsDev *out);
DensMap standard_map(int n);
DensMap interleaved_map(int n);

// ------------------------------------------------------------------------ circuits

void free_graphs(gbvqc_circuit *c);
gbvqc_status csr_upload(const std::vector<int> &slot_param, int n_params, int **d_ptr, int **d_slots);
// Device copies of the circuit's records, dynamic-record list and per-gate CSR.
gbvqc_status ensure_device(gbvqc_circuit *c);
// Largest tile the fused kernels take for dtype.
int max_tile(int dtype);
// Fused plan for (dtype, layout), host side only (no GPU needed); batch: the plan of a
// batch member; jit: the plan of the specialised passes (its own register-qubit counts).
gbvqc_status get_host_plan(gbvqc_circuit *c, int dtype, bool grad_layout, DevPlan **out, bool batch = false,
                           bool jit = false);
// The same with its device copies.
gbvqc_status get_plan(gbvqc_circuit *c, int dtype, bool grad_layout, DevPlan **out, bool batch = false,
                      bool jit = false);
bool fused_supported(const gbvqc_circuit *c, int dtype);
double state_bytes(const gbvqc_circuit *c, int dtype);
