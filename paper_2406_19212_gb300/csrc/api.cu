// C ABI of libgbvqc (declared in include/gbvqc.h): states, circuits, observables,
// apply / expect / grad.  Host-side gate matrices, structural classification, the
// per-gate (plain) schedule, the fused tile schedule and CUDA-graph replay of grad.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <iomanip>
#include <map>
#include <sstream>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include <sys/stat.h>

#include "gbvqc.h"
#include "kernels.h"
#include "planner.h"

static void mkdir_quiet(const char *p) { mkdir(p, 0755); }

using namespace gbvqc;
typedef std::complex<double> cd;

// ------------------------------------------------------------------------ errors

static thread_local std::string g_last_error;

static gbvqc_status fail(gbvqc_status st, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return st;
}

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

// ----------------------------------------------------------------- profiling hooks

// When grad_profile is active, every launch of the gradient sequence is bracketed by
// CUDA events and tagged with its algorithmic flops and bytes.
struct ProfRec {
    std::string name;
    cudaEvent_t a, b;
    double flops, bytes;
};
static thread_local std::vector<ProfRec> *g_prof = nullptr;

template <typename F>
static gbvqc_status run_k(const char *name, double flops, double bytes, cudaStream_t s, F &&launch)
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
static double shape_flops(int sh)
{
    switch (sh) {
    case SH_DENSE1: return 14;  // two complex products and a sum per output
    case SH_DENSE2: return 30;  // four complex products and three sums per output
    case SH_CTRL2: return 7;    // a dense 2x2 on half of the amplitudes
    case SH_BLOCK2: return 10;  // a dense 2x2 on half, one phase on each remaining quarter
    case SH_IMAG1: return 6;    // two real products and a sum per output
    case SH_DENSE4: return 126; // sixteen complex products and fifteen sums per output
    case SH_PAR2: return 14;    // a dense 2x2 on every amplitude pair
    case SH_CX: return 0;      // data movement only
    case SH_CZ: return 0.5;    // a sign on a quarter of the amplitudes
    case SH_REAL1: return 6;
    default: return 6;          // one complex product
    }
}

// ------------------------------------------------------------------ host matrices

typedef std::vector<cd> Mat;  // row-major d x d

static Mat mat_from(const double *m, int d)
{
    Mat M(d * d);
    for (int i = 0; i < d * d; i++) M[i] = cd(m[2 * i], m[2 * i + 1]);
    return M;
}

static void mat_to(const Mat &M, double *m)
{
    for (int i = 0; i < 32; i++) m[i] = 0.0;
    for (size_t i = 0; i < M.size(); i++) {
        m[2 * i] = M[i].real();
        m[2 * i + 1] = M[i].imag();
    }
}

static Mat mat_dagger(const Mat &M, int d)
{
    Mat D(d * d);
    for (int r = 0; r < d; r++)
        for (int c = 0; c < d; c++) D[r * d + c] = std::conj(M[c * d + r]);
    return D;
}

static Mat mat_conj(const Mat &M)
{
    Mat D(M.size());
    for (size_t i = 0; i < M.size(); i++) D[i] = std::conj(M[i]);
    return D;
}

// Inverse by Gauss-Jordan elimination with partial pivoting (channels are not unitary).
static bool mat_inverse(const Mat &A, int d, Mat &out)
{
    std::vector<cd> m(d * 2 * d);
    for (int r = 0; r < d; r++)
        for (int c = 0; c < 2 * d; c++) m[r * 2 * d + c] = c < d ? A[r * d + c] : cd(c - d == r ? 1 : 0);
    for (int k = 0; k < d; k++) {
        int piv = k;
        for (int r = k + 1; r < d; r++)
            if (std::abs(m[r * 2 * d + k]) > std::abs(m[piv * 2 * d + k])) piv = r;
        if (std::abs(m[piv * 2 * d + k]) < 1e-14) return false;
        for (int c = 0; c < 2 * d; c++) std::swap(m[k * 2 * d + c], m[piv * 2 * d + c]);
        cd p = m[k * 2 * d + k];
        for (int c = 0; c < 2 * d; c++) m[k * 2 * d + c] /= p;
        for (int r = 0; r < d; r++)
            if (r != k) {
                cd f = m[r * 2 * d + k];
                for (int c = 0; c < 2 * d; c++) m[r * 2 * d + c] -= f * m[k * 2 * d + c];
            }
    }
    out.assign(d * d, 0);
    for (int r = 0; r < d; r++)
        for (int c = 0; c < d; c++) out[r * d + c] = m[r * 2 * d + d + c];
    return true;
}

static bool is_channel(int kind) { return kind >= GBVQC_DEPOL && kind <= GBVQC_KRAUS2; }
static bool is_channel2(int kind) { return kind == GBVQC_DEPOL2 || kind == GBVQC_KRAUS2; }
static bool is_rotation(int kind) { return kind == GBVQC_RX || kind == GBVQC_RY || kind == GBVQC_RZ; }
static int kind_qubits(int kind)
{
    return (kind >= GBVQC_CNOT && kind <= GBVQC_CONTROL) || kind == GBVQC_DENSE2 || is_channel2(kind) ? 2 : 1;
}

// Matrix of a unitary op with its fixed parameters (Sec. II.B); rotations use params[0].
static Mat gate_matrix(const gbvqc_op &op)
{
    const double r2 = 1.0 / std::sqrt(2.0);
    const cd I(0, 1);
    if (is_rotation(op.kind)) {
        double m[8];
        rot2(op.kind - GBVQC_RX, VAR_FWD, op.params[0], m);
        return mat_from(m, 2);
    }
    switch (op.kind) {
    case GBVQC_X: return {0, 1, 1, 0};
    case GBVQC_Y: return {0, -I, I, 0};
    case GBVQC_Z: return {1, 0, 0, -1};
    case GBVQC_H: return {r2, r2, r2, -r2};
    case GBVQC_S: return {1, 0, 0, I};
    case GBVQC_T: return {1, 0, 0, std::exp(I * (M_PI / 4))};
    case GBVQC_SX: return {cd(0.5, 0.5), cd(0.5, -0.5), cd(0.5, -0.5), cd(0.5, 0.5)};
    case GBVQC_SY: return {cd(0.5, 0.5), cd(-0.5, -0.5), cd(0.5, 0.5), cd(0.5, 0.5)};
    case GBVQC_SW: return {cd(0.5, 0.5), cd(0, -r2), cd(r2, 0), cd(0.5, 0.5)};
    case GBVQC_DENSE1: return mat_from(op.data, 2);
    default: break;
    }
    Mat M(16, 0);
    auto at = [&](int r, int c) -> cd & { return M[r * 4 + c]; };
    switch (op.kind) {
    case GBVQC_CNOT:  // control = qubits[0] (matrix bit 0), target = qubits[1]
        at(0, 0) = 1; at(2, 2) = 1; at(1, 3) = 1; at(3, 1) = 1;
        break;
    case GBVQC_CZ: at(0, 0) = 1; at(1, 1) = 1; at(2, 2) = 1; at(3, 3) = -1; break;
    case GBVQC_SWAP: at(0, 0) = 1; at(1, 2) = 1; at(2, 1) = 1; at(3, 3) = 1; break;
    case GBVQC_ISWAP: at(0, 0) = 1; at(1, 2) = I; at(2, 1) = I; at(3, 3) = 1; break;
    case GBVQC_FSIM: {  // Eq. (FSIM)
        double th = op.params[0], ph = op.params[1], dp = op.params[2], dm = op.params[3],
               dmo = op.params[4];
        at(0, 0) = 1;
        at(1, 1) = std::exp(I * (dp + dm)) * std::cos(th);
        at(1, 2) = -I * std::exp(I * (dp - dmo)) * std::sin(th);
        at(2, 1) = -I * std::exp(I * (dp + dmo)) * std::sin(th);
        at(2, 2) = std::exp(I * (dp - dm)) * std::cos(th);
        at(3, 3) = std::exp(I * (2 * dp - ph));
        break;
    }
    case GBVQC_CONTROL:
        at(0, 0) = 1; at(2, 2) = 1;
        at(1, 1) = cd(op.data[0], op.data[1]);
        at(1, 3) = cd(op.data[2], op.data[3]);
        at(3, 1) = cd(op.data[4], op.data[5]);
        at(3, 3) = cd(op.data[6], op.data[7]);
        break;
    case GBVQC_DENSE2: return mat_from(op.data, 4);
    default: break;
    }
    return M;
}

// Kraus operators of a single-qubit channel (Sec. II.B; depolarising with p/4 weights).
static std::vector<Mat> channel_kraus(int kind, double g, const double *kraus, int n_kraus)
{
    const cd I(0, 1);
    switch (kind) {
    case GBVQC_AMPDAMP: return {{1, 0, 0, std::sqrt(1 - g)}, {0, std::sqrt(g), 0, 0}};
    case GBVQC_PHASEDAMP: return {{1, 0, 0, std::sqrt(1 - g)}, {0, 0, 0, std::sqrt(g)}};
    case GBVQC_DEPOL: {
        double a = std::sqrt(1 - 0.75 * g), b = std::sqrt(0.25 * g);
        return {{a, 0, 0, a}, {0, b, b, 0}, {0, -I * b, I * b, 0}, {b, 0, 0, -b}};
    }
    default: {
        std::vector<Mat> ks;
        for (int s = 0; s < n_kraus; s++) ks.push_back(mat_from(kraus + 8 * s, 2));
        return ks;
    }
    }
}

// Kraus operators (4x4, matrix bit 0 = the first qubit) of a two-qubit channel.
static std::vector<Mat> channel_kraus2(int kind, double g, const double *kraus, int n_kraus)
{
    std::vector<Mat> ks;
    if (kind == GBVQC_KRAUS2) {
        for (int s = 0; s < n_kraus; s++) ks.push_back(mat_from(kraus + 32 * s, 4));
        return ks;
    }
    const cd I(0, 1);
    const cd P[4][4] = {{1, 0, 0, 1}, {0, 1, 1, 0}, {0, -I, I, 0}, {1, 0, 0, -1}};  // I, X, Y, Z
    for (int b = 0; b < 4; b++)      // Pauli on the second qubit
        for (int a = 0; a < 4; a++) {  // Pauli on the first qubit
            const double w = (a == 0 && b == 0) ? std::sqrt(1 - 15 * g / 16) : std::sqrt(g / 16);
            Mat K(16, 0);
            for (int r = 0; r < 4; r++)
                for (int c = 0; c < 4; c++)
                    K[r * 4 + c] = w * P[a][2 * (r & 1) + (c & 1)] * P[b][2 * (r >> 1) + (c >> 1)];
            ks.push_back(K);
        }
    return ks;
}

// Superoperator of a two-qubit channel on (ket q0, ket q1, bra q0, bra q1) (matrix bits
// 0..3): S[(r + 4 r'), (c + 4 c')] = sum_s K[r][c] conj(K[r'][c']), 16 x 16.
static Mat superop2(const std::vector<Mat> &ks)
{
    Mat S(256, 0);
    for (const Mat &K : ks)
        for (int r = 0; r < 4; r++)
            for (int r2 = 0; r2 < 4; r2++)
                for (int c = 0; c < 4; c++)
                    for (int c2 = 0; c2 < 4; c2++)
                        S[(r + 4 * r2) * 16 + (c + 4 * c2)] += K[r * 4 + c] * std::conj(K[r2 * 4 + c2]);
    return S;
}

// Superoperator on (ket q, bra q): S[(r1 + 2 r2), (c1 + 2 c2)] = sum_s K[r1][c1] conj(K[r2][c2])
// (Eq. channel2 with the conjugate on the bra index: vec(K rho K^dag)).
static Mat superop(const std::vector<Mat> &ks)
{
    Mat S(16, 0);
    for (const Mat &K : ks)
        for (int r1 = 0; r1 < 2; r1++)
            for (int r2 = 0; r2 < 2; r2++)
                for (int c1 = 0; c1 < 2; c1++)
                    for (int c2 = 0; c2 < 2; c2++)
                        S[(r1 + 2 * r2) * 4 + (c1 + 2 * c2)] += K[r1 * 2 + c1] * std::conj(K[r2 * 2 + c2]);
    return S;
}

static bool nz(cd v) { return v.real() != 0.0 || v.imag() != 0.0; }

static int classify(const Mat &M)
{
    if (M.size() == 4) {
        if (!nz(M[1]) && !nz(M[2])) return SH_DIAG1;
        if (!nz(M[0]) && !nz(M[3])) return SH_ANTI1;
        bool real = true;
        for (cd v : M) real = real && v.imag() == 0.0;
        if (real) return SH_REAL1;
        const bool imag = M[0].imag() == 0.0 && M[3].imag() == 0.0 && M[1].real() == 0.0 && M[2].real() == 0.0;
        return imag ? SH_IMAG1 : SH_DENSE1;
    }
    bool diag = true;
    for (int r = 0; r < 4; r++)
        for (int c = 0; c < 4; c++)
            if (r != c && nz(M[r * 4 + c])) diag = false;
    if (diag) return M[0] == cd(1) && M[5] == cd(1) && M[10] == cd(1) && M[15] == cd(-1) ? SH_CZ : SH_DIAG2;
    // exactly CNOT with the first qubit as control (rows 1 and 3 swapped, unit entries)
    if (M[0] == cd(1) && M[10] == cd(1) && M[7] == cd(1) && M[13] == cd(1)) {
        int others = 0;
        for (int i = 0; i < 16; i++) others += nz(M[i]);
        if (others == 4) return SH_CX;
    }
    // controlled: identity on the q0 = 0 block (indices 0, 2), no coupling to 1, 3
    bool ctrl = M[0] == cd(1) && M[10] == cd(1) && !nz(M[2]) && !nz(M[8]);
    for (int r : {0, 2})
        for (int c : {1, 3}) ctrl = ctrl && !nz(M[r * 4 + c]) && !nz(M[c * 4 + r]);
    if (ctrl) return SH_CTRL2;
    bool perm = true;
    for (int r = 0; r < 4 && perm; r++) {
        int cnt = 0, cntc = 0;
        for (int c = 0; c < 4; c++) {
            cnt += nz(M[r * 4 + c]);
            cntc += nz(M[c * 4 + r]);
        }
        perm = cnt == 1 && cntc == 1;
    }
    if (perm) return SH_PERM2;
    // block: only (0,0), (3,3) and the 2x2 on rows/columns {1, 2} are non-zero
    bool block = true;
    for (int r = 0; r < 4; r++)
        for (int c = 0; c < 4; c++) {
            const bool inside = (r == c && (r == 0 || r == 3)) || ((r == 1 || r == 2) && (c == 1 || c == 2));
            if (!inside && nz(M[r * 4 + c])) block = false;
        }
    if (block) return SH_BLOCK2;
    // parity-preserving: entry (r, c) is zero unless r ^ c is 0 or 3, i.e. |00> couples
    // only to |11> and |01> only to |10>
    bool par = true, real = true;
    for (int r = 0; r < 4; r++)
        for (int c = 0; c < 4; c++) {
            if (((r ^ c) == 1 || (r ^ c) == 2) && nz(M[r * 4 + c])) par = false;
            real = real && M[r * 4 + c].imag() == 0.0;
        }
    if (par) return real ? SH_RPAR2 : SH_PAR2;
    return SH_DENSE2;
}

static int perm_bits(const Mat &M)
{
    int bits = 0;
    for (int r = 0; r < 4; r++)
        for (int c = 0; c < 4; c++)
            if (nz(M[r * 4 + c])) bits |= c << (2 * r);
    return bits;
}

// Shape that covers two matrices (reverse sweeps apply different matrices to Phi, Psi).
static int join_shape(int a, int b)
{
    if (a == b) return a;
    if (shape_qubits(a) == 1) return SH_DENSE1;
    auto par = [](int s) { return s == SH_DIAG2 || s == SH_BLOCK2 || s == SH_PAR2 || s == SH_RPAR2; };
    return par(a) && par(b) ? SH_PAR2 : SH_DENSE2;
}

static int ftype_of(int sh)
{
    switch (sh) {
    case SH_DENSE1: return FT_DENSE1;
    case SH_REAL1: return FT_REAL1;
    case SH_ANTI1: return FT_ANTI1;
    case SH_DIAG1: return FT_DIAG1;
    case SH_DENSE2: return FT_DENSE2;
    case SH_DIAG2: return FT_DIAG2;
    case SH_PERM2: return FT_PERM2;
    case SH_BLOCK2: return FT_BLOCK2;
    case SH_IMAG1: return FT_IMAG1;
    case SH_CZ: return FT_DIAG2;
    case SH_PAR2: return FT_PAR2;
    case SH_RPAR2: return FT_RPAR2;
    default: return FT_CTRL2;
    }
}

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
    ObsDev dev() const { return ObsDev{d_groups, d_terms, (int)groups.size(), (int)terms.size()}; }
    // device copies with the X/Z masks permuted to a gradient layout (key: the layout)
    std::map<std::vector<int8_t>, std::pair<ObsGroup *, ObsTerm *>> perm_dev;
};

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
    int *d_csr_ptr = nullptr, *d_csr_slots = nullptr;
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
    std::map<int, cudaGraphExec_t> graphs;           // key: dtype*2 + mode
    const void *graph_obs = nullptr;                 // observable the graphs were captured with
    int n_param_ops = 0;                             // ops driven by a parameter
    size_t partials_cap = 0;                         // doubles in ws.d_slot_partials
    bool dev_ready = false;                          // records, CSR and stream on the device
    std::vector<int> plain_slot_param;
    std::mutex mu;
};

// ------------------------------------------------------------------------- basics

extern "C" const char *gbvqc_last_error(void) { return g_last_error.c_str(); }
void gbvqc_internal_set_error(const char *msg) { g_last_error = msg; }
extern "C" int gbvqc_version(void) { return 100; }

static size_t amp_size(int dtype) { return dtype == GBVQC_C64 ? 8 : 16; }

template <typename T>
static gbvqc_status dev_alloc(T **p, size_t count)
{
    *p = nullptr;
    if (count == 0) count = 1;
    cudaError_t e = cudaMalloc((void **)p, sizeof(T) * count);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return fail(e == cudaErrorMemoryAllocation ? GBVQC_ERR_OOM : GBVQC_ERR_CUDA,
                    "cudaMalloc of %zu bytes: %s", sizeof(T) * count, cudaGetErrorString(e));
    }
    return GBVQC_OK;
}

template <typename T>
static gbvqc_status upload(T **p, const std::vector<T> &v)
{
    ST_TRY(dev_alloc(p, v.size()));
    if (!v.empty()) CUDA_TRY(cudaMemcpy(*p, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice));
    return GBVQC_OK;
}

static gbvqc_status sv_init_common(gbvqc_sv *s)
{
    ST_TRY(dev_alloc(&s->d_scratch, kMaxRedBlocks + 8));
    ST_TRY(dev_alloc(&s->d_counter, 1));
    ST_TRY(dev_alloc(&s->d_rec, 1));
    CUDA_TRY(cudaMemset(s->d_counter, 0, sizeof(unsigned)));
    return GBVQC_OK;
}

static void sv_release(gbvqc_sv *s)
{
    if (!s) return;
    if (s->owned && s->data) cudaFree(s->data);
    if (s->d_scratch) cudaFree(s->d_scratch);
    if (s->d_counter) cudaFree(s->d_counter);
    if (s->d_rec) cudaFree(s->d_rec);
    delete s;
}

static gbvqc_status check_state_args(int n_qubits, int dtype, int is_density)
{
    if (dtype != GBVQC_C64 && dtype != GBVQC_C128) return fail(GBVQC_ERR_ARG, "dtype %d", dtype);
    int np = is_density ? 2 * n_qubits : n_qubits;
    if (n_qubits < 1 || np > 34) return fail(GBVQC_ERR_ARG, "qubit count %d out of range", n_qubits);
    return GBVQC_OK;
}

extern "C" gbvqc_status sv_alloc(int n_qubits, int dtype, int is_density, void *stream, sv_handle *out)
{
    if (!out) return fail(GBVQC_ERR_ARG, "out is NULL");
    *out = nullptr;
    ST_TRY(check_state_args(n_qubits, dtype, is_density));
    gbvqc_sv *s = new gbvqc_sv();
    s->n_log = n_qubits;
    s->n_phys = is_density ? 2 * n_qubits : n_qubits;
    s->dtype = dtype;
    s->density = is_density ? 1 : 0;
    s->stream = (cudaStream_t)stream;
    s->owned = true;
    gbvqc_status st = dev_alloc((unsigned char **)&s->data, s->bytes());
    if (st == GBVQC_OK) st = sv_init_common(s);
    if (st == GBVQC_OK) {
        cudaError_t e = launch_zero_state(dtype, s->data, s->n_phys, s->stream);
        if (e != cudaSuccess) st = fail(GBVQC_ERR_CUDA, "zero state: %s", cudaGetErrorString(e));
    }
    if (st != GBVQC_OK) {
        sv_release(s);
        return st;
    }
    *out = s;
    return GBVQC_OK;
}

extern "C" gbvqc_status sv_wrap(void *device_ptr, int n_qubits, int dtype, int is_density, void *stream,
                                sv_handle *out)
{
    if (!out || !device_ptr) return fail(GBVQC_ERR_ARG, "NULL argument");
    *out = nullptr;
    if (((uintptr_t)device_ptr) & 15) return fail(GBVQC_ERR_ARG, "device pointer not 16-byte aligned");
    ST_TRY(check_state_args(n_qubits, dtype, is_density));
    gbvqc_sv *s = new gbvqc_sv();
    s->n_log = n_qubits;
    s->n_phys = is_density ? 2 * n_qubits : n_qubits;
    s->dtype = dtype;
    s->density = is_density ? 1 : 0;
    s->stream = (cudaStream_t)stream;
    s->data = device_ptr;
    s->owned = false;
    gbvqc_status st = sv_init_common(s);
    if (st != GBVQC_OK) {
        sv_release(s);
        return st;
    }
    *out = s;
    return GBVQC_OK;
}

extern "C" gbvqc_status sv_free(sv_handle sv)
{
    sv_release(sv);
    return GBVQC_OK;
}

extern "C" gbvqc_status sv_reset(sv_handle sv)
{
    if (!sv) return fail(GBVQC_ERR_ARG, "NULL state");
    CUDA_TRY(launch_zero_state(sv->dtype, sv->data, sv->n_phys, sv->stream));
    return GBVQC_OK;
}

extern "C" gbvqc_status sv_set(sv_handle sv, const void *src, size_t n_amps, int src_is_host)
{
    if (!sv || !src) return fail(GBVQC_ERR_ARG, "NULL argument");
    if (n_amps != sv->amps()) return fail(GBVQC_ERR_ARG, "expected %zu amplitudes, got %zu", sv->amps(), n_amps);
    CUDA_TRY(cudaMemcpyAsync(sv->data, src, sv->bytes(),
                             src_is_host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, sv->stream));
    if (src_is_host) CUDA_TRY(cudaStreamSynchronize(sv->stream));
    return GBVQC_OK;
}

extern "C" gbvqc_status sv_get(sv_handle sv, void *dst, size_t n_amps, int dst_is_host)
{
    if (!sv || !dst) return fail(GBVQC_ERR_ARG, "NULL argument");
    if (n_amps != sv->amps()) return fail(GBVQC_ERR_ARG, "expected %zu amplitudes, got %zu", sv->amps(), n_amps);
    CUDA_TRY(cudaMemcpyAsync(dst, sv->data, sv->bytes(),
                             dst_is_host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, sv->stream));
    CUDA_TRY(cudaStreamSynchronize(sv->stream));
    return GBVQC_OK;
}

extern "C" gbvqc_status sv_info(sv_handle sv, int *n_qubits, int *dtype, int *is_density, void **device_ptr)
{
    if (!sv) return fail(GBVQC_ERR_ARG, "NULL state");
    if (n_qubits) *n_qubits = sv->n_log;
    if (dtype) *dtype = sv->dtype;
    if (is_density) *is_density = sv->density;
    if (device_ptr) *device_ptr = sv->data;
    return GBVQC_OK;
}

// --------------------------------------------------------------------- observables

extern "C" gbvqc_status obs_create(const gbvqc_pauli *terms, int n_terms, int n_qubits, obs_handle *out)
{
    if (!out || (!terms && n_terms > 0) || n_terms < 0) return fail(GBVQC_ERR_ARG, "bad arguments");
    *out = nullptr;
    if (n_qubits < 1 || n_qubits > 34) return fail(GBVQC_ERR_ARG, "qubit count %d", n_qubits);
    const uint64_t valid = n_qubits >= 64 ? ~0ull : ((uint64_t(1) << n_qubits) - 1);
    std::map<uint64_t, std::vector<ObsTerm>> by_x;
    for (int i = 0; i < n_terms; i++) {
        if ((terms[i].x_mask | terms[i].z_mask) & ~valid)
            return fail(GBVQC_ERR_ARG, "term %d touches a qubit >= %d", i, n_qubits);
        ObsTerm t{};
        t.coeff = terms[i].coeff;
        t.coeff_f = (float)terms[i].coeff;
        t.z = terms[i].z_mask;
        t.ph = __builtin_popcountll(terms[i].x_mask & terms[i].z_mask) & 3;  // Y = i X Z
        by_x[terms[i].x_mask].push_back(t);
    }
    gbvqc_obs *h = new gbvqc_obs();
    h->n_qubits = n_qubits;
    for (auto &kv : by_x) {
        ObsGroup g{};
        g.x = kv.first;
        g.t_begin = (int)h->terms.size();
        for (auto &t : kv.second) h->terms.push_back(t);
        g.t_end = (int)h->terms.size();
        h->groups.push_back(g);
    }
    *out = h;  // device copies are made on first use (ensure_obs)
    return GBVQC_OK;
}

static gbvqc_status ensure_obs(gbvqc_obs *h)
{
    if (h->d_groups) return GBVQC_OK;
    CUDA_TRY(pauli_prepare());
    ST_TRY(upload(&h->d_terms, h->terms));
    ST_TRY(upload(&h->d_groups, h->groups));
    return GBVQC_OK;
}

static uint64_t permute_mask(uint64_t m, const std::vector<int8_t> &perm)
{
    uint64_t r = 0;
    for (size_t q = 0; q < perm.size(); q++)
        if ((m >> q) & 1) r |= uint64_t(1) << perm[q];
    return r;
}

// The observable in a permuted qubit layout (device copies made once per layout; call
// outside stream capture).
static gbvqc_status obs_dev_perm(gbvqc_obs *h, const std::vector<int8_t> &perm, ObsDev *out)
{
    if (perm.empty()) {
        *out = h->dev();
        return GBVQC_OK;
    }
    auto it = h->perm_dev.find(perm);
    if (it == h->perm_dev.end()) {
        std::vector<ObsGroup> g = h->groups;
        std::vector<ObsTerm> t = h->terms;
        for (ObsGroup &x : g) x.x = permute_mask(x.x, perm);
        for (ObsTerm &x : t) x.z = permute_mask(x.z, perm);
        std::pair<ObsGroup *, ObsTerm *> d{nullptr, nullptr};
        ST_TRY(upload(&d.first, g));
        ST_TRY(upload(&d.second, t));
        it = h->perm_dev.emplace(perm, d).first;
    }
    *out = ObsDev{it->second.first, it->second.second, (int)h->groups.size(), (int)h->terms.size()};
    return GBVQC_OK;
}

extern "C" gbvqc_status obs_free(obs_handle h)
{
    if (!h) return GBVQC_OK;
    if (h->d_groups) cudaFree(h->d_groups);
    if (h->d_terms) cudaFree(h->d_terms);
    for (auto &kv : h->perm_dev) {
        cudaFree(kv.second.first);
        cudaFree(kv.second.second);
    }
    delete h;
    return GBVQC_OK;
}

static DensMap standard_map(int n)
{
    DensMap m{};
    for (int q = 0; q < n; q++) {
        m.ket[q] = (int8_t)q;
        m.bra[q] = (int8_t)(q + n);
    }
    return m;
}

static DensMap interleaved_map(int n)
{
    DensMap m{};
    for (int q = 0; q < n; q++) {
        m.ket[q] = (int8_t)(2 * q);
        m.bra[q] = (int8_t)(2 * q + 1);
    }
    return m;
}

extern "C" gbvqc_status measure(sv_handle sv, int qubit, double u, int *outcome, double *prob)
{
    if (!sv || !outcome || !prob) return fail(GBVQC_ERR_ARG, "NULL argument");
    if (qubit < 0 || qubit >= sv->n_log) return fail(GBVQC_ERR_ARG, "qubit %d of %d", qubit, sv->n_log);
    if (!(u >= 0.0 && u < 1.0)) return fail(GBVQC_ERR_ARG, "u = %g outside [0, 1)", u);
    // scratch: 2 partials per block (508 blocks) then the two weights
    const int max_blocks = 508;
    double *d_w = sv->d_scratch + 2 * max_blocks;
    CUDA_TRY(launch_measure_sums(sv->dtype, sv->data, sv->n_log, sv->density, qubit, sv->d_scratch, max_blocks,
                                 d_w, sv->stream));
    double w[2];
    CUDA_TRY(cudaMemcpyAsync(w, d_w, sizeof(w), cudaMemcpyDeviceToHost, sv->stream));
    CUDA_TRY(cudaStreamSynchronize(sv->stream));
    const double total = w[0] + w[1];
    if (!(total > 0.0)) return fail(GBVQC_ERR_ARG, "state has zero norm");
    const int k = u < w[0] / total ? 0 : 1;
    *outcome = k;
    *prob = w[k] / total;
    const double scale = sv->density ? 1.0 / w[k] : 1.0 / std::sqrt(w[k]);
    CUDA_TRY(launch_collapse(sv->dtype, sv->data, sv->n_log, sv->density, qubit, k, scale, sv->stream));
    return GBVQC_OK;
}

extern "C" gbvqc_status sample(sv_handle sv, const double *u, int n_shots, int64_t *out)
{
    if (!sv || (n_shots > 0 && (!u || !out)) || n_shots < 0) return fail(GBVQC_ERR_ARG, "bad arguments");
    for (int i = 0; i < n_shots; i++)
        if (!(u[i] >= 0.0 && u[i] < 1.0)) return fail(GBVQC_ERR_ARG, "u[%d] = %g outside [0, 1)", i, u[i]);
    if (n_shots == 0) return GBVQC_OK;
    const int n = sv->n_log;  // the weights live on the 2^n diagonal (density) or amplitudes
    const int cbits = std::min(n, std::max(5, n - 16));
    const size_t m = size_t(1) << (n - cbits);
    double *d_buf = nullptr;
    ST_TRY(dev_alloc(&d_buf, 2 * m + (size_t)n_shots));
    int64_t *d_out = nullptr;
    gbvqc_status st = dev_alloc(&d_out, (size_t)n_shots);
    cudaError_t e = cudaSuccess;
    if (st == GBVQC_OK) {
        e = cudaMemcpyAsync(d_buf + 2 * m, u, sizeof(double) * n_shots, cudaMemcpyHostToDevice, sv->stream);
        if (e == cudaSuccess)
            e = launch_sample(sv->dtype, sv->data, n, sv->density, cbits, d_buf, d_buf + m, d_buf + 2 * m, n_shots,
                              d_out, sv->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(out, d_out, sizeof(int64_t) * n_shots, cudaMemcpyDeviceToHost, sv->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(sv->stream);
    }
    cudaFree(d_buf);
    cudaFree(d_out);
    if (st != GBVQC_OK) return st;
    CUDA_TRY(e);
    return GBVQC_OK;
}

extern "C" gbvqc_status expect(sv_handle sv, obs_handle h, double *out_energy)
{
    if (!sv || !h || !out_energy) return fail(GBVQC_ERR_ARG, "NULL argument");
    if (h->n_qubits != sv->n_log) return fail(GBVQC_ERR_ARG, "observable has %d qubits, state %d", h->n_qubits, sv->n_log);
    ST_TRY(ensure_obs(h));
    RedScratch red{sv->d_scratch, sv->d_counter};
    double *d_out = sv->d_scratch + kMaxRedBlocks;
    if (sv->density)
        CUDA_TRY(launch_density_expect(sv->dtype, sv->data, sv->n_log, standard_map(sv->n_log), h->dev(), red,
                                       d_out, sv->stream));
    else
        CUDA_TRY(launch_pauli_expect(sv->dtype, sv->data, nullptr, sv->n_phys, h->dev(), red, d_out, sv->stream));
    CUDA_TRY(cudaMemcpyAsync(out_energy, d_out, sizeof(double), cudaMemcpyDeviceToHost, sv->stream));
    CUDA_TRY(cudaStreamSynchronize(sv->stream));
    return GBVQC_OK;
}

extern "C" gbvqc_status apply_channel(sv_handle sv, int kind, int qubit, double strength, const double *kraus,
                                      int n_kraus)
{
    if (!sv) return fail(GBVQC_ERR_ARG, "NULL state");
    if (!sv->density) return fail(GBVQC_ERR_NOT_DENSITY, "apply_channel needs a density state");
    if (!is_channel(kind)) return fail(GBVQC_ERR_ARG, "kind %d is not a channel", kind);
    if (is_channel2(kind)) return fail(GBVQC_ERR_ARG, "two-qubit channels run inside circuits");
    if (qubit < 0 || qubit >= sv->n_log) return fail(GBVQC_ERR_ARG, "qubit %d out of range", qubit);
    if (kind == GBVQC_KRAUS && (!kraus || n_kraus < 1 || n_kraus > 4))
        return fail(GBVQC_ERR_ARG, "KRAUS needs 1..4 operators");
    if (kind != GBVQC_KRAUS && !(strength >= 0.0 && strength <= 1.0))
        return fail(GBVQC_ERR_ARG, "channel strength %g outside [0, 1]", strength);
    Mat S = superop(channel_kraus(kind, strength, kraus, n_kraus));
    MatRec r;
    double m[32];
    mat_to(S, m);
    for (int i = 0; i < 32; i++) {
        r.d[i] = m[i];
        r.f[i] = (float)m[i];
    }
    CUDA_TRY(cudaMemcpyAsync(sv->d_rec, &r, sizeof r, cudaMemcpyHostToDevice, sv->stream));
    CUDA_TRY(launch_gate(sv->dtype, sv->data, sv->n_phys, classify(S), qubit, qubit + sv->n_log, sv->d_rec,
                         sv->stream));
    CUDA_TRY(cudaStreamSynchronize(sv->stream));  // the host record must outlive the copy
    return GBVQC_OK;
}

// ------------------------------------------------------------------------ circuits

static int add_rec(gbvqc_circuit *c, const Mat &M)
{
    MatRec r{};
    double m[32];
    mat_to(M, m);
    for (int i = 0; i < 32; i++) {
        r.d[i] = m[i];
        r.f[i] = (float)m[i];
    }
    c->recs.push_back(r);
    return (int)c->recs.size() - 1;
}

// A 16 x 16 matrix as 16 consecutive records (record base + r holds row r); returns base.
static int add_rec16(gbvqc_circuit *c, const Mat &M)
{
    const int base = (int)c->recs.size();
    for (int r = 0; r < 16; r++) {
        MatRec rec{};
        for (int col = 0; col < 16; col++) {
            rec.d[2 * col] = M[r * 16 + col].real();
            rec.d[2 * col + 1] = M[r * 16 + col].imag();
            rec.f[2 * col] = (float)rec.d[2 * col];
            rec.f[2 * col + 1] = (float)rec.d[2 * col + 1];
        }
        c->recs.push_back(rec);
    }
    return base;
}

// Forward, inverse and adjoint superoperators of a two-qubit channel (records of 16 rows).
struct Chan2Recs {
    int f, i, a;
};
static Chan2Recs channel2_records(gbvqc_circuit *c, const gbvqc_op &op)
{
    const Mat S = superop2(channel_kraus2(op.kind, op.params[0], op.kraus, op.n_kraus));
    Mat Si;
    mat_inverse(S, 16, Si);  // invertibility checked by circuit_create
    return Chan2Recs{add_rec16(c, S), add_rec16(c, Si), add_rec16(c, mat_dagger(S, 16))};
}

static int add_dyn(gbvqc_circuit *c, int param, int rot, int variant, int domain)
{
    DynRec d{};
    d.rec = (int)c->recs.size();
    d.param = param;
    d.rot = rot;
    d.variant = variant;
    d.domain = domain;
    MatRec r{};  // zero: materialisation writes only the entries a matrix uses
    const double zero[5] = {0, 0, 0, 0, 0};
    materialize(d, zero, &r);  // placeholder, refreshed from theta before every use
    c->recs.push_back(r);
    c->dyn.push_back(d);
    return d.rec;
}

static bool is_var_fsim(const gbvqc_op &op) { return op.kind == GBVQC_FSIM && op.param_index >= 0; }

// theta-dependent FSIM record (variant FWD / INV / DER / GEN; comp = FSIM parameter;
// domain BRA: the complex conjugate, for the bra qubits of a density matrix)
static int add_dyn_fsim(gbvqc_circuit *c, const gbvqc_op &op, int variant, int comp, int domain = DOM_KET)
{
    DynRec d{};
    d.rec = (int)c->recs.size();
    d.param = op.param_index;
    d.rot = ROT_FSIM;
    d.variant = variant;
    d.domain = domain;
    d.comp = comp;
    d.mask = op.param_mask;
    for (int k = 0; k < 5; k++) d.fixed[k] = op.params[k];
    MatRec r{};
    const double zero[5] = {0, 0, 0, 0, 0};
    materialize(d, zero, &r);
    c->recs.push_back(r);
    c->dyn.push_back(d);
    return d.rec;
}

// Records of one unitary op in a domain: forward, inverse, derivative (or -1), and shape;
// a variational FSIM lists per variational parameter its derivative record (dU/dp), its
// generator record ((dU/dp) U^dag) and its theta index.
struct OpComp {
    int der, gen, param;
};
struct OpRecs {
    int f, i, d, shape, dshape;
    Mat Mf, Mi;
    std::vector<OpComp> comps;
};

static OpRecs op_records(gbvqc_circuit *c, const gbvqc_op &op, int domain)
{
    OpRecs o{};
    o.d = -1;
    if (is_var_fsim(op)) {  // ket or bra side (a density matrix applies U and conj(U))
        o.f = add_dyn_fsim(c, op, VAR_FWD, 0, domain);
        o.i = add_dyn_fsim(c, op, VAR_INV, 0, domain);
        o.shape = SH_BLOCK2;  // every FSIM (and its conjugate) has the block structure
        o.dshape = SH_DENSE2;
        for (int k = 0, j = 0; k < 5; k++)
            if ((op.param_mask >> k) & 1)
                o.comps.push_back(OpComp{add_dyn_fsim(c, op, VAR_DER, k, domain),
                                         add_dyn_fsim(c, op, VAR_GEN, k, domain), op.param_index + j++});
        return o;
    }
    if (is_rotation(op.kind) && op.param_index >= 0) {
        int rot = op.kind - GBVQC_RX;
        o.f = add_dyn(c, op.param_index, rot, VAR_FWD, domain);
        o.i = add_dyn(c, op.param_index, rot, VAR_INV, domain);
        o.d = add_dyn(c, op.param_index, rot, VAR_DER, domain);
        if (domain == DOM_SUPER) o.shape = rot == ROT_Z ? SH_DIAG2 : SH_DENSE2;
        else o.shape = rot == ROT_Z ? SH_DIAG1 : rot == ROT_Y ? SH_REAL1 : SH_IMAG1;
        o.dshape = o.shape;
        return o;
    }
    Mat U = gate_matrix(op);
    int d = (int)std::lround(std::sqrt((double)U.size()));
    if (domain == DOM_BRA) U = mat_conj(U);
    if (domain == DOM_SUPER) {
        Mat S(16, 0);
        for (int a = 0; a < 2; a++)
            for (int b = 0; b < 2; b++)
                for (int cc = 0; cc < 2; cc++)
                    for (int dd = 0; dd < 2; dd++)
                        S[(a + 2 * b) * 4 + (cc + 2 * dd)] = U[a * 2 + cc] * std::conj(U[b * 2 + dd]);
        U = S;
        d = 4;
    }
    o.Mf = U;
    o.Mi = mat_dagger(U, d);
    o.f = add_rec(c, o.Mf);
    o.i = add_rec(c, o.Mi);
    o.shape = join_shape(classify(o.Mf), classify(o.Mi));
    return o;
}

static void free_plan(DevPlan *p)
{
    if (!p) return;
    cudaFree(p->d_fwd); cudaFree(p->d_rev); cudaFree(p->d_fsubs); cudaFree(p->d_rsubs);
    cudaFree(p->d_fgates); cudaFree(p->d_rgates); cudaFree(p->d_fents); cudaFree(p->d_rents);
    cudaFree(p->d_funits); cudaFree(p->d_runits); cudaFree(p->d_csr_ptr); cudaFree(p->d_csr_slots);
    cudaFree(p->d_fimg); cudaFree(p->d_rimg);
}

static void free_graphs(gbvqc_circuit *c)
{
    for (auto &kv : c->graphs) cudaGraphExecDestroy(kv.second);
    c->graphs.clear();
}

static void free_workspace(Workspace &w)
{
    cudaFree(w.phi); cudaFree(w.psi); cudaFree(w.d_theta); cudaFree(w.d_energy); cudaFree(w.d_grad);
    cudaFree(w.d_slot_grad); cudaFree(w.d_slot_partials); cudaFree(w.d_red); cudaFree(w.d_counter);
    w = Workspace();
}

extern "C" gbvqc_status circuit_free(circuit_handle c)
{
    if (!c) return GBVQC_OK;
    free_graphs(c);
    for (auto &kv : c->plans) free_plan(kv.second.get());
    free_workspace(c->ws);
    cudaFree(c->d_recs); cudaFree(c->d_dyn); cudaFree(c->d_plain_ptr); cudaFree(c->d_plain_slots);
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    delete c;
    return GBVQC_OK;
}

static gbvqc_status csr_upload(const std::vector<int> &slot_param, int n_params, int **d_ptr, int **d_slots)
{
    std::vector<int> ptr(n_params + 1, 0), slots;
    for (int p : slot_param)
        if (p >= 0) ptr[p + 1]++;
    for (int p = 0; p < n_params; p++) ptr[p + 1] += ptr[p];
    slots.assign(ptr[n_params], 0);
    std::vector<int> fill(ptr.begin(), ptr.end() - 1);
    for (size_t s = 0; s < slot_param.size(); s++)
        if (slot_param[s] >= 0) slots[fill[slot_param[s]]++] = (int)s;
    ST_TRY(upload(d_ptr, ptr));
    ST_TRY(upload(d_slots, slots));
    return GBVQC_OK;
}

// A general one-qubit unitary U = e^{i alpha} V with V real (SH_REAL1) or with a real
// diagonal and an imaginary off-diagonal (SH_IMAG1): sqrt(Y) and sqrt(X) are of this
// kind up to the phase e^{i pi/4}, and V costs 6 instead of 14 flops per amplitude.
// Components that the pattern makes zero are set to exactly zero (they are below
// 1e-13 of the largest entry).
static bool phase_normalize(const Mat &U, Mat &V, double &alpha)
{
    double mx = 0.0;
    int kmax = 0;
    for (int k = 0; k < 4; k++)
        if (std::abs(U[k]) > mx) mx = std::abs(U[k]), kmax = k;
    if (mx == 0.0) return false;
    const double tol = 1e-13 * mx;
    for (int pattern = 0; pattern < 2; pattern++) {
        double a;
        if (pattern == 0) a = std::arg(U[kmax]);  // real: any largest entry sets the phase
        else {                                    // imaginary off-diagonal: the diagonal does
            const int kd = std::abs(U[0]) >= std::abs(U[3]) ? 0 : 3;
            if (std::abs(U[kd]) <= tol) continue;
            a = std::arg(U[kd]);
        }
        const cd ph = std::polar(1.0, -a);
        Mat W(4);
        bool ok = true;
        for (int k = 0; k < 4; k++) {
            W[k] = U[k] * ph;
            const bool diag = k == 0 || k == 3;
            if (pattern == 0 || diag) {
                ok = ok && std::abs(W[k].imag()) <= tol;
                W[k] = cd(W[k].real(), 0.0);
            } else {
                ok = ok && std::abs(W[k].real()) <= tol;
                W[k] = cd(0.0, W[k].imag());
            }
        }
        if (ok) {
            V = W;
            alpha = a;
            return true;
        }
    }
    return false;
}

// Fixed one-qubit gate of shape SH_DENSE1 -> phase-normalised records (alpha returned).
static bool normalize_fixed(gbvqc_circuit *c, const gbvqc_op &op, OpRecs &r, double &alpha)
{
    alpha = 0.0;
    if (r.shape != SH_DENSE1 || (is_rotation(op.kind) && op.param_index >= 0) || r.Mf.size() != 4) return false;
    Mat V;
    if (!phase_normalize(r.Mf, V, alpha)) return false;
    r.Mf = V;
    r.Mi = mat_dagger(V, 2);
    r.f = add_rec(c, r.Mf);
    r.i = add_rec(c, r.Mi);
    r.shape = join_shape(classify(r.Mf), classify(r.Mi));
    return true;
}

static Mat mat_scaled(const Mat &M, cd z)
{
    Mat D(M.size());
    for (size_t i = 0; i < M.size(); i++) D[i] = M[i] * z;
    return D;
}

// Physical gate list of the fused engine for a density layout `map` (or pure, map unused).
// Fixed one-qubit gates are phase-normalised (normalize_fixed).  On a density matrix the
// phases cancel between the ket (U) and bra (conj U) sides; on a pure state their sum is
// multiplied into one fixed gate whose shape is kept by a complex scale, or, if there is
// none, undone on the first normalised gate, so the fused sweeps give the exact state.
static void fused_gates_of(gbvqc_circuit *c, const DensMap &map, std::vector<PGate> &out)
{
    out.clear();
    double phase = 0.0;              // pure: sum of the phases taken out
    int fold = -1, first_norm = -1;  // pure: gate that takes the phase back
    Mat fold_f, fold_i, norm_f;
    for (const gbvqc_op &op : c->ops) {
        if (!c->density) {
            OpRecs r = op_records(c, op, DOM_KET);
            double alpha = 0.0;
            if (normalize_fixed(c, op, r, alpha)) {
                phase += alpha;
                if (first_norm < 0) first_norm = (int)out.size(), norm_f = r.Mf;
            }
            // (CZ is applied as a sign flip that ignores its matrix: never a fold target)
            const bool fixed = !(is_rotation(op.kind) && op.param_index >= 0) && !r.Mf.empty() &&
                               op.kind != GBVQC_CZ;
            const bool scalable = r.shape == SH_DENSE1 || r.shape == SH_DENSE2 || r.shape == SH_BLOCK2 ||
                                  r.shape == SH_PAR2 ||
                                  r.shape == SH_DIAG1 || r.shape == SH_DIAG2 || r.shape == SH_PERM2 ||
                                  r.shape == SH_ANTI1;
            if (fold < 0 && fixed && scalable) fold = (int)out.size(), fold_f = r.Mf, fold_i = r.Mi;
            PGate g{};
            g.k = kind_qubits(op.kind);
            g.q[0] = op.qubits[0];
            g.q[1] = g.k == 2 ? op.qubits[1] : 0;
            g.diag = shape_is_diag(r.shape);
            g.ftype = ftype_of(r.shape);
            g.rec_f = r.f;
            g.rec_i = r.i;
            g.rec_a = r.i;
            g.perm_f = r.Mf.size() == 16 ? perm_bits(r.Mf) : 0;
            g.perm_r = r.Mi.size() == 16 ? perm_bits(r.Mi) : 0;
            g.gen = GEN_NONE;
            g.param = -1;
            g.cz = op.kind == GBVQC_CZ;
            if (is_rotation(op.kind) && op.param_index >= 0) {
                g.gen = op.kind == GBVQC_RX ? GEN_X : op.kind == GBVQC_RY ? GEN_Y : GEN_Z;
                g.gq = op.qubits[0];
                g.coef = 1.0f;
                g.param = op.param_index;
            }
            out.push_back(g);
            // variational FSIM: one gradient probe per parameter, right after the gate
            // (the reverse sweep reads 2 Re <Psi| (dU/dp) U^dag |Phi> before uncomputing U)
            for (const OpComp &cp : r.comps) {
                PGate pr = g;
                pr.ftype = FT_PROBE2;
                pr.diag = false;
                pr.rec_f = pr.rec_i = pr.rec_a = cp.gen;
                pr.perm_f = pr.perm_r = 0;
                pr.gen = GEN_M2;
                pr.gq = op.qubits[0];
                pr.coef = 2.0f;
                pr.param = cp.param;
                pr.cz = false;
                out.push_back(pr);
            }
            continue;
        }
        if (is_channel2(op.kind)) {  // a four-qubit superoperator: its own pass (barrier)
            const Chan2Recs r = channel2_records(c, op);
            PGate g{};
            g.k = 4;
            g.q[0] = map.ket[op.qubits[0]];
            g.q[1] = map.ket[op.qubits[1]];
            g.q[2] = map.bra[op.qubits[0]];
            g.q[3] = map.bra[op.qubits[1]];
            g.ftype = FT_DENSE4;
            g.rec_f = r.f;
            g.rec_i = r.i;
            g.rec_a = r.a;
            g.gen = GEN_NONE;
            g.param = -1;
            out.push_back(g);
            continue;
        }
        if (is_channel(op.kind)) {
            Mat S = superop(channel_kraus(op.kind, op.params[0], op.data, op.n_kraus)), Si;
            mat_inverse(S, 4, Si);
            Mat Sa = mat_dagger(S, 4);
            PGate g{};
            g.k = 2;
            g.q[0] = map.ket[op.qubits[0]];
            g.q[1] = map.bra[op.qubits[0]];
            int sh = join_shape(join_shape(classify(S), classify(Si)), classify(Sa));
            if (sh == SH_PERM2 || sh == SH_CTRL2 || sh == SH_CX) sh = SH_DENSE2;
            if (sh == SH_CZ) sh = SH_DIAG2;
            g.diag = sh == SH_DIAG2;
            g.ftype = ftype_of(sh);
            g.rec_f = add_rec(c, S);
            g.rec_i = add_rec(c, Si);
            g.rec_a = add_rec(c, Sa);
            g.gen = GEN_NONE;
            g.param = -1;
            out.push_back(g);
            continue;
        }
        // unitary on a density matrix: U on the ket qubits, conj(U) on the bra qubits
        for (int side = 0; side < 2; side++) {
            OpRecs r = op_records(c, op, side == 0 ? DOM_KET : DOM_BRA);
            double alpha;
            normalize_fixed(c, op, r, alpha);  // conj side: conj(V) with phase -alpha
            PGate g{};
            g.k = kind_qubits(op.kind);
            const int8_t *pos = side == 0 ? map.ket : map.bra;
            g.q[0] = pos[op.qubits[0]];
            g.q[1] = g.k == 2 ? pos[op.qubits[1]] : 0;
            g.diag = shape_is_diag(r.shape);
            g.ftype = ftype_of(r.shape);
            g.rec_f = r.f;
            g.rec_i = r.i;
            g.rec_a = r.i;
            g.perm_f = r.Mf.size() == 16 ? perm_bits(r.Mf) : 0;
            g.perm_r = r.Mi.size() == 16 ? perm_bits(r.Mi) : 0;
            g.gen = GEN_NONE;
            g.param = -1;
            g.cz = op.kind == GBVQC_CZ;  // real: conj(CZ) = CZ on the bra side
            if (is_rotation(op.kind) && op.param_index >= 0) {
                g.gen = op.kind == GBVQC_RX ? GEN_X : op.kind == GBVQC_RY ? GEN_Y : GEN_Z;
                g.gq = g.q[0];
                // ket: Re<<Psi|(-i/2)P|Phi>> = Im/2; bra: Re<<Psi|(i/2)P*|Phi>>, P* = -Y for Y
                g.coef = side == 0 ? 0.5f : (op.kind == GBVQC_RY ? 0.5f : -0.5f);
                g.param = op.param_index;
            }
            out.push_back(g);
            // variational FSIM: Re <<Psi| (dU/dp) U^-1 |Phi>> on this side (K conjugated on
            // the bra side) per parameter, read after the side's gate
            for (const OpComp &cp : r.comps) {
                PGate pr = g;
                pr.ftype = FT_PROBE2;
                pr.diag = false;
                pr.rec_f = pr.rec_i = pr.rec_a = cp.gen;
                pr.perm_f = pr.perm_r = 0;
                pr.gen = GEN_M2;
                pr.gq = g.q[0];
                pr.coef = 1.0f;
                pr.param = cp.param;
                pr.cz = false;
                out.push_back(pr);
            }
        }
    }
    const double ph = std::remainder(phase, 2.0 * M_PI);
    if (c->density || ph == 0.0) return;
    const cd z = std::polar(1.0, ph);
    if (fold >= 0) {  // shape kept: same ftype and permutation bits
        out[fold].rec_f = add_rec(c, mat_scaled(fold_f, z));
        out[fold].rec_i = out[fold].rec_a = add_rec(c, mat_scaled(fold_i, std::conj(z)));
    } else if (first_norm >= 0) {  // back to a general 2x2 on the first normalised gate
        const Mat W = mat_scaled(norm_f, z);
        out[first_norm].rec_f = add_rec(c, W);
        out[first_norm].rec_i = out[first_norm].rec_a = add_rec(c, mat_dagger(W, 2));
        out[first_norm].ftype = FT_DENSE1;
    }
}

extern "C" gbvqc_status circuit_create(const gbvqc_op *ops, int n_ops, int n_qubits, int n_params,
                                       int is_density, circuit_handle *out)
{
    if (!out || (!ops && n_ops > 0) || n_ops < 0 || n_params < 0) return fail(GBVQC_ERR_ARG, "bad arguments");
    *out = nullptr;
    int n_phys = is_density ? 2 * n_qubits : n_qubits;
    if (n_qubits < 1 || n_phys > 34) return fail(GBVQC_ERR_ARG, "qubit count %d out of range", n_qubits);
    for (int j = 0; j < n_ops; j++) {
        const gbvqc_op &op = ops[j];
        if (op.kind < 0 || op.kind >= GBVQC_NUM_KINDS) return fail(GBVQC_ERR_ARG, "op %d: kind %d", j, op.kind);
        int k = kind_qubits(op.kind);
        for (int u = 0; u < k; u++)
            if (op.qubits[u] < 0 || op.qubits[u] >= n_qubits)
                return fail(GBVQC_ERR_ARG, "op %d: qubit %d out of range", j, op.qubits[u]);
        if (k == 2 && op.qubits[0] == op.qubits[1]) return fail(GBVQC_ERR_ARG, "op %d: repeated qubit", j);
        if (op.param_index >= 0 && op.kind == GBVQC_FSIM) {
            if (op.param_mask < 1 || op.param_mask > 31)
                return fail(GBVQC_ERR_ARG, "op %d: FSIM param_mask %d", j, op.param_mask);
            if (op.param_index + __builtin_popcount(op.param_mask) > n_params)
                return fail(GBVQC_ERR_ARG, "op %d: FSIM parameters beyond n_params", j);
        } else if (op.param_index >= 0 && (!is_rotation(op.kind) || op.param_index >= n_params)) {
            return fail(GBVQC_ERR_ARG, "op %d: bad param_index %d", j, op.param_index);
        }
        if (op.param_index < -1) return fail(GBVQC_ERR_ARG, "op %d: bad param_index %d", j, op.param_index);
        if (is_channel2(op.kind)) {
            if (!is_density) return fail(GBVQC_ERR_NOT_DENSITY, "op %d: channel in a pure-state circuit", j);
            if (op.kind == GBVQC_KRAUS2 && (!op.kraus || op.n_kraus < 1 || op.n_kraus > 16))
                return fail(GBVQC_ERR_ARG, "op %d: KRAUS2 needs 1..16 operators", j);
            if (op.kind == GBVQC_DEPOL2 && !(op.params[0] >= 0.0 && op.params[0] <= 1.0))
                return fail(GBVQC_ERR_ARG, "op %d: channel strength %g", j, op.params[0]);
            Mat Si;
            if (!mat_inverse(superop2(channel_kraus2(op.kind, op.params[0], op.kraus, op.n_kraus)), 16, Si))
                return fail(GBVQC_ERR_ARG, "op %d: channel superoperator is singular", j);
        } else if (is_channel(op.kind)) {
            if (!is_density) return fail(GBVQC_ERR_NOT_DENSITY, "op %d: channel in a pure-state circuit", j);
            if (op.kind == GBVQC_KRAUS && (op.n_kraus < 1 || op.n_kraus > 4))
                return fail(GBVQC_ERR_ARG, "op %d: n_kraus %d", j, op.n_kraus);
            if (op.kind != GBVQC_KRAUS && !(op.params[0] >= 0.0 && op.params[0] <= 1.0))
                return fail(GBVQC_ERR_ARG, "op %d: channel strength %g", j, op.params[0]);
            if (op.kind == GBVQC_KRAUS || op.params[0] > 0.0) {
                Mat S = superop(channel_kraus(op.kind, op.params[0], op.data, op.n_kraus)), Si;
                if (!mat_inverse(S, 4, Si))
                    return fail(GBVQC_ERR_ARG, "op %d: channel superoperator is singular", j);
            }
        }
    }
    gbvqc_circuit *c = new gbvqc_circuit();
    c->n_log = n_qubits;
    c->n_phys = n_phys;
    c->n_params = n_params;
    c->density = is_density ? 1 : 0;
    c->ops.assign(ops, ops + n_ops);
    c->kraus_store.reserve(n_ops);
    for (gbvqc_op &op : c->ops) {
        if (op.kind == GBVQC_KRAUS2) {
            c->kraus_store.emplace_back(op.kraus, op.kraus + 32 * op.n_kraus);
            op.kraus = c->kraus_store.back().data();
        } else {
            op.kraus = nullptr;
        }
    }
    for (const gbvqc_op &op : c->ops)
        c->n_param_ops += op.param_index < 0 ? 0 : is_var_fsim(op) ? __builtin_popcount(op.param_mask) : 1;
    // per-gate schedule in the standard layout
    for (const gbvqc_op &op : c->ops) {
        int k = kind_qubits(op.kind);
        if (!c->density) {
            OpRecs r = op_records(c, op, DOM_KET);
            PlainGate g{r.shape, op.qubits[0], k == 2 ? op.qubits[1] : 0, r.f, r.i, r.i, 1, op.qubits[0], 0,
                        r.d, op.param_index, 2.0, -1};
            if (!r.comps.empty()) {  // variational FSIM: dU/dp on both qubits per parameter
                g.der_k = 2;
                g.dq1 = op.qubits[1];
                g.rec_d = r.comps[0].der;
                g.param = r.comps[0].param;
                for (size_t e = 1; e < r.comps.size(); e++) {
                    g.ex_rec[g.n_extra] = r.comps[e].der;
                    g.ex_param[g.n_extra] = r.comps[e].param;
                    g.n_extra++;
                }
            }
            c->plain.push_back(g);
        } else if (is_channel2(op.kind)) {
            const Chan2Recs r = channel2_records(c, op);
            PlainGate g{SH_DENSE4, op.qubits[0], op.qubits[1], r.f, r.i, r.a, 0, 0, 0, -1, -1, 1.0, -1};
            g.q2 = op.qubits[0] + n_qubits;
            g.q3 = op.qubits[1] + n_qubits;
            c->plain.push_back(g);
        } else if (is_channel(op.kind)) {
            Mat S = superop(channel_kraus(op.kind, op.params[0], op.data, op.n_kraus)), Si;
            mat_inverse(S, 4, Si);
            Mat Sa = mat_dagger(S, 4);
            int sh = join_shape(join_shape(classify(S), classify(Si)), classify(Sa));
            PlainGate g{sh, op.qubits[0], op.qubits[0] + n_qubits, add_rec(c, S), add_rec(c, Si), add_rec(c, Sa),
                        2, op.qubits[0], op.qubits[0] + n_qubits, -1, -1, 1.0, -1};
            c->plain.push_back(g);
        } else if (k == 1) {
            OpRecs r = op_records(c, op, DOM_SUPER);
            PlainGate g{r.shape, op.qubits[0], op.qubits[0] + n_qubits, r.f, r.i, r.i, 2, op.qubits[0],
                        op.qubits[0] + n_qubits, r.d, op.param_index, 1.0, -1};
            c->plain.push_back(g);
        } else {
            for (int side = 0; side < 2; side++) {
                OpRecs r = op_records(c, op, side == 0 ? DOM_KET : DOM_BRA);
                int off = side == 0 ? 0 : n_qubits;
                PlainGate g{r.shape, op.qubits[0] + off, op.qubits[1] + off, r.f, r.i, r.i, 1, 0, 0, -1, -1, 1.0, -1};
                if (!r.comps.empty()) {  // variational FSIM: Re <<Psi| dU (side) |Phi>> per parameter
                    g.der_k = 2;
                    g.dq0 = op.qubits[0] + off;
                    g.dq1 = op.qubits[1] + off;
                    g.rec_d = r.comps[0].der;
                    g.param = r.comps[0].param;
                    for (size_t e = 1; e < r.comps.size(); e++) {
                        g.ex_rec[g.n_extra] = r.comps[e].der;
                        g.ex_param[g.n_extra] = r.comps[e].param;
                        g.n_extra++;
                    }
                }
                c->plain.push_back(g);
            }
        }
    }
    std::vector<int> slot_param;  // parameter of each per-gate gradient slot
    for (PlainGate &g : c->plain) {
        if (g.param >= 0 && g.rec_d >= 0) {
            g.slot = (int)slot_param.size();
            slot_param.push_back(g.param);
        }
        for (int e = 0; e < g.n_extra; e++) {
            g.ex_slot[e] = (int)slot_param.size();
            slot_param.push_back(g.ex_param[e]);
        }
    }
    c->plain_slots = (int)slot_param.size();
    c->map_std = standard_map(n_qubits);
    c->map_grad = interleaved_map(n_qubits);
    fused_gates_of(c, c->map_std, c->pg_std);
    if (c->density) fused_gates_of(c, c->map_grad, c->pg_grad);
    c->plain_slot_param = slot_param;
    *out = c;
    return GBVQC_OK;
}

// Device copies of the circuit's matrix records, dynamic-record list and per-gate CSR,
// and the capture stream: made on the first call that launches work.
static gbvqc_status ensure_device(gbvqc_circuit *c)
{
    if (c->dev_ready) return GBVQC_OK;
    ST_TRY(csr_upload(c->plain_slot_param, c->n_params, &c->d_plain_ptr, &c->d_plain_slots));
    ST_TRY(upload(&c->d_recs, c->recs));
    ST_TRY(upload(&c->d_dyn, c->dyn));
    CUDA_TRY(cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
    c->dev_ready = true;
    return GBVQC_OK;
}

static int default_tile(int) { return 12; }

static int ilog2(int x)
{
    int r = 0;
    while ((1 << (r + 1)) <= x) r++;
    return r;
}

// Largest tile: 2^(t - NR) threads per CTA within both fused kernels' launch bounds.
static int max_tile(int dtype)
{
    const int nf = fused_nr(dtype, false), nr = fused_nr(dtype, true);
    return std::min(nf + ilog2(fused_max_threads(nf, false)), nr + ilog2(fused_max_threads(nr, true)));
}
static int default_low(int dtype) { return dtype == GBVQC_C64 ? 4 : 3; }

// Fused plan for (dtype, layout); built on first use (host only).
// Gradient layout of a pure circuit: the `low` physical low qubits (always in every
// tile) are the logical qubits that give the fewest passes; the evaluation starts from
// |0...0>, which is the same in every layout, and the observable's masks are permuted
// to match, so the layout never leaves the gradient call.  Candidates: every pair (one
// qubit if low = 1), the best pair grown greedily, and every window of `low` consecutive
// qubits; ties keep the identity layout.
static std::vector<int8_t> choose_grad_layout(const std::vector<PGate> &pg, int n, const PlanOptions &opt)
{
    const int low = std::max(1, std::min(opt.low, std::min(opt.t, n)));
    auto mapped = [&](const std::vector<int> &lows, std::vector<int8_t> &perm) {
        perm.assign(n, -1);
        int next = 0;
        for (int q : lows) perm[q] = (int8_t)next++;
        for (int q = 0; q < n; q++)
            if (perm[q] < 0) perm[q] = (int8_t)next++;
        std::vector<PGate> G = pg;
        for (PGate &g : G) {
            g.q[0] = perm[g.q[0]];
            if (g.k == 2) g.q[1] = perm[g.q[1]];
            if (g.gen != GEN_NONE) g.gq = perm[g.gq];
        }
        return count_passes(G, n, opt);
    };
    std::vector<int> ident;
    for (int q = 0; q < low; q++) ident.push_back(q);
    std::vector<int8_t> perm;
    int best = mapped(ident, perm);
    if (best < 0 || pg.size() > 20000) return {};
    std::vector<int> best_set = ident;
    std::vector<int> cur;
    if (low >= 2) {
        for (int a = 0; a < n; a++)
            for (int b = a + 1; b < n; b++) {
                std::vector<int> s2 = {a, b};
                const int v = mapped(s2, perm);
                if (v >= 0 && v < best) best = v, best_set = s2;
            }
        cur = best_set.size() == 2 ? best_set : std::vector<int>{0, 1};
        while ((int)cur.size() < low) {  // extend greedily
            int bq = -1, bv = 1 << 30;
            for (int q = 0; q < n; q++) {
                if (std::find(cur.begin(), cur.end(), q) != cur.end()) continue;
                std::vector<int> s3 = cur;
                s3.push_back(q);
                const int v = mapped(s3, perm);
                if (v >= 0 && v < bv) bv = v, bq = q;
            }
            if (bq < 0) break;
            cur.push_back(bq);
            if ((int)cur.size() == low && bv < best) best = bv, best_set = cur;
        }
    } else {
        for (int a = 1; a < n; a++) {
            std::vector<int> s1 = {a};
            const int v = mapped(s1, perm);
            if (v >= 0 && v < best) best = v, best_set = s1;
        }
    }
    for (int a = 1; a + low <= n; a++) {  // contiguous windows (chains, ladders, bricks)
        std::vector<int> win;
        for (int q = a; q < a + low; q++) win.push_back(q);
        const int v = mapped(win, perm);
        if (v >= 0 && v < best) best = v, best_set = win;
    }
    if ((int)best_set.size() != low || best_set == ident) return {};
    std::sort(best_set.begin(), best_set.end());
    mapped(best_set, perm);
    return perm;
}

// Shared memory per CTA that still leaves two reverse-pass CTAs on one SM (228 KB per SM,
// 1 KB reserved per CTA), less a margin for alignment and the phase-block constants.
constexpr int kTwoCtaSmem = 110 * 1024;

// batch: the plan a batch member runs with (launches shared by all members take the
// largest member's shared memory, so its passes keep the smaller slot budget that leaves
// two CTAs per SM; a single circuit takes larger passes, fewer tile loads and stores).
static gbvqc_status get_host_plan(gbvqc_circuit *c, int dtype, bool grad_layout, DevPlan **out, bool batch = false)
{
    int key = dtype * 2 + (grad_layout ? 1 : 0) + (batch ? 4 : 0);
    auto it = c->plans.find(key);
    if (it != c->plans.end()) {
        *out = it->second.get();
        return GBVQC_OK;
    }
    const std::vector<PGate> &pg0 = (grad_layout && c->density) ? c->pg_grad : c->pg_std;
    PlanOptions opt;
    opt.t = c->tile_qubits ? c->tile_qubits : default_tile(dtype);
    opt.low = c->low_qubits ? c->low_qubits : default_low(dtype);
    opt.nr_f = fused_nr(dtype, false);
    opt.nr_r = fused_nr(dtype, true);
    opt.t = std::min(opt.t, max_tile(dtype));
    opt.elem_bytes = dtype == GBVQC_C64 ? 4 : 8;
    opt.max_slots = batch ? 128 : 512;
    opt.gate_smem = batch ? 40 * 1024 : 64 * 1024;
    std::vector<int8_t> perm;
    std::vector<PGate> permuted;
    if (grad_layout && !c->density) perm = choose_grad_layout(pg0, c->n_phys, opt);
    if (!perm.empty()) {
        permuted = pg0;
        for (PGate &g : permuted) {
            g.q[0] = perm[g.q[0]];
            if (g.k == 2) g.q[1] = perm[g.q[1]];
            if (g.gen != GEN_NONE) g.gq = perm[g.gq];
        }
    }
    const std::vector<PGate> &pg = perm.empty() ? pg0 : permuted;
    std::unique_ptr<DevPlan> dp(new DevPlan());
    dp->elem = opt.elem_bytes;
    dp->perm = perm;
    std::string err;
    for (int attempt = 0;; attempt++) {
        dp->p = FusedPlan();
        dp->fwd_smem.clear();
        dp->rev_smem.clear();
        if (!build_fused_plan(pg, c->n_phys, opt, dp->p, err))
            return fail(GBVQC_ERR_UNSUPPORTED, "fused plan: %s", err.c_str());
        size_t worst = 0;
        for (const PassDesc &d : dp->p.fwd) dp->fwd_smem.push_back(pass_smem_bytes(dp->p, d, false, opt.elem_bytes));
        for (const PassDesc &d : dp->p.rev) {
            dp->rev_smem.push_back(pass_smem_bytes(dp->p, d, true, opt.elem_bytes));
            worst = std::max(worst, dp->rev_smem.back());
        }
        // larger passes only while every reverse pass still fits two CTAs per SM
        if (batch || worst <= (size_t)kTwoCtaSmem || opt.gate_smem <= 24 * 1024 || attempt >= 4) break;
        opt.gate_smem = opt.gate_smem * 3 / 4;
        opt.max_slots = std::max(128, opt.max_slots / 2);
    }
    for (size_t b : dp->fwd_smem)
        if (b > 200 * 1024) return fail(GBVQC_ERR_UNSUPPORTED, "fused pass needs %zu bytes of shared memory", b);
    for (size_t b : dp->rev_smem)
        if (b > 200 * 1024) return fail(GBVQC_ERR_UNSUPPORTED, "fused pass needs %zu bytes of shared memory", b);
    *out = dp.get();
    c->plans[key] = std::move(dp);
    return GBVQC_OK;
}

// Fused plan with its device copies.
static gbvqc_status get_plan(gbvqc_circuit *c, int dtype, bool grad_layout, DevPlan **out, bool batch = false)
{
    DevPlan *dp = nullptr;
    ST_TRY(get_host_plan(c, dtype, grad_layout, &dp, batch));
    if (!dp->uploaded) {
        CUDA_TRY(fused_prepare());
        ST_TRY(upload(&dp->d_fwd, dp->p.fwd));
        ST_TRY(upload(&dp->d_rev, dp->p.rev));
        ST_TRY(upload(&dp->d_fsubs, dp->p.fsubs));
        ST_TRY(upload(&dp->d_rsubs, dp->p.rsubs));
        ST_TRY(upload(&dp->d_fgates, dp->p.fgates));
        ST_TRY(upload(&dp->d_rgates, dp->p.rgates));
        ST_TRY(upload(&dp->d_fents, dp->p.fents));
        ST_TRY(upload(&dp->d_rents, dp->p.rents));
        ST_TRY(upload(&dp->d_funits, dp->p.funits));
        ST_TRY(upload(&dp->d_runits, dp->p.runits));
        const size_t eb = dtype == GBVQC_C64 ? 4 : 8;
        ST_TRY(dev_alloc((unsigned char **)&dp->d_fimg, std::max<size_t>(1, 8 * eb * dp->p.funits.size())));
        ST_TRY(dev_alloc((unsigned char **)&dp->d_rimg, std::max<size_t>(1, 8 * eb * dp->p.runits.size())));
        ST_TRY(csr_upload(dp->p.slot_param, c->n_params, &dp->d_csr_ptr, &dp->d_csr_slots));
        dp->uploaded = true;
    }
    *out = dp;
    return GBVQC_OK;
}

static bool fused_supported(const gbvqc_circuit *c, int dtype)
{
    return c->n_phys >= std::max(fused_nr(dtype, false), fused_nr(dtype, true)) + 1;
}

#define GBVQC_SAME(a, b) ((int)(a) == (int)(b))
static_assert(GBVQC_SAME(GBVQC_SHAPE_DENSE1, SH_DENSE1) && GBVQC_SAME(GBVQC_SHAPE_DIAG1, SH_DIAG1) &&
                  GBVQC_SAME(GBVQC_SHAPE_ANTI1, SH_ANTI1) && GBVQC_SAME(GBVQC_SHAPE_REAL1, SH_REAL1) &&
                  GBVQC_SAME(GBVQC_SHAPE_DENSE2, SH_DENSE2) && GBVQC_SAME(GBVQC_SHAPE_DIAG2, SH_DIAG2) &&
                  GBVQC_SAME(GBVQC_SHAPE_PERM2, SH_PERM2) && GBVQC_SAME(GBVQC_SHAPE_CTRL2, SH_CTRL2) &&
                  GBVQC_SAME(GBVQC_SHAPE_BLOCK2, SH_BLOCK2) && GBVQC_SAME(GBVQC_SHAPE_IMAG1, SH_IMAG1) &&
                  GBVQC_SAME(GBVQC_SHAPE_PAR2, SH_PAR2) && GBVQC_SAME(GBVQC_SHAPE_RPAR2, SH_RPAR2) &&
                  GBVQC_SAME(GBVQC_SHAPE_CX, SH_CX) && GBVQC_SAME(GBVQC_SHAPE_CZ, SH_CZ),
              "public shape codes follow the kernels' shapes");
#undef GBVQC_SAME

extern "C" gbvqc_status gate_shape(const double *matrix, int dim, int *shape)
{
    if (!matrix || !shape || (dim != 2 && dim != 4)) return fail(GBVQC_ERR_ARG, "gate_shape: matrix, dim 2 or 4, shape");
    Mat M(dim * dim);
    for (int i = 0; i < dim * dim; i++) M[i] = cd(matrix[2 * i], matrix[2 * i + 1]);
    *shape = classify(M);
    return GBVQC_OK;
}

extern "C" gbvqc_status circuit_set_tiling(circuit_handle c, int tile_qubits, int low_qubits)
{
    if (!c) return fail(GBVQC_ERR_ARG, "NULL circuit");
    if (tile_qubits != 0 && (tile_qubits < 6 || tile_qubits > 13)) return fail(GBVQC_ERR_ARG, "tile_qubits %d", tile_qubits);
    if (low_qubits != 0 && (low_qubits < 1 || low_qubits > 6)) return fail(GBVQC_ERR_ARG, "low_qubits %d", low_qubits);
    std::lock_guard<std::mutex> lk(c->mu);
    free_graphs(c);
    for (auto &kv : c->plans) free_plan(kv.second.get());
    c->plans.clear();
    cudaFree(c->ws.d_slot_partials);
    c->ws.d_slot_partials = nullptr;
    c->partials_cap = 0;
    c->tile_qubits = tile_qubits;
    c->low_qubits = low_qubits;
    return GBVQC_OK;
}

extern "C" gbvqc_status circuit_plan_info(circuit_handle c, int *n_passes, int *n_gates, int *tile_qubits)
{
    if (!c) return fail(GBVQC_ERR_ARG, "NULL circuit");
    std::lock_guard<std::mutex> lk(c->mu);
    DevPlan *p = nullptr;
    if (!fused_supported(c, GBVQC_C64)) return fail(GBVQC_ERR_UNSUPPORTED, "too few qubits for tiles");
    ST_TRY(get_host_plan(c, GBVQC_C64, c->density != 0, &p));
    if (n_passes) *n_passes = (int)p->p.fwd.size();
    if (n_gates) *n_gates = (int)p->p.fgates.size();  // forward gate records (phase blocks count once)
    if (tile_qubits) *tile_qubits = p->p.t;
    return GBVQC_OK;
}

extern "C" gbvqc_status circuit_plan_stats(circuit_handle c, int dtype, int for_grad, int64_t *stats, int n_stats)
{
    if (!c || !stats || n_stats < 0) return fail(GBVQC_ERR_ARG, "NULL argument");
    if (dtype != GBVQC_C64 && dtype != GBVQC_C128) return fail(GBVQC_ERR_ARG, "dtype %d", dtype);
    std::lock_guard<std::mutex> lk(c->mu);
    if (!fused_supported(c, dtype)) return fail(GBVQC_ERR_UNSUPPORTED, "too few qubits for tiles");
    DevPlan *p = nullptr;
    ST_TRY(get_host_plan(c, dtype, for_grad != 0, &p));
    int64_t blocks = 0;
    for (const FGate &g : p->p.fgates) blocks += g.type == FT_DIAGB;
    int64_t v[10] = {p->p.t, (int64_t)p->p.fwd.size(), (int64_t)p->p.fsubs.size(), (int64_t)p->p.fgates.size(),
                     blocks, (int64_t)p->p.rsubs.size(), p->p.n_slots,
                     (int64_t)*std::max_element(p->fwd_smem.begin(), p->fwd_smem.end()),
                     (int64_t)*std::max_element(p->rev_smem.begin(), p->rev_smem.end()),
                     (int64_t)((for_grad && c->density) ? c->pg_grad.size() : c->pg_std.size())};
    for (int i = 0; i < n_stats && i < 10; i++) stats[i] = v[i];
    return GBVQC_OK;
}

// ------------------------------------------------------------------- execution

static gbvqc_status ensure_theta(gbvqc_circuit *c)
{
    if (!c->ws.d_theta) ST_TRY(dev_alloc(&c->ws.d_theta, c->n_params + 1));
    return GBVQC_OK;
}

static gbvqc_status stage_theta(gbvqc_circuit *c, const double *theta, int n_theta, int loc, cudaStream_t s)
{
    if (n_theta != c->n_params) return fail(GBVQC_ERR_ARG, "expected %d parameters, got %d", c->n_params, n_theta);
    if (n_theta > 0 && !theta) return fail(GBVQC_ERR_ARG, "theta is NULL");
    ST_TRY(ensure_theta(c));
    if (n_theta > 0)
        CUDA_TRY(cudaMemcpyAsync(c->ws.d_theta, theta, sizeof(double) * n_theta,
                                 loc == GBVQC_PTR_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
    return GBVQC_OK;
}

static double state_bytes(const gbvqc_circuit *c, int dtype) { return double(size_t(1) << c->n_phys) * amp_size(dtype); }

// Four-qubit superoperator (16 rows from record rec) on physical qubits q[0..3].
static gbvqc_status gate4(gbvqc_circuit *c, int dtype, void *psi, const int *q, int rec, cudaStream_t s)
{
    const double amps = double(size_t(1) << c->n_phys), sb = state_bytes(c, dtype);
    return run_k("gate4q", shape_flops(SH_DENSE4) * amps, 2.0 * sb, s, [&] {
        return launch_gate4(dtype, psi, c->n_phys, q[0], q[1], q[2], q[3], c->d_recs + rec, s);
    });
}

static gbvqc_status plain_gate(gbvqc_circuit *c, int dtype, void *psi, const PlainGate &g, int rec, cudaStream_t s)
{
    const double amps = double(size_t(1) << c->n_phys), sb = state_bytes(c, dtype);
    if (g.shape == SH_DENSE4) {
        const int q[4] = {g.q0, g.q1, g.q2, g.q3};
        return gate4(c, dtype, psi, q, rec, s);
    }
    const bool one = shape_qubits(g.shape) == 1;
    // complex64 runs CNOT through the controlled-2x2 kernel (launch_gate)
    const int fsh = g.shape == SH_CX && dtype == GBVQC_C64 ? SH_CTRL2 : g.shape;
    return run_k(one ? "gate1q" : "gate2q", shape_flops(fsh) * amps, (g.shape == SH_CTRL2 || g.shape == SH_CX ? 1.0 : g.shape == SH_CZ ? 0.5 : 2.0) * sb, s,
                 [&] { return launch_gate(dtype, psi, c->n_phys, g.shape, g.q0, g.q1, c->d_recs + rec, s); });
}

static gbvqc_status run_plain_forward(gbvqc_circuit *c, int dtype, void *psi, cudaStream_t s)
{
    for (const PlainGate &g : c->plain) ST_TRY(plain_gate(c, dtype, psi, g, g.rec_f, s));
    return GBVQC_OK;
}

// Matrix images of the plan's forward (and reverse) unit lists from this step's records.
static gbvqc_status gather_images(gbvqc_circuit *c, DevPlan *p, int dtype, bool with_rev, cudaStream_t s)
{
    return run_k("gather_units", 0, 0, s, [&] {
        return launch_gather_units(dtype, p->d_funits, (int)p->p.funits.size(), p->d_fimg, p->d_runits,
                                   with_rev ? (int)p->p.runits.size() : 0, p->d_rimg, c->d_recs, s);
    });
}

static gbvqc_status run_fused_forward(gbvqc_circuit *c, DevPlan *p, int dtype, void *psi, cudaStream_t s)
{
    const double amps = double(size_t(1) << c->n_phys), sb = state_bytes(c, dtype);
    const FusedDev fd{p->d_fwd, p->d_fsubs, p->d_fgates, p->d_fents, p->d_funits, c->d_recs, p->d_fimg};
    for (size_t i = 0; i < p->p.fwd.size(); i++) {
        if (p->p.barrier[i] >= 0) {  // two-qubit channel between the tile passes
            const PGate &g = p->p.barrier_gates[p->p.barrier[i]];
            ST_TRY(gate4(c, dtype, psi, g.q, g.rec_f, s));
            continue;
        }
        ST_TRY(run_k("fused_forward", p->p.fwd_flops[i] * amps, 2 * sb, s, [&] {
            return launch_fused_forward(dtype, psi, fd, (int)i, p->p.fwd[i], p->fwd_smem[i], s);
        }));
    }
    return GBVQC_OK;
}

extern "C" gbvqc_status apply_circuit(sv_handle sv, circuit_handle c, const double *theta, int n_theta, int theta_loc,
                                      int mode)
{
    if (!sv || !c) return fail(GBVQC_ERR_ARG, "NULL argument");
    if (sv->n_log != c->n_log || sv->density != c->density)
        return fail(GBVQC_ERR_ARG, "state (%d qubits, density %d) does not match circuit (%d, %d)", sv->n_log,
                    sv->density, c->n_log, c->density);
    if (mode != GBVQC_MODE_PLAIN && mode != GBVQC_MODE_FUSED) return fail(GBVQC_ERR_ARG, "mode %d", mode);
    std::lock_guard<std::mutex> lk(c->mu);
    cudaStream_t s = sv->stream;
    ST_TRY(ensure_device(c));
    ST_TRY(stage_theta(c, theta, n_theta, theta_loc, s));
    CUDA_TRY(launch_materialize(c->d_dyn, (int)c->dyn.size(), c->ws.d_theta, c->d_recs, s));
    if (mode == GBVQC_MODE_FUSED && fused_supported(c, sv->dtype)) {
        DevPlan *p = nullptr;
        ST_TRY(get_plan(c, sv->dtype, false, &p));
        ST_TRY(gather_images(c, p, sv->dtype, false, s));
        return run_fused_forward(c, p, sv->dtype, sv->data, s);
    }
    return run_plain_forward(c, sv->dtype, sv->data, s);
}

// ------------------------------------------------------------------------ gradient

static gbvqc_status ensure_workspace(gbvqc_circuit *c, int dtype)
{
    Workspace &w = c->ws;
    if (w.dtype != dtype) {
        free_graphs(c);
        cudaFree(w.phi);
        cudaFree(w.psi);
        w.phi = w.psi = nullptr;
        size_t bytes = (size_t(1) << c->n_phys) * amp_size(dtype);
        ST_TRY(dev_alloc((unsigned char **)&w.phi, bytes));
        ST_TRY(dev_alloc((unsigned char **)&w.psi, bytes));
        w.dtype = dtype;
    }
    ST_TRY(ensure_theta(c));
    if (!w.d_energy) ST_TRY(dev_alloc(&w.d_energy, 1));
    if (!w.d_grad) ST_TRY(dev_alloc(&w.d_grad, c->n_params + 1));
    if (!w.d_red) ST_TRY(dev_alloc(&w.d_red, kMaxRedBlocks));
    if (!w.d_counter) {
        ST_TRY(dev_alloc(&w.d_counter, 1));
        CUDA_TRY(cudaMemset(w.d_counter, 0, sizeof(unsigned)));
    }
    return GBVQC_OK;
}

// The whole gradient evaluation as a stream-ordered launch sequence (capturable).
static gbvqc_status enqueue_grad(gbvqc_circuit *c, obs_handle h, int dtype, int mode, DevPlan *p, cudaStream_t s)
{
    Workspace &w = c->ws;
    RedScratch red{w.d_red, w.d_counter};
    const bool fused = mode == GBVQC_MODE_FUSED && p;
    const double amps = double(size_t(1) << c->n_phys), sb = state_bytes(c, dtype);
    ST_TRY(run_k("materialize", 0, 0, s, [&] {
        return launch_materialize(c->d_dyn, (int)c->dyn.size(), w.d_theta, c->d_recs, s);
    }));
    if (fused) ST_TRY(gather_images(c, p, dtype, true, s));
    ST_TRY(run_k("zero_state", 0, sb, s, [&] { return launch_zero_state(dtype, w.phi, c->n_phys, s); }));
    if (fused) ST_TRY(run_fused_forward(c, p, dtype, w.phi, s));
    else ST_TRY(run_plain_forward(c, dtype, w.phi, s));
    // energy and adjoint seed
    if (c->density) {
        const DensMap &m = fused ? c->map_grad : c->map_std;
        ST_TRY(run_k("density_expect", 0, 0, s, [&] {
            return launch_density_expect(dtype, w.phi, c->n_log, m, h->dev(), red, w.d_energy, s);
        }));
        ST_TRY(run_k("density_seed", 0, sb, s, [&] {
            return launch_density_seed(dtype, w.psi, c->n_log, m, h->dev(), s);
        }));
    } else {
        ObsDev od;  // in the plan's gradient layout (copies made before any capture)
        ST_TRY(obs_dev_perm(h, fused ? p->perm : std::vector<int8_t>(), &od));
        ST_TRY(run_k("pauli_expect_seed", (8.0 * h->groups.size() + 4) * amps, 2 * sb, s, [&] {
            return launch_pauli_expect(dtype, w.phi, w.psi, c->n_phys, od, red, w.d_energy, s);
        }));
    }
    if (fused) {
        const int tiles = 1 << (c->n_phys - p->p.t);
        const FusedDev fd{p->d_rev, p->d_rsubs, p->d_rgates, p->d_rents, p->d_runits, c->d_recs, p->d_rimg};
        for (int i = (int)p->p.rev.size() - 1; i >= 0; i--) {
            if (p->p.barrier[i] >= 0) {  // Phi <- S^-1 Phi, Psi <- S^dag Psi (no parameters)
                const PGate &g = p->p.barrier_gates[p->p.barrier[i]];
                ST_TRY(gate4(c, dtype, w.phi, g.q, g.rec_i, s));
                ST_TRY(gate4(c, dtype, w.psi, g.q, g.rec_a, s));
                continue;
            }
            ST_TRY(run_k("fused_reverse", p->p.rev_flops[i] * amps, 4 * sb, s, [&] {
                return launch_fused_reverse(dtype, w.phi, w.psi, fd, i, p->p.rev[i], p->rev_smem[i],
                                            w.d_slot_partials, tiles, s);
            }));
        }
        ST_TRY(run_k("reduce_slots", 0, 0, s, [&] {
            return launch_reduce_slots(w.d_slot_partials, p->p.n_slots, tiles, tiles, w.d_slot_grad, s);
        }));
        ST_TRY(run_k("accumulate", 0, 0, s, [&] {
            return launch_accumulate(w.d_slot_grad, p->d_csr_ptr, p->d_csr_slots, c->n_params, w.d_grad, s);
        }));
    } else {
        // Algorithm 2: Phi <- Q^-1 Phi; g = scale Re <Psi|dQ|Phi>; Psi <- Q^-1 Psi (Q^dag for channels)
        for (int j = (int)c->plain.size() - 1; j >= 0; j--) {
            const PlainGate &g = c->plain[j];
            ST_TRY(plain_gate(c, dtype, w.phi, g, g.rec_i, s));
            if (g.slot >= 0)
                ST_TRY(run_k("dot_derivative", (shape_flops(g.der_k == 1 ? SH_DENSE1 : SH_DENSE2) + 4) * amps, 2 * sb, s,
                             [&] {
                                 return launch_dot_matrix(dtype, w.psi, w.phi, c->n_phys, g.der_k, g.dq0, g.dq1,
                                                          c->d_recs + g.rec_d, g.gscale, red, w.d_slot_grad + g.slot, s);
                             }));
            for (int e = 0; e < g.n_extra; e++)
                ST_TRY(run_k("dot_derivative", (shape_flops(SH_DENSE2) + 4) * amps, 2 * sb, s, [&] {
                    return launch_dot_matrix(dtype, w.psi, w.phi, c->n_phys, g.der_k, g.dq0, g.dq1,
                                             c->d_recs + g.ex_rec[e], g.gscale, red, w.d_slot_grad + g.ex_slot[e], s);
                }));
            ST_TRY(plain_gate(c, dtype, w.psi, g, g.rec_a, s));
        }
        ST_TRY(run_k("accumulate", 0, 0, s, [&] {
            return launch_accumulate(w.d_slot_grad, c->d_plain_ptr, c->d_plain_slots, c->n_params, w.d_grad, s);
        }));
    }
    return GBVQC_OK;
}

extern "C" gbvqc_status grad(circuit_handle c, const double *theta, int n_theta, obs_handle h, int dtype, int mode,
                             int ptr_loc, void *stream, double *energy, double *grad_out)
{
    if (!c || !h || !energy || (!grad_out && c->n_params > 0)) return fail(GBVQC_ERR_ARG, "NULL argument");
    if (dtype != GBVQC_C64 && dtype != GBVQC_C128) return fail(GBVQC_ERR_ARG, "dtype %d", dtype);
    if (mode != GBVQC_MODE_PLAIN && mode != GBVQC_MODE_FUSED) return fail(GBVQC_ERR_ARG, "mode %d", mode);
    if (ptr_loc != GBVQC_PTR_HOST && ptr_loc != GBVQC_PTR_DEVICE) return fail(GBVQC_ERR_ARG, "ptr_loc %d", ptr_loc);
    if (h->n_qubits != c->n_log) return fail(GBVQC_ERR_ARG, "observable has %d qubits, circuit %d", h->n_qubits, c->n_log);
    std::lock_guard<std::mutex> lk(c->mu);
    cudaStream_t s = (cudaStream_t)stream;
    ST_TRY(ensure_device(c));
    ST_TRY(ensure_obs(h));
    DevPlan *p = nullptr;
    if (mode == GBVQC_MODE_FUSED && fused_supported(c, dtype)) ST_TRY(get_plan(c, dtype, true, &p));
    else mode = GBVQC_MODE_PLAIN;
    if (p && !c->density) {
        ObsDev od;
        ST_TRY(obs_dev_perm(h, p->perm, &od));
    }
    ST_TRY(ensure_workspace(c, dtype));
    Workspace &w = c->ws;
    // a gradient slot per variational physical gate: at most two per op (ket and bra)
    if (!w.d_slot_grad) ST_TRY(dev_alloc(&w.d_slot_grad, (size_t)2 * c->n_param_ops + 1));
    if (p) {
        size_t need = (size_t)p->p.n_slots * (size_t(1) << (c->n_phys - p->p.t));
        if (need > c->partials_cap) {
            free_graphs(c);
            cudaFree(w.d_slot_partials);
            w.d_slot_partials = nullptr;
            ST_TRY(dev_alloc(&w.d_slot_partials, std::max<size_t>(need, 1)));
            c->partials_cap = std::max<size_t>(need, 1);
        }
    }
    ST_TRY(stage_theta(c, theta, n_theta, ptr_loc, s));
    if (g_prof) {  // grad_profile: plain stream launches with events
        ST_TRY(enqueue_grad(c, h, dtype, mode, p, s));
        cudaMemcpyKind k = ptr_loc == GBVQC_PTR_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
        CUDA_TRY(cudaMemcpyAsync(energy, w.d_energy, sizeof(double), k, s));
        if (c->n_params > 0) CUDA_TRY(cudaMemcpyAsync(grad_out, w.d_grad, sizeof(double) * c->n_params, k, s));
        CUDA_TRY(cudaStreamSynchronize(s));
        return GBVQC_OK;
    }
    // replay the captured launch sequence
    if ((const void *)h != c->graph_obs) {
        free_graphs(c);
        c->graph_obs = h;
    }
    const int gkey = dtype * 2 + mode;
    auto it = c->graphs.find(gkey);
    if (it == c->graphs.end()) {
        cudaGraph_t graph = nullptr;
        CUDA_TRY(cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
        gbvqc_status st = enqueue_grad(c, h, dtype, mode, p, c->cap_stream);
        cudaError_t e = cudaStreamEndCapture(c->cap_stream, &graph);
        if (st != GBVQC_OK) {
            if (graph) cudaGraphDestroy(graph);
            return st;
        }
        CUDA_TRY(e);
        cudaGraphExec_t exec = nullptr;
        e = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        CUDA_TRY(e);
        it = c->graphs.emplace(gkey, exec).first;
    }
    CUDA_TRY(cudaGraphLaunch(it->second, s));
    cudaMemcpyKind kind = ptr_loc == GBVQC_PTR_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    CUDA_TRY(cudaMemcpyAsync(energy, w.d_energy, sizeof(double), kind, s));
    if (c->n_params > 0) CUDA_TRY(cudaMemcpyAsync(grad_out, w.d_grad, sizeof(double) * c->n_params, kind, s));
    if (ptr_loc == GBVQC_PTR_HOST) CUDA_TRY(cudaStreamSynchronize(s));
    return GBVQC_OK;
}

extern "C" gbvqc_status grad_profile(circuit_handle c, const double *theta, int n_theta, obs_handle h, int dtype,
                                     int mode, void *stream, gbvqc_kernel_stat *stats, int max_stats, int *n_stats)
{
    if (!stats || !n_stats || max_stats < 0) return fail(GBVQC_ERR_ARG, "NULL argument");
    std::vector<ProfRec> recs;
    std::vector<double> g(c ? std::max(c->n_params, 1) : 1);
    double e = 0;
    g_prof = &recs;
    gbvqc_status st = grad(c, theta, n_theta, h, dtype, mode, GBVQC_PTR_HOST, stream, &e, g.data());
    g_prof = nullptr;
    std::vector<gbvqc_kernel_stat> agg;
    for (ProfRec &r : recs) {
        float ms = 0;
        if (st == GBVQC_OK && cudaEventElapsedTime(&ms, r.a, r.b) != cudaSuccess)
            st = fail(GBVQC_ERR_CUDA, "event timing failed");
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
        size_t i = 0;
        while (i < agg.size() && r.name != agg[i].name) i++;
        if (i == agg.size()) {
            gbvqc_kernel_stat k{};
            snprintf(k.name, sizeof k.name, "%s", r.name.c_str());
            agg.push_back(k);
        }
        agg[i].launches++;
        agg[i].ms += ms;
        agg[i].alg_flops += r.flops;
        agg[i].alg_bytes += r.bytes;
    }
    if (st != GBVQC_OK) return st;
    *n_stats = (int)std::min<size_t>(agg.size(), (size_t)max_stats);
    for (int i = 0; i < *n_stats; i++) stats[i] = agg[i];
    return GBVQC_OK;
}

// ---------------------------------------------------------------------- autotuner

// FNV-1a hash of the circuit's structure (kinds, qubits, variational flags, sizes).
static uint64_t circuit_key(const gbvqc_circuit *c, int dtype)
{
    uint64_t h = 1469598103934665603ull;
    auto mix = [&](uint64_t v) {
        for (int i = 0; i < 8; i++) {
            h ^= (v >> (8 * i)) & 0xff;
            h *= 1099511628211ull;
        }
    };
    mix((uint64_t)c->n_log);
    mix((uint64_t)c->density);
    mix((uint64_t)dtype);
    for (const gbvqc_op &op : c->ops) {
        mix((uint64_t)op.kind);
        mix((uint64_t)op.qubits[0] | ((uint64_t)op.qubits[1] << 32));
        mix((uint64_t)(op.param_index >= 0));
    }
    return h;
}

static std::string tune_cache_path()
{
    const char *env = getenv("GBVQC_TUNE_CACHE");
    if (env && strcmp(env, "off") == 0) return "";
    if (env && *env) return env;
    const char *home = getenv("HOME");
    if (!home) return "";
    return std::string(home) + "/.cache/gbvqc/autotune.txt";
}

static std::string device_name()
{
    int dev = 0;
    cudaDeviceProp prop{};
    if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&prop, dev) != cudaSuccess) return "unknown";
    std::string n = prop.name;
    for (char &ch : n)
        if (ch == ' ') ch = '_';
    return n;
}

extern "C" gbvqc_status circuit_autotune(circuit_handle c, const double *theta, int n_theta, obs_handle h, int dtype,
                                         void *stream, int *best_tile, int *best_low, double *best_ms)
{
    if (!c || !h || !best_tile || !best_low || !best_ms) return fail(GBVQC_ERR_ARG, "NULL argument");
    if (dtype != GBVQC_C64 && dtype != GBVQC_C128) return fail(GBVQC_ERR_ARG, "dtype %d", dtype);
    if (n_theta != c->n_params) return fail(GBVQC_ERR_ARG, "expected %d parameters, got %d", c->n_params, n_theta);
    if (!fused_supported(c, dtype)) return fail(GBVQC_ERR_UNSUPPORTED, "too few qubits for tiles");
    const std::string path = tune_cache_path(), dev = device_name();
    char key[64];
    snprintf(key, sizeof key, "%016llx", (unsigned long long)circuit_key(c, dtype));
    if (!path.empty()) {
        std::ifstream in(path);
        std::string line;
        while (std::getline(in, line)) {
            std::istringstream ls(line);
            std::string k, d;
            int t = 0, lo = 0;
            double ms = 0;
            if ((ls >> k >> d >> t >> lo >> ms) && k == key && d == dev) {
                ST_TRY(circuit_set_tiling(c, t, lo));
                *best_tile = t;
                *best_low = lo;
                *best_ms = ms;
                return GBVQC_OK;
            }
        }
    }
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<double> g(std::max(c->n_params, 1));
    double e = 0;
    cudaEvent_t e0, e1;
    CUDA_TRY(cudaEventCreate(&e0));
    CUDA_TRY(cudaEventCreate(&e1));
    const int nr_max = std::max(fused_nr(dtype, false), fused_nr(dtype, true));
    const int t_hi = std::min(c->n_phys, max_tile(dtype));
    // median over `batches` timed batches of `per` gradient evaluations
    auto time_grad = [&](int batches, int per, double *out_ms) -> gbvqc_status {
        std::vector<double> runs;
        for (int r = 0; r < batches; r++) {
            cudaEventRecord(e0, s);
            for (int k = 0; k < per; k++)
                ST_TRY(grad(c, theta, n_theta, h, dtype, GBVQC_MODE_FUSED, GBVQC_PTR_HOST, s, &e, g.data()));
            cudaEventRecord(e1, s);
            cudaEventSynchronize(e1);
            float ms = 0;
            cudaEventElapsedTime(&ms, e0, e1);
            runs.push_back(ms / per);
        }
        std::sort(runs.begin(), runs.end());
        *out_ms = runs[runs.size() / 2];
        return GBVQC_OK;
    };
    struct Cand {
        double ms;
        int t, lo;
    };
    std::vector<Cand> cands;
    gbvqc_status st = GBVQC_OK;
    for (int t = std::max(8, nr_max + 1); t <= t_hi && st == GBVQC_OK; t++) {
        for (int lo = 2; lo <= 4 && st == GBVQC_OK; lo++) {
            if (lo > t) continue;
            st = circuit_set_tiling(c, t, lo);
            if (st == GBVQC_OK) st = grad(c, theta, n_theta, h, dtype, GBVQC_MODE_FUSED, GBVQC_PTR_HOST, s, &e, g.data());
            if (st != GBVQC_OK) {
                if (st == GBVQC_ERR_UNSUPPORTED) st = GBVQC_OK;  // e.g. a plan exceeding shared memory
                continue;
            }
            double ms = 0;
            st = time_grad(3, 2, &ms);  // coarse: median of three batches of two
            if (st == GBVQC_OK) cands.push_back(Cand{ms, t, lo});
        }
    }
    // refine the three fastest with longer measurements (close candidates differ by ~1%)
    std::sort(cands.begin(), cands.end(), [](const Cand &x, const Cand &y) { return x.ms < y.ms; });
    double best = 1e30;
    int bt = 0, bl = 0;
    for (size_t i = 0; i < cands.size() && i < 3 && st == GBVQC_OK; i++) {
        st = circuit_set_tiling(c, cands[i].t, cands[i].lo);
        double ms = 0;
        if (st == GBVQC_OK) st = time_grad(7, 6, &ms);
        if (st == GBVQC_OK && ms < best) {
            best = ms;
            bt = cands[i].t;
            bl = cands[i].lo;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != GBVQC_OK) return st;
    if (bt == 0) return fail(GBVQC_ERR_UNSUPPORTED, "no tiling could be planned");
    ST_TRY(circuit_set_tiling(c, bt, bl));
    *best_tile = bt;
    *best_low = bl;
    *best_ms = best;
    if (!path.empty()) {
        const size_t slash = path.rfind('/');
        if (slash != std::string::npos) {
            std::string dir = path.substr(0, slash), cmd;
            for (size_t i = 1; i <= dir.size(); i++)  // mkdir -p
                if (i == dir.size() || dir[i] == '/') {
                    std::string sub = dir.substr(0, i);
                    if (!sub.empty()) mkdir_quiet(sub.c_str());
                }
        }
        std::ofstream out(path, std::ios::app);
        if (out) out << key << ' ' << dev << ' ' << bt << ' ' << bl << ' ' << std::setprecision(17) << best << '\n';
    }
    return GBVQC_OK;
}

// ------------------------------------------------------------------------ batches

struct BatchLaunch {
    bool twoq;
    int t;
    FusedBatchEntry *d_entries = nullptr;
    int n_entries = 0;
    int64_t tiles = 0;
    size_t smem = 0;
};

struct gbvqc_batch {
    std::vector<gbvqc_circuit *> circs;
    std::vector<gbvqc_obs *> obs;
    int dtype = 0, n = 0, total_params = 0;
    std::vector<int> param_off;
    void *phi_all = nullptr, *psi_all = nullptr;
    size_t state_bytes = 0;
    int64_t *d_amp_off = nullptr;
    BatchDyn *d_dyn = nullptr;
    int n_dyn = 0;
    double *d_theta = nullptr, *d_energies = nullptr, *d_grads = nullptr, *d_slot_grad = nullptr;
    double *d_slot_partials = nullptr, *d_pauli_partials = nullptr;
    std::vector<BatchLaunch> fwd, rev;
    PauliBatchEntry *d_pauli = nullptr;
    int64_t pauli_chunks = 0;
    size_t pauli_smem = 0;  // staged observables' shared memory (0: global-memory path)
    SlotBatchEntry *d_slots = nullptr;
    int64_t total_slots = 0;
    int *d_csr_ptr = nullptr, *d_csr_slots = nullptr;
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t graph = nullptr;
};

extern "C" gbvqc_status batch_free(batch_handle b)
{
    if (!b) return GBVQC_OK;
    if (b->graph) cudaGraphExecDestroy(b->graph);
    if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
    for (auto *L : {&b->fwd, &b->rev})
        for (BatchLaunch &l : *L) cudaFree(l.d_entries);
    cudaFree(b->phi_all); cudaFree(b->psi_all); cudaFree(b->d_amp_off); cudaFree(b->d_dyn);
    cudaFree(b->d_theta); cudaFree(b->d_energies); cudaFree(b->d_grads); cudaFree(b->d_slot_grad);
    cudaFree(b->d_slot_partials); cudaFree(b->d_pauli_partials); cudaFree(b->d_pauli);
    cudaFree(b->d_slots); cudaFree(b->d_csr_ptr); cudaFree(b->d_csr_slots);
    delete b;
    return GBVQC_OK;
}

static gbvqc_status batch_build(gbvqc_batch *b)
{
    const int n = b->n, dtype = b->dtype;
    const size_t amp = amp_size(dtype);
    std::vector<DevPlan *> plans(n);
    std::vector<int64_t> amp_off(n), slot_off(n), part_off(n), chunk_off(n);
    int64_t amps = 0, slots = 0, parts = 0, chunks = 0;
    int max_passes = 0;
    std::vector<BatchDyn> dyn;
    for (int i = 0; i < n; i++) {
        gbvqc_circuit *c = b->circs[i];
        ST_TRY(ensure_device(c));
        ST_TRY(ensure_obs(b->obs[i]));
        ST_TRY(get_plan(c, dtype, true, &plans[i], true));
        for (int bi : plans[i]->p.barrier)
            if (bi >= 0) return fail(GBVQC_ERR_UNSUPPORTED, "batch member %d holds a two-qubit channel", i);
        const FusedPlan &P = plans[i]->p;
        amp_off[i] = amps;
        amps += int64_t(1) << c->n_phys;
        slot_off[i] = slots;
        slots += P.n_slots;
        part_off[i] = parts;
        parts += (int64_t)P.n_slots << (c->n_phys - P.t);
        chunk_off[i] = chunks;
        chunks += ((int64_t(1) << c->n_phys) + (1 << kPauliChunkBits) - 1) >> kPauliChunkBits;
        max_passes = std::max(max_passes, (int)P.fwd.size());
        for (const DynRec &d : c->dyn)
            dyn.push_back(BatchDyn{c->d_recs + d.rec, b->param_off[i] + d.param, 0, d});
    }
    b->state_bytes = (size_t)amps * amp;
    ST_TRY(dev_alloc((unsigned char **)&b->phi_all, b->state_bytes));
    ST_TRY(dev_alloc((unsigned char **)&b->psi_all, b->state_bytes));
    ST_TRY(upload(&b->d_amp_off, amp_off));
    ST_TRY(upload(&b->d_dyn, dyn));
    b->n_dyn = (int)dyn.size();
    ST_TRY(dev_alloc(&b->d_theta, b->total_params + 1));
    ST_TRY(dev_alloc(&b->d_energies, n));
    ST_TRY(dev_alloc(&b->d_grads, b->total_params + 1));
    ST_TRY(dev_alloc(&b->d_slot_grad, slots + 1));
    ST_TRY(dev_alloc(&b->d_slot_partials, parts + 1));
    ST_TRY(dev_alloc(&b->d_pauli_partials, chunks + 1));
    b->total_slots = slots;
    b->pauli_chunks = chunks;
    auto state_ptr = [&](void *base, int i) { return (void *)((unsigned char *)base + amp_off[i] * amp); };
    // fused launches: pass p of every circuit that has one, grouped by tile size
    CUDA_TRY(fused_batch_prepare());
    for (int dir = 0; dir < 2; dir++) {
        const bool rev = dir == 1;
        for (int r = 0; r < max_passes; r++) {
            std::map<int, std::vector<int>> by_t;
            for (int i = 0; i < n; i++) {
                const int np = (int)plans[i]->p.fwd.size();
                const int p = rev ? np - 1 - r : r;
                if (p >= 0 && p < np) by_t[plans[i]->p.t].push_back(i);
            }
            for (auto &kv : by_t) {
                BatchLaunch L;
                L.t = kv.first;
                L.twoq = false;
                std::vector<FusedBatchEntry> ents;
                for (int i : kv.second) {
                    DevPlan *dp = plans[i];
                    const int np = (int)dp->p.fwd.size();
                    const int p = rev ? np - 1 - r : r;
                    const PassDesc &d = rev ? dp->p.rev[p] : dp->p.fwd[p];
                    FusedBatchEntry e{};
                    if (rev)
                        e.args = FusedArgs{dp->d_rev + p, dp->d_rsubs, dp->d_rgates, dp->d_rents, dp->d_runits,
                                           b->circs[i]->d_recs, nullptr, b->d_slot_partials + part_off[i],
                                           1 << (b->circs[i]->n_phys - dp->p.t)};
                    else
                        e.args = FusedArgs{dp->d_fwd + p, dp->d_fsubs, dp->d_fgates, dp->d_fents, dp->d_funits,
                                           b->circs[i]->d_recs, nullptr, nullptr, 0};
                    e.phi = state_ptr(b->phi_all, i);
                    e.psi = rev ? state_ptr(b->psi_all, i) : nullptr;
                    e.begin = L.tiles;
                    L.tiles += int64_t(1) << (b->circs[i]->n_phys - dp->p.t);
                    L.twoq = L.twoq || d.has_2q;
                    L.smem = std::max(L.smem, rev ? dp->rev_smem[p] : dp->fwd_smem[p]);
                    ents.push_back(e);
                }
                L.n_entries = (int)ents.size();
                ST_TRY(upload(&L.d_entries, ents));
                (rev ? b->rev : b->fwd).push_back(L);
            }
        }
    }
    std::vector<PauliBatchEntry> pe(n);
    std::vector<SlotBatchEntry> se(n);
    std::vector<int> gslot_param(slots, -1);
    for (int i = 0; i < n; i++) {
        ObsDev od;
        ST_TRY(obs_dev_perm(b->obs[i], plans[i]->perm, &od));
        pe[i] = PauliBatchEntry{state_ptr(b->phi_all, i), state_ptr(b->psi_all, i), od,
                                b->d_pauli_partials + chunk_off[i], b->circs[i]->n_phys, 0, chunk_off[i]};
        se[i] = SlotBatchEntry{b->d_slot_partials + part_off[i], 1 << (b->circs[i]->n_phys - plans[i]->p.t), 0,
                               slot_off[i]};
        for (int s = 0; s < plans[i]->p.n_slots; s++)
            gslot_param[slot_off[i] + s] = b->param_off[i] + plans[i]->p.slot_param[s];
    }
    bool staged = true;
    for (int i = 0; i < n; i++) {
        ObsDev od;
        ST_TRY(obs_dev_perm(b->obs[i], plans[i]->perm, &od));
        staged = staged && obs_stageable(od, b->dtype);
        b->pauli_smem = std::max(b->pauli_smem, obs_smem_bytes(od, b->dtype));
    }
    if (!staged) b->pauli_smem = 0;
    ST_TRY(upload(&b->d_pauli, pe));
    ST_TRY(upload(&b->d_slots, se));
    ST_TRY(csr_upload(gslot_param, b->total_params, &b->d_csr_ptr, &b->d_csr_slots));
    CUDA_TRY(cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking));
    return GBVQC_OK;
}

static gbvqc_status batch_enqueue(gbvqc_batch *b, cudaStream_t s)
{
    CUDA_TRY(launch_batch_init(b->d_dyn, b->n_dyn, b->d_theta, b->dtype, b->phi_all, b->state_bytes, b->d_amp_off,
                               b->n, s));
    for (const BatchLaunch &L : b->fwd)
        CUDA_TRY(launch_fused_batch(b->dtype, false, L.twoq, L.t, L.d_entries, L.n_entries, L.tiles, L.smem, s));
    CUDA_TRY(launch_pauli_batch(b->dtype, b->d_pauli, b->n, b->pauli_chunks, b->pauli_smem, b->d_energies, s));
    for (const BatchLaunch &L : b->rev)
        CUDA_TRY(launch_fused_batch(b->dtype, true, L.twoq, L.t, L.d_entries, L.n_entries, L.tiles, L.smem, s));
    CUDA_TRY(launch_slots_batch(b->d_slots, b->n, b->total_slots, b->d_slot_grad, s));
    CUDA_TRY(launch_accumulate(b->d_slot_grad, b->d_csr_ptr, b->d_csr_slots, b->total_params, b->d_grads, s));
    return GBVQC_OK;
}

extern "C" gbvqc_status batch_create(const circuit_handle *circuits, const obs_handle *observables, int n_circuits,
                                     int dtype, batch_handle *out)
{
    if (!out || !circuits || !observables || n_circuits < 1) return fail(GBVQC_ERR_ARG, "bad arguments");
    *out = nullptr;
    if (dtype != GBVQC_C64 && dtype != GBVQC_C128) return fail(GBVQC_ERR_ARG, "dtype %d", dtype);
    gbvqc_batch *b = new gbvqc_batch();
    b->dtype = dtype;
    b->n = n_circuits;
    for (int i = 0; i < n_circuits; i++) {
        gbvqc_circuit *c = circuits[i];
        gbvqc_obs *h = observables[i];
        if (!c || !h) { batch_free(b); return fail(GBVQC_ERR_ARG, "circuit or observable %d is NULL", i); }
        if (c->density) { batch_free(b); return fail(GBVQC_ERR_ARG, "circuit %d is a density circuit", i); }
        if (h->n_qubits != c->n_log) { batch_free(b); return fail(GBVQC_ERR_ARG, "observable %d qubit count", i); }
        if (!fused_supported(c, dtype)) { batch_free(b); return fail(GBVQC_ERR_UNSUPPORTED, "circuit %d: too few qubits", i); }
        b->circs.push_back(c);
        b->obs.push_back(h);
        b->param_off.push_back(b->total_params);
        b->total_params += c->n_params;
    }
    gbvqc_status st = batch_build(b);
    if (st != GBVQC_OK) {
        batch_free(b);
        return st;
    }
    *out = b;
    return GBVQC_OK;
}

extern "C" gbvqc_status batch_grad(batch_handle b, const double *theta_all, int n_theta_total, int ptr_loc,
                                   void *stream, double *energies, double *grads)
{
    if (!b || !energies || (!grads && b->total_params > 0)) return fail(GBVQC_ERR_ARG, "NULL argument");
    if (n_theta_total != b->total_params)
        return fail(GBVQC_ERR_ARG, "expected %d parameters, got %d", b->total_params, n_theta_total);
    if (n_theta_total > 0 && !theta_all) return fail(GBVQC_ERR_ARG, "theta is NULL");
    if (ptr_loc != GBVQC_PTR_HOST && ptr_loc != GBVQC_PTR_DEVICE) return fail(GBVQC_ERR_ARG, "ptr_loc %d", ptr_loc);
    cudaStream_t s = (cudaStream_t)stream;
    const cudaMemcpyKind in = ptr_loc == GBVQC_PTR_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    const cudaMemcpyKind outk = ptr_loc == GBVQC_PTR_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (n_theta_total > 0) CUDA_TRY(cudaMemcpyAsync(b->d_theta, theta_all, sizeof(double) * n_theta_total, in, s));
    if (!b->graph) {
        cudaGraph_t graph = nullptr;
        CUDA_TRY(cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal));
        gbvqc_status st = batch_enqueue(b, b->cap_stream);
        cudaError_t e = cudaStreamEndCapture(b->cap_stream, &graph);
        if (st != GBVQC_OK) {
            if (graph) cudaGraphDestroy(graph);
            return st;
        }
        CUDA_TRY(e);
        e = cudaGraphInstantiate(&b->graph, graph, 0);
        cudaGraphDestroy(graph);
        CUDA_TRY(e);
    }
    CUDA_TRY(cudaGraphLaunch(b->graph, s));
    CUDA_TRY(cudaMemcpyAsync(energies, b->d_energies, sizeof(double) * b->n, outk, s));
    if (b->total_params > 0)
        CUDA_TRY(cudaMemcpyAsync(grads, b->d_grads, sizeof(double) * b->total_params, outk, s));
    if (ptr_loc == GBVQC_PTR_HOST) CUDA_TRY(cudaStreamSynchronize(s));
    return GBVQC_OK;
}

extern "C" gbvqc_status grad_batch(const circuit_handle *circuits, const obs_handle *observables, int n_circuits,
                                   const double *theta_all, void *stream, double *energies, double *grads)
{
    batch_handle b = nullptr;
    ST_TRY(batch_create(circuits, observables, n_circuits, GBVQC_C64, &b));
    gbvqc_status st = batch_grad(b, theta_all, b->total_params, GBVQC_PTR_HOST, stream, energies, grads);
    batch_free(b);
    return st;
}
