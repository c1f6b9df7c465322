// C ABI: errors, states (Sec. II.A), observables and expectation (Sec. II.E),
// measurement and sampling (Sec. II.D), single channels on density states.
#include <cstdarg>
#include <unordered_map>
#include <sys/stat.h>

#include "api_internal.h"

// ------------------------------------------------------------------------ errors

static thread_local std::string g_last_error;

gbvqc_status fail(gbvqc_status st, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return st;
}


// ----------------------------------------------------------------- profiling hooks

thread_local std::vector<ProfRec> *g_prof = nullptr;


// Real floating-point operations per amplitude of one matrix application.
double shape_flops(int sh)
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


// ------------------------------------------------------------------------- basics

extern "C" const char *gbvqc_last_error(void) { return g_last_error.c_str(); }
void gbvqc_internal_set_error(const char *msg) { g_last_error = msg; }
extern "C" int gbvqc_version(void) { return 200; }

// ----------------------------------------------------------------- device memory

namespace {
std::mutex g_mem_mu;
std::unordered_map<void *, size_t> g_mem_live;  // the library's live allocations
int64_t g_mem_bytes = 0, g_mem_count = 0;       // live bytes, allocations ever made
int64_t g_mem_limit = -2;                        // -2: not read yet, -1: no limit

int64_t mem_limit()
{
    if (g_mem_limit == -2) {
        const char *env = getenv("GBVQC_DEVICE_ALLOC_LIMIT");
        char *end = nullptr;
        const long long v = env && *env ? strtoll(env, &end, 10) : -1;
        g_mem_limit = (env && *env && end && *end == '\0' && v >= 0) ? (int64_t)v : -1;
    }
    return g_mem_limit;
}
}  // namespace

gbvqc_status dev_alloc_bytes(void **p, size_t bytes)
{
    *p = nullptr;
    std::lock_guard<std::mutex> lk(g_mem_mu);
    const int64_t limit = mem_limit();
    if (limit >= 0 && g_mem_bytes + (int64_t)bytes > limit)
        return fail(GBVQC_ERR_OOM, "device allocation of %zu bytes exceeds GBVQC_DEVICE_ALLOC_LIMIT (%lld live of %lld)",
                    bytes, (long long)g_mem_bytes, (long long)limit);
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return fail(e == cudaErrorMemoryAllocation ? GBVQC_ERR_OOM : GBVQC_ERR_CUDA, "cudaMalloc of %zu bytes: %s",
                    bytes, cudaGetErrorString(e));
    }
    g_mem_live[*p] = bytes;
    g_mem_bytes += (int64_t)bytes;
    g_mem_count++;
    return GBVQC_OK;
}

void dev_free(void *p)
{
    if (!p) return;
    {
        std::lock_guard<std::mutex> lk(g_mem_mu);
        auto it = g_mem_live.find(p);
        if (it != g_mem_live.end()) {
            g_mem_bytes -= (int64_t)it->second;
            g_mem_live.erase(it);
        }
    }
    cudaFree(p);
}

extern "C" gbvqc_status gbvqc_mem_info(int64_t *live_bytes, int64_t *allocations)
{
    std::lock_guard<std::mutex> lk(g_mem_mu);
    if (live_bytes) *live_bytes = g_mem_bytes;
    if (allocations) *allocations = g_mem_count;
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
    if (s->owned && s->data) dev_free(s->data);
    if (s->d_scratch) dev_free(s->d_scratch);
    if (s->d_counter) dev_free(s->d_counter);
    if (s->d_rec) dev_free(s->d_rec);
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

std::vector<unsigned char> chunk_image(const std::vector<ObsGroup> &groups, const std::vector<ObsTerm> &terms)
{
    const int G = (int)groups.size(), T = (int)terms.size();
    std::vector<unsigned char> img(chunk_image_bytes(G, T), 0);
    ChunkGroup *cg = reinterpret_cast<ChunkGroup *>(img.data());
    ChunkTermF *tf = reinterpret_cast<ChunkTermF *>(img.data() + chunk_terms_f_offset(G));
    ChunkTermD *td = reinterpret_cast<ChunkTermD *>(img.data() + chunk_terms_d_offset(G, T));
    for (int g = 0; g < G; g++) {
        const uint64_t x = groups[g].x;
        uint32_t flags = 0, real = 1, zany = 0;
        for (int k = groups[g].t_begin; k < groups[g].t_end; k++) {
            const ObsTerm &t = terms[k];
            real &= (t.ph & 1) == 0;
            zany |= t.z != 0;
            // i^{ph} (-1)^{popcount(x & z)}: the coefficient as seen from amplitude a
            const int ph = (t.ph + 2 * (__builtin_popcountll(x & t.z) & 1)) & 3;
            uint32_t rpat = 0;
            const uint32_t zr = (uint32_t)(t.z >> kPauliTB) & (kPauliPV - 1);
            for (int r = 0; r < kPauliPV; r++) rpat |= (uint32_t)(__builtin_popcount(r & zr) & 1) << r;
            const double c = t.coeff;
            const float cf = t.coeff_f;
            tf[k] = ChunkTermF{(uint32_t)t.z, (uint32_t)(t.z >> 32), rpat, ph == 0 ? cf : ph == 2 ? -cf : 0.0f,
                               ph == 1 ? cf : ph == 3 ? -cf : 0.0f, 0u};
            td[k] = ChunkTermD{(uint32_t)t.z, (uint32_t)(t.z >> 32), rpat, 0u, ph == 0 ? c : ph == 2 ? -c : 0.0,
                               ph == 1 ? c : ph == 3 ? -c : 0.0};
        }
        if (real) flags |= CG_REAL;
        if (x == 0) flags |= CG_SELF;
        if ((x >> kPauliC) == 0) flags |= CG_CHUNK;
        if (!zany) flags |= CG_CONST;
        cg[g] = ChunkGroup{(uint32_t)x, (uint32_t)(x >> 32), (uint16_t)groups[g].t_begin, (uint16_t)groups[g].t_end,
                           flags};
    }
    return img;
}

gbvqc_status ensure_obs(gbvqc_obs *h)
{
    if (h->d_groups) return GBVQC_OK;
    CUDA_TRY(pauli_prepare());
    ST_TRY(upload(&h->d_terms, h->terms));
    ST_TRY(upload(&h->d_groups, h->groups));
    if (h->terms.size() < 65536) ST_TRY(upload(&h->d_chunk, chunk_image(h->groups, h->terms)));
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
gbvqc_status obs_dev_perm(gbvqc_obs *h, const std::vector<int8_t> &perm, ObsDev *out)
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
        gbvqc_obs::PermDev d{nullptr, nullptr, nullptr};
        ST_TRY(upload(&d.groups, g));
        ST_TRY(upload(&d.terms, t));
        if (t.size() < 65536) ST_TRY(upload(&d.chunk, chunk_image(g, t)));
        it = h->perm_dev.emplace(perm, d).first;
    }
    *out = ObsDev{it->second.groups, it->second.terms, (int)h->groups.size(), (int)h->terms.size(), it->second.chunk};
    return GBVQC_OK;
}

extern "C" gbvqc_status obs_free(obs_handle h)
{
    if (!h) return GBVQC_OK;
    if (h->d_groups) dev_free(h->d_groups);
    if (h->d_terms) dev_free(h->d_terms);
    if (h->d_chunk) dev_free(h->d_chunk);
    for (auto &kv : h->perm_dev) {
        dev_free(kv.second.groups);
        dev_free(kv.second.terms);
        dev_free(kv.second.chunk);
    }
    delete h;
    return GBVQC_OK;
}

DensMap standard_map(int n)
{
    DensMap m{};
    for (int q = 0; q < n; q++) {
        m.ket[q] = (int8_t)q;
        m.bra[q] = (int8_t)(q + n);
    }
    return m;
}

DensMap interleaved_map(int n)
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
    dev_free(d_buf);
    dev_free(d_out);
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
