// C ABI: the tile autotuner (times grad over tilings, caches the choice on disk).
#include <fstream>
#include <iomanip>
#include <sstream>
#include <sys/stat.h>

#include "api_internal.h"

static void mkdir_quiet(const char *p) { mkdir(p, 0755); }

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
