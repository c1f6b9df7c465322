// Plan-time specialisation of the fused tile passes: code generation from the plan's
// records, runtime compilation with NVRTC (loaded on first use, so the library itself
// does not depend on it), an on-disk cubin cache, and module loading through the CUDA
// runtime's library API.
#include "jit.h"

#include <cuda_runtime.h>
#include <dlfcn.h>
#include <nvrtc.h>
#include <sys/stat.h>
#include <unistd.h>

#include <atomic>
#include <chrono>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <mutex>
#include <sstream>
#include <thread>

namespace gbvqc {

// Device headers the generated source includes, embedded at build time (jit_headers.cpp,
// written by build.py from the csrc/ headers).
extern const int kJitHeaderCount;
extern const char *const kJitHeaderNames[];
extern const char *const kJitHeaderSources[];

namespace {

// --------------------------------------------------------------------------- NVRTC

struct Nvrtc {
    bool ok = false;
    std::string why;
    nvrtcResult (*create)(nvrtcProgram *, const char *, const char *, int, const char *const *,
                          const char *const *) = nullptr;
    nvrtcResult (*compile)(nvrtcProgram, int, const char *const *) = nullptr;
    nvrtcResult (*log_size)(nvrtcProgram, size_t *) = nullptr;
    nvrtcResult (*log)(nvrtcProgram, char *) = nullptr;
    nvrtcResult (*cubin_size)(nvrtcProgram, size_t *) = nullptr;
    nvrtcResult (*cubin)(nvrtcProgram, char *) = nullptr;
    nvrtcResult (*destroy)(nvrtcProgram *) = nullptr;
    nvrtcResult (*version)(int *, int *) = nullptr;
};

const Nvrtc &nvrtc()
{
    static Nvrtc lib;
    static std::once_flag once;
    std::call_once(once, [] {
        const char *names[] = {"libnvrtc.so.13", "libnvrtc.so", "/usr/local/cuda/lib64/libnvrtc.so.13",
                               "/usr/local/cuda/lib64/libnvrtc.so"};
        void *h = nullptr;
        for (const char *n : names)
            if ((h = dlopen(n, RTLD_NOW | RTLD_LOCAL))) break;
        if (!h) {
            lib.why = "NVRTC (libnvrtc.so.13) could not be loaded";
            return;
        }
        auto sym = [&](const char *n) { return dlsym(h, n); };
        lib.create = (decltype(lib.create))sym("nvrtcCreateProgram");
        lib.compile = (decltype(lib.compile))sym("nvrtcCompileProgram");
        lib.log_size = (decltype(lib.log_size))sym("nvrtcGetProgramLogSize");
        lib.log = (decltype(lib.log))sym("nvrtcGetProgramLog");
        lib.cubin_size = (decltype(lib.cubin_size))sym("nvrtcGetCUBINSize");
        lib.cubin = (decltype(lib.cubin))sym("nvrtcGetCUBIN");
        lib.destroy = (decltype(lib.destroy))sym("nvrtcDestroyProgram");
        lib.version = (decltype(lib.version))sym("nvrtcVersion");
        lib.ok = lib.create && lib.compile && lib.log_size && lib.log && lib.cubin_size && lib.cubin && lib.destroy &&
                 lib.version;
        if (!lib.ok) lib.why = "NVRTC is missing an entry point";
    });
    return lib;
}

const char *kArch = "--gpu-architecture=sm_103a";

bool compile_source(const std::string &src, const std::string &name, std::string &cubin, std::string &err)
{
    const Nvrtc &L = nvrtc();
    if (!L.ok) {
        err = L.why;
        return false;
    }
    nvrtcProgram prog = nullptr;
    if (L.create(&prog, src.c_str(), (name + ".cu").c_str(), kJitHeaderCount, kJitHeaderSources, kJitHeaderNames) !=
        NVRTC_SUCCESS) {
        err = "nvrtcCreateProgram failed";
        return false;
    }
    const char *opts[] = {kArch, "-std=c++17", "-default-device", "--fmad=true"};
    const nvrtcResult r = L.compile(prog, 4, opts);
    if (r != NVRTC_SUCCESS) {
        size_t n = 0;
        L.log_size(prog, &n);
        std::string log(n, '\0');
        if (n) L.log(prog, &log[0]);
        err = "NVRTC compilation of " + name + " failed: " + log.substr(0, 2000);
        L.destroy(&prog);
        return false;
    }
    size_t n = 0;
    L.cubin_size(prog, &n);
    cubin.assign(n, '\0');
    L.cubin(prog, &cubin[0]);
    L.destroy(&prog);
    return true;
}

// ------------------------------------------------------------------------- cache

uint64_t fnv1a(const std::string &s, uint64_t h = 1469598103934665603ull)
{
    for (unsigned char ch : s) {
        h ^= ch;
        h *= 1099511628211ull;
    }
    return h;
}

std::string cache_dir()
{
    const char *env = getenv("GBVQC_JIT_CACHE");
    if (env && strcmp(env, "off") == 0) return "";
    if (env && *env) return env;
    const char *home = getenv("HOME");
    return home ? std::string(home) + "/.cache/gbvqc/jit" : "";
}

void mkdir_p(const std::string &dir)
{
    for (size_t i = 1; i <= dir.size(); i++)
        if (i == dir.size() || dir[i] == '/') mkdir(dir.substr(0, i).c_str(), 0755);
}

// ------------------------------------------------------------------------ codegen

std::string flit(float v)  // exact literal of a float coefficient
{
    char buf[64];
    snprintf(buf, sizeof buf, "(Rt)%af", (double)v);
    return buf;
}

const char *gen_name(int g) { return g == GEN_X ? "GEN_X" : "GEN_Y"; }

// Bit deposit as shifts and masks: bit i of var goes to position pos[i]; runs of
// consecutive bits landing on consecutive positions are one term.
std::string deposit_expr(const char *var, const std::vector<int> &pos, const char *type)
{
    std::ostringstream o;
    bool first = true;
    for (size_t i = 0; i < pos.size();) {
        size_t j = i + 1;
        while (j < pos.size() && pos[j] == pos[j - 1] + 1) j++;
        const unsigned long long mask = (j - i) >= 64 ? ~0ull : ((1ull << (j - i)) - 1);
        o << (first ? "" : " | ") << "(((" << type << ")(" << var << ") >> " << i << ") & (" << type << ")0x" << std::hex
          << mask << std::dec << "ull) << " << pos[i];
        first = false;
        i = j;
    }
    if (first) o << "(" << type << ")0";
    return o.str();
}

void emit_gate(std::ostringstream &o, const FusedPlan &P, const PassDesc &d, const FGate &g, bool rev, int NR)
{
    const std::vector<DEnt> &E = rev ? P.rents : P.fents;
    const char *ind = "    ";
    if (g.type == FT_LAYER1) {
        o << ind << "{\n";
        std::vector<std::pair<int, std::string>> reads;  // (pass-local slot, value)
        for (int i = 0; i < g.n_ent; i++) {
            const DEnt &e = E[d.ent_begin + g.ent + i];
            const int K = e.ca, SH = e.k;
            if (rev && (e.cls == GEN_X || e.cls == GEN_Y)) {
                const std::string v = "g" + std::to_string(reads.size());
                o << ind << "const Rt " << v << " = gen_xy<Rt, NR, " << K << ", " << gen_name(e.cls) << ">(a, b) * "
                  << flit(e.coef) << ";\n";
                reads.push_back({e.slot - d.slot_begin, v});
            }
            o << ind << "rg1<Rt, NR, " << K << ", " << SH << ">(a, smat + " << 8 * e.mat << ");\n";
            if (rev) o << ind << "rg1<Rt, NR, " << K << ", " << SH << ">(b, smat + " << 8 * e.mat2 << ");\n";
        }
        if (!reads.empty()) {
            bool seq = true;  // the planner numbers a record's gradient slots consecutively
            for (size_t i = 0; i < reads.size(); i++) seq = seq && reads[i].first == reads[0].first + (int)i;
            o << ind << "{ Rt lv[" << reads.size() << "] = {";
            for (size_t i = 0; i < reads.size(); i++) o << (i ? ", " : "") << reads[i].second;
            if (seq) {
                o << "}; emit_partials_seq<Rt, " << reads.size() << ">(rc, " << reads[0].first << ", lv); }\n";
            } else {
                o << "}; const int ls[" << reads.size() << "] = {";
                for (size_t i = 0; i < reads.size(); i++) o << (i ? ", " : "") << reads[i].first;
                o << "}; emit_partials<Rt, " << reads.size() << ">(rc, ls, lv); }\n";
            }
        }
        o << ind << "}\n";
        return;
    }
    if (g.type == FT_DIAGB) {
        const int off = g.ent + (rev ? g.nz : 0);
        if (rev && g.nz > 0) {
            bool seq = true;
            for (int i = 0; i < g.nz; i++)
                seq = seq && E[d.ent_begin + g.ent + i].slot == E[d.ent_begin + g.ent].slot + i;
            o << ind << "{ Rt tot, dk[NR]; z_sums<Rt, NR>(a, b, tot, dk);\n" << ind << "  const int ls[" << (int)g.nz
              << "] = {";
            for (int i = 0; i < g.nz; i++) o << (i ? ", " : "") << E[d.ent_begin + g.ent + i].slot - d.slot_begin;
            o << "};\n" << ind << "  (void)ls;\n" << ind << "  Rt lv[" << (int)g.nz << "] = {";
            for (int i = 0; i < g.nz; i++) {
                const DEnt &z = E[d.ent_begin + g.ent + i];
                if (i) o << ", ";
                if (z.ca >= 0 && z.ca < NR) o << "dk[" << (int)z.ca << "] * " << flit(z.coef);
                else o << "(const_bit<NR>(" << (int)z.ca << ", base, tilebase) ? -tot : tot) * " << flit(z.coef);
            }
            if (seq)
                o << "};\n" << ind << "  emit_partials_seq<Rt, " << (int)g.nz << ">(rc, "
                  << E[d.ent_begin + g.ent].slot - d.slot_begin << ", lv); }\n";
            else
                o << "};\n" << ind << "  emit_partials<Rt, " << (int)g.nz << ">(rc, ls, lv); }\n";
        }
        const bool table = g.flags & FLAG_TABLE, sep = rev && (g.flags & FLAG_SEPARATE);
        const int cs = 4 * g.slot;
        auto call = [&](const char *x, const char *y, bool second) {
            o << ind << (table ? "phase_table" : "phase_block") << "<Rt, NR>(sents + " << off << ", " << g.perm
              << ", smat, ";
            if (table) o << (second ? g.mat2 : g.mat) << ", ";
            o << (second ? "true" : "false") << ", c.sconst[" << cs + (second ? 2 : 0) << "], c.sconst["
              << cs + (second ? 3 : 1) << "], " << x << ", " << y << ", base, tilebase);\n";
        };
        if (!rev) call("a", "nullptr", false);
        else if (sep) {
            call("a", "nullptr", false);
            call("b", "nullptr", true);
        } else {
            call("a", "b", false);
        }
        return;
    }
    if (g.type == FT_PROBE2) {
        if (rev)
            o << ind << "emit_partial<Rt>(rc, " << g.slot << ", probe2_dispatch<Rt, NR>(" << (int)g.a << ", "
              << (int)g.b << ", a, b, smat + " << 8 * g.mat << ") * " << flit(g.coef) << ");\n";
        return;
    }
    if (rev && (g.gen == GEN_X || g.gen == GEN_Y))
        o << ind << "emit_partial<Rt>(rc, " << g.slot << ", gen_xy<Rt, NR, " << (int)g.gpos << ", " << gen_name(g.gen)
          << ">(a, b) * " << flit(g.coef) << ");\n";
    if (g.type == FT_BLOCK2 && (g.perm & BLOCK2_VARIANT)) {  // fixed matrix: its own structure
        const int inner = (g.perm & 3) == 1 ? SH_IMAG1 : (g.perm & 3) == 2 ? SH_REAL1 : SH_DENSE1;
        std::ostringstream t;
        t << "rg2_block2v<Rt, NR, " << (int)g.a << ", " << (int)g.b << ", " << inner << ", "
          << ((g.perm & BLOCK2_P00_ONE) ? "false" : "true") << ", " << ((g.perm & BLOCK2_P11_ONE) ? "false" : "true")
          << ">";
        o << ind << t.str() << "(a, smat + " << 8 * g.mat << ");\n";
        if (rev) o << ind << t.str() << "(b, smat + " << 8 * g.mat2 << ");\n";
        return;
    }
    const char *twoq = d.has_2q ? "true" : "false";
    o << ind << "apply_fgate<Rt, NR, " << twoq << ">(" << (int)g.type << ", " << (int)g.a << ", " << (int)g.b << ", "
      << g.perm << ", smat + " << 8 * g.mat << ", a);\n";
    if (rev)
        o << ind << "apply_fgate<Rt, NR, " << twoq << ">(" << (int)g.type << ", " << (int)g.a << ", " << (int)g.b
          << ", " << g.perm << ", smat + " << 8 * g.mat2 << ", b);\n";
}

}  // namespace

int jit_nr(int dtype, bool reverse, int64_t tiles)
{
    if (dtype != 0) return reverse ? 3 : 4;
    // measured: a 20-qubit state (256 tiles) forward 5 -> 4 takes the gradient step from
    // 0.767 to 0.663 ms (twice the warps); a 28-qubit one (65536 tiles) is 73.5 -> 79.0 ms
    // slower with 4 (warps to spare, fewer sub-runs with 5)
    if (reverse) return 4;
    return tiles < 1024 ? 4 : 5;
}

// CTAs per SM the register budget is cut for: 128-thread passes (the 12-qubit tiles of
// large states) fit four at 128 registers without spills (complex64); measured on the
// 28-qubit sweep: two CTAs per SM 71.0 ms, three 61.8 ms
int jit_min_blocks(int threads) { return threads >= 256 ? 2 : threads == 128 ? 4 : 3; }

std::string jit_kernel_name(int p, bool rev) { return std::string(rev ? "gbvqc_jit_r" : "gbvqc_jit_f") + std::to_string(p); }

std::string jit_source(const FusedPlan &P, int p, bool rev, int dtype)
{
    const PassDesc &d = rev ? P.rev[p] : P.fwd[p];
    const std::vector<SubRun> &subs = rev ? P.rsubs : P.fsubs;
    const std::vector<FGate> &gates = rev ? P.rgates : P.fgates;
    const int NR = rev ? P.nr_r : P.nr_f;
    // the pass's tile geometry as literals: tile index -> qubits outside the tile (ascending),
    // high local bits -> tile qubits low..t-1
    std::vector<int> ns, hs;
    for (int i = 0; i < d.n - d.t; i++) ns.push_back(d.NS[i]);
    for (int i = d.low; i < d.t; i++) hs.push_back(d.S[i]);
    const std::string geom = "struct Geom {\n  static constexpr bool kStatic = true;\n  static constexpr int kThreads = " +
                             std::to_string(1 << (d.t - NR)) + ";\n"
                             "  __device__ static int64_t tilebase(int64_t tile) { return " +
                             deposit_expr("tile", ns, "int64_t") +
                             "; }\n  __device__ static int64_t hi(int h) { return " + deposit_expr("h", hs, "int64_t") +
                             "; }\n};\n";
    std::ostringstream o;
    o << "// specialised " << (rev ? "reverse" : "forward") << " tile pass " << p << " (generated)\n"
      << "#include \"fused_tile.cuh\"\nusing namespace gbvqc;\n"
      << "typedef " << (dtype == 0 ? "float" : "double") << " Rt;\ntypedef CT<Rt>::T Tt;\n"
      << geom << "extern \"C\" __global__ void __launch_bounds__(" << (1 << (d.t - NR)) << ", "
      << jit_min_blocks(1 << (d.t - NR)) << ") " << jit_kernel_name(p, rev)
      << "(Tt *__restrict__ phi, Tt *__restrict__ psi, const FusedArgs args)\n{\n"
      << "  constexpr int NR = " << NR << ";\n  constexpr bool REV = " << (rev ? "true" : "false") << ";\n"
      << "  // a code-prefetch launch (args.dry) runs tile 0 and CTA s walks sub-run s only\n"
      << "  const int64_t tile = args.dry ? 0 : blockIdx.x;\n"
      << "  TileCtx<Rt, NR, REV> c;\n  if (!tile_begin<Rt, NR, REV, Geom>(phi, psi, args, tile, c)) return;\n"
      << "  Tt a[1 << NR], b[REV ? (1 << NR) : 1];\n"
      << "  const Rt *smat = c.smat;\n  const DEnt *sents = c.sents;\n  const RedCtx<Rt> &rc = c.rc;\n"
      << "  const int64_t tilebase = c.tilebase;\n  (void)sents; (void)rc; (void)tilebase; (void)b;\n";
    for (int s = 0; s < d.n_sub; s++) {
        const SubRun &sr = subs[d.sub_begin + s];
        // thread bit i -> i-th lowest tile position outside the sub-run's registers
        std::vector<int> bpos;
        for (int q = 0; q < d.t; q++) {
            bool reg = false;
            for (int k = 0; k < NR; k++) reg = reg || sr.R[k] == q;
            if (!reg) bpos.push_back(q);
        }
        o << "  if (!args.dry || blockIdx.x == " << s << ") {  // sub-run " << s << "\n    const int off[NR] = {";
        for (int k = 0; k < NR; k++) o << (k ? ", " : "") << (1 << (int)sr.R[k]);
        o << "};\n    const int base = " << deposit_expr("threadIdx.x", bpos, "int")
          << ";\n    subrun_gather<Rt, NR, REV>(c, base, off, a, b);\n";
        for (int gi = sr.g_begin; gi < sr.g_end; gi++) emit_gate(o, P, d, gates[d.gate_begin + gi], rev, NR);
        o << "    subrun_store<Rt, NR, REV>(c, base, off, a, b);\n  }\n";
    }
    o << "  tile_end<Rt, NR, REV, Geom>(phi, psi, args, tile, c);\n}\n";
    return o.str();
}

bool jit_compile(const FusedPlan &P, int dtype, bool want_rev, std::vector<JitModule> &tasks, double &secs,
                 std::string &err)
{
    const Nvrtc &L = nvrtc();
    const size_t np = P.fwd.size();
    typedef JitModule Task;
    tasks.clear();
    for (int dir = 0; dir < (want_rev ? 2 : 1); dir++)
        for (size_t p = 0; p < np; p++) {
            if (P.barrier[p] >= 0) continue;  // a two-qubit channel: the per-gate kernel runs it
            Task t;
            t.p = (int)p;
            t.rev = dir == 1;
            t.name = jit_kernel_name(t.p, t.rev);
            t.src = jit_source(P, t.p, t.rev, dtype);
            tasks.push_back(std::move(t));
        }
    // the cache key covers the source, the embedded headers, NVRTC's version and the options
    int vmaj = 0, vmin = 0;
    if (L.ok) L.version(&vmaj, &vmin);
    uint64_t hdr = fnv1a(std::string(kArch) + "|" + std::to_string(vmaj) + "." + std::to_string(vmin));
    for (int i = 0; i < kJitHeaderCount; i++) hdr = fnv1a(kJitHeaderSources[i], fnv1a(kJitHeaderNames[i], hdr));
    const std::string dir = cache_dir();
    if (!dir.empty()) mkdir_p(dir);
    for (Task &t : tasks) {
        char key[32];
        snprintf(key, sizeof key, "%016llx", (unsigned long long)fnv1a(t.src, hdr));
        if (dir.empty()) continue;
        t.path = dir + "/" + key + ".cubin";
        std::ifstream in(t.path, std::ios::binary);
        if (in) {
            std::stringstream ss;
            ss << in.rdbuf();
            t.cubin = ss.str();
            t.from_cache = !t.cubin.empty();
        }
    }
    // compile what the cache does not hold, in parallel (independent NVRTC programs)
    std::vector<size_t> todo;
    for (size_t i = 0; i < tasks.size(); i++)
        if (!tasks[i].from_cache) todo.push_back(i);
    const auto t0 = std::chrono::steady_clock::now();
    if (!todo.empty()) {
        std::atomic<size_t> next(0);
        std::mutex emu;
        std::string first_err;
        const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
        const size_t nthreads = std::min<size_t>(todo.size(), hw);
        std::vector<std::thread> pool;
        for (size_t w = 0; w < nthreads; w++)
            pool.emplace_back([&] {
                for (size_t k; (k = next++) < todo.size();) {
                    Task &t = tasks[todo[k]];
                    std::string e;
                    if (!compile_source(t.src, t.name, t.cubin, e)) {
                        std::lock_guard<std::mutex> lk(emu);
                        if (first_err.empty()) first_err = e;
                    }
                }
            });
        for (std::thread &th : pool) th.join();
        if (!first_err.empty()) {
            err = first_err;
            return false;
        }
        for (size_t i : todo) {
            Task &t = tasks[i];
            if (t.path.empty()) continue;
            const std::string tmp = t.path + ".tmp" + std::to_string((long long)getpid());
            std::ofstream f(tmp, std::ios::binary);
            if (f && f.write(t.cubin.data(), (std::streamsize)t.cubin.size())) {
                f.close();
                rename(tmp.c_str(), t.path.c_str());
            } else {
                remove(tmp.c_str());
            }
        }
    }
    secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    return true;
}

bool jit_build(const FusedPlan &P, int dtype, bool want_rev, JitPlan &out, std::string &err)
{
    out = JitPlan();
    out.dtype = dtype;
    const size_t np = P.fwd.size();
    out.fwd.assign(np, JitPass());
    out.rev.assign(want_rev ? np : 0, JitPass());
    std::vector<JitModule> tasks;
    if (!jit_compile(P, dtype, want_rev, tasks, out.compile_s, err)) return false;
    for (JitModule &t : tasks) {
        JitPass jp;
        cudaLibrary_t lib = nullptr;
        cudaError_t e = cudaLibraryLoadData(&lib, t.cubin.data(), nullptr, nullptr, 0, nullptr, nullptr, 0);
        cudaKernel_t k = nullptr;
        if (e == cudaSuccess) e = cudaLibraryGetKernel(&k, lib, t.name.c_str());
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute((const void *)k, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        if (e != cudaSuccess) {
            if (lib) cudaLibraryUnload(lib);
            jit_free(out);
            err = std::string("loading specialised pass ") + t.name + ": " + cudaGetErrorString(e);
            return false;
        }
        jp.lib = (void *)lib;
        jp.kern = (void *)k;
        (t.rev ? out.rev : out.fwd)[t.p] = jp;
        (t.from_cache ? out.cached : out.compiled)++;
    }
    return true;
}

void jit_free(JitPlan &jp)
{
    for (auto *v : {&jp.fwd, &jp.rev})
        for (JitPass &p : *v)
            if (p.lib) {
                cudaLibraryUnload((cudaLibrary_t)p.lib);
                p.lib = p.kern = nullptr;
            }
}

cudaError_t jit_launch(const JitPass &jp, void *phi, void *psi, const FusedArgs &args, unsigned tiles, int threads,
                       size_t smem, cudaStream_t s, bool dry)
{
    FusedArgs a = args;
    a.dry = dry ? 1 : 0;
    void *params[] = {&phi, &psi, &a};
    return cudaLaunchKernel((const void *)jp.kern, dim3(tiles), dim3(threads), params, smem, s);
}

}  // namespace gbvqc
