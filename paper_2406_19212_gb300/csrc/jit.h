// Plan-time specialisation of the fused tile passes.
//
// A circuit's structure (its gates, their qubits and which ones are variational) is fixed
// across the many evaluations of a variational optimisation; only theta changes.  The
// record interpreter of the tile kernels (fused_tile.cuh) decodes every gate record, slot
// and phase-block entry at run time; a specialised pass is the same sequence of device
// functions with every record field written as a literal, compiled once (NVRTC, sm_103a)
// into straight-line code with no decode, no dispatch and the register positions known
// to the compiler.  Matrices stay runtime data (the per-step matrix image), so one
// compilation serves every theta.
#pragma once

#include <string>
#include <vector>

#include "kernels.h"
#include "planner.h"

namespace gbvqc {

struct JitPass {
    void *lib = nullptr;   // cudaLibrary_t of the pass's module
    void *kern = nullptr;  // cudaKernel_t of its kernel
};

struct JitPlan {
    int dtype = 0;
    std::vector<JitPass> fwd, rev;  // per pass of the plan (empty for barrier passes)
    double compile_s = 0;           // wall time of the compilations (0 when all were cached)
    int compiled = 0, cached = 0;   // passes compiled now / loaded from the on-disk cache
};

// Register qubits of the specialised passes' sub-runs (their plans are built with these),
// for a state of `tiles` tiles: complex64 4 in reverse, and forward 4 below 1024 tiles
// (few CTAs per SM: straight-line code gains from twice the warps and half the code per
// gate) else 5 (the interpreter's choice); complex128 as the interpreter.
int jit_nr(int dtype, bool reverse, int64_t tiles);
// CTAs per SM the specialised kernels are compiled for (launch bounds), by CTA size.
int jit_min_blocks(int threads);

// CUDA source of the specialised kernel of pass p of the plan (rev: the reverse sweep).
std::string jit_source(const FusedPlan &plan, int p, bool rev, int dtype);
std::string jit_kernel_name(int p, bool rev);

// One compiled pass: its kernel name, source and cubin (from_cache: read from the cache).
struct JitModule {
    int p = 0;
    bool rev = false;
    std::string name, src, cubin, path;
    bool from_cache = false;
};

// Host only (no GPU): generate and compile every tile pass of the forward sweep (and the
// reverse sweep with want_rev), reading and filling the on-disk cache; secs = wall time
// of the compilations.
bool jit_compile(const FusedPlan &plan, int dtype, bool want_rev, std::vector<JitModule> &mods, double &secs,
                 std::string &err);

// Compile (or load from the cache) every tile pass of the plan's forward sweep and, with
// want_rev, of its reverse sweep, and load them on the current device.  The cache holds
// one cubin per distinct source in the directory named by GBVQC_JIT_CACHE (default
// $HOME/.cache/gbvqc/jit; "off" disables it).  Returns false with a message in err.
bool jit_build(const FusedPlan &plan, int dtype, bool want_rev, JitPlan &out, std::string &err);
void jit_free(JitPlan &jp);

// Launch a specialised pass: 2^(n-t) tiles of 2^(t-NR) threads with smem bytes of dynamic
// shared memory, the same arguments as the interpreter's kernel.  dry: a code-prefetch
// launch with args.dry = 1 and one CTA per sub-run of the pass (tiles = its sub-run
// count): CTA s runs tile 0 through sub-run s's code only, pulling it into L2, and writes
// nothing to global memory.
cudaError_t jit_launch(const JitPass &jp, void *phi, void *psi, const FusedArgs &args, unsigned tiles, int threads,
                       size_t smem, cudaStream_t s, bool dry = false);

}  // namespace gbvqc
