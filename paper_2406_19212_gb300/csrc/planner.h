// Host planner of the fused tile engine: partitions a physical gate list into tile
// passes and register sub-runs, groups runs of diagonal gates into phase blocks, and
// numbers the gradient slots of the reverse sweep.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "common.cuh"

namespace gbvqc {

// One physical gate as the planner sees it.
struct PGate {
    int k;            // 1, 2 or 4 physical qubits (4: a two-qubit channel's superoperator)
    int q[4];         // physical qubits (q[0] = matrix bit 0)
    bool diag;        // diagonal matrix (commutes with other diagonal gates)
    int ftype;        // FType
    int rec_f;        // forward matrix record
    int rec_i;        // reverse: matrix applied to Phi (inverse)
    int rec_a;        // reverse: matrix applied to Psi (adjoint)
    int perm_f;       // FT_PERM2 source columns of the forward / reverse matrices
    int perm_r;
    int gen;          // GenType of a variational gate, GEN_NONE otherwise
    int gq;           // physical qubit of the generator
    float coef;       // gradient weight
    int param;        // parameter index or -1
    bool cz = false;  // exactly diag(1, 1, 1, -1) in every direction (CZ)
    bool rdiag = false;  // FT_DENSE1 whose matrices (every direction) have an exactly real diagonal
    bool rot = false;    // FT_REAL1 whose matrices are rotations [[c, -s], [s, c]] (Ry)
};

struct PlanOptions {
    int t = 12;            // tile qubits (clamped to n)
    int low = 4;           // contiguous low qubits kept in every tile
    int nr_f = 5, nr_r = 4;  // register qubits of forward / reverse sub-runs
    int max_slots = 128;   // gradient slots per pass
    int elem_bytes = 4;    // real element size (4: complex64, 8: complex128)
    int gate_smem = 24 * 1024;  // shared-memory budget of a pass's gate data
    bool phase_tables = false;  // table-mode phase blocks (needs the per-step matrix image)
    bool rot_shears = false;    // rotations as SH_ROT1 layer entries (gradient plans: a
                                // global sign per gate is allowed)
};

struct FusedPlan {
    int t = 0, low = 0, n = 0, nr_f = 0, nr_r = 0;
    std::vector<PassDesc> fwd, rev;
    std::vector<SubRun> fsubs, rsubs;
    std::vector<FGate> fgates, rgates;
    std::vector<DEnt> fents, rents;
    std::vector<MatUnit> funits, runits;
    // register phase tables of table-mode blocks (computed per step into the images)
    std::vector<TabDesc> ftabs, rtabs;
    std::vector<TabEnt> ftabents, rtabents;
    int n_slots = 0;                // gradient slots over all passes
    std::vector<int> slot_param;    // parameter of each slot
    int max_pass_slots = 0;
    // algorithmic flops per amplitude of every pass (forward / reverse)
    std::vector<double> fwd_flops, rev_flops;
    // passes that are one four-qubit gate (a two-qubit channel), run by the per-gate
    // kernel between the tile passes: index into barrier_gates, -1 for a tile pass
    std::vector<int> barrier;
    std::vector<PGate> barrier_gates;
};

bool build_fused_plan(const std::vector<PGate> &gates, int n, const PlanOptions &opt, FusedPlan &out,
                      std::string &err);

// The tile qubit set and the gates of one pass, from the greedy pass selection; a
// four-qubit gate is a pass of its own (barrier >= 0: its gate index).
struct PassSel {
    uint64_t S = 0;
    std::vector<int> gates;
    int barrier = -1;
};
bool select_passes(const std::vector<PGate> &gates, int n, int t, int low, const PlanOptions &opt,
                   std::vector<PassSel> &passes, std::string &err);
// Number of passes build_fused_plan would make (-1 if it cannot plan).
int count_passes(const std::vector<PGate> &gates, int n, const PlanOptions &opt);

// Shared-memory bytes the fused kernel needs for pass p of `plan`.
size_t pass_smem_bytes(const FusedPlan &plan, const PassDesc &d, bool reverse, int elem_bytes);

}  // namespace gbvqc
