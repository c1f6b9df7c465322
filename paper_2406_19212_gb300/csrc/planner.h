// Host planner of the fused tile engine: partitions a physical gate list into tile
// passes and register sub-runs, and numbers the gradient slots of the reverse sweep.
#pragma once

#include <string>
#include <vector>

#include "common.cuh"

namespace gbvqc {

// One physical gate as the planner sees it.
struct PGate {
    int k;            // 1 or 2 physical qubits
    int q[2];         // physical qubits (q[0] = matrix bit 0)
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
};

struct FusedPlan {
    int t = 0, low = 0, n = 0, nr_f = 0, nr_r = 0;
    std::vector<PassDesc> fwd, rev;
    std::vector<SubRun> fsubs, rsubs;
    std::vector<FGate> fgates, rgates;
    int n_slots = 0;                // gradient slots over all passes
    std::vector<int> slot_param;    // parameter of each slot
    int max_pass_slots = 0;
};

// Build the schedule.  t = tile qubits (clamped to n), low = contiguous low qubits kept
// in every tile, nr_f / nr_r = register qubits of forward / reverse sub-runs,
// max_slots = cap on gradient slots per pass.  Returns false with a message on failure.
bool build_fused_plan(const std::vector<PGate> &gates, int n, int t, int low, int nr_f, int nr_r,
                      int max_slots, FusedPlan &out, std::string &err);

}  // namespace gbvqc
