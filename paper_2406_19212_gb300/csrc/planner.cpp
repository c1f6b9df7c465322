// Host planner of the fused tile engine.
//
// Passes: walk the circuit in order and greedily absorb every gate that (a) does not
// touch a qubit blocked by an earlier rejected gate and (b) fits in the tile set S of t
// qubits (the lowest `low` qubits are always in S).  Diagonal gates never need to be in
// S: their phase depends on bits every thread knows.  A rejected gate blocks its qubits
// for the rest of the pass, which keeps every gate after all gates it does not commute
// with (the light-cone rule of gate fusion).
//
// Sub-runs: inside a pass, repeatedly pick up to NR tile positions and take, in circuit
// order, every ready gate whose non-diagonal qubits fit in those positions; a gate is
// ready when every earlier gate of the pass sharing a qubit with it is done (two
// diagonal gates commute and do not order each other).
#include "planner.h"

#include <algorithm>
#include <cstdint>

namespace gbvqc {

namespace {

inline uint64_t qmask(const PGate &g)
{
    uint64_t m = uint64_t(1) << g.q[0];
    if (g.k == 2) m |= uint64_t(1) << g.q[1];
    return m;
}

struct PassBuild {
    uint64_t S = 0;
    std::vector<int> gates;   // gate indices in circuit order
};

// Emit the sub-runs of one pass (gate order `order`, already reversed for the reverse
// sweep) into subs / fgates.  Reverse passes also number their gradient slots.
void build_subruns(const std::vector<int> &order, const std::vector<PGate> &G, const int *local_of,
                   int t, int NR, bool reverse, int &slot_counter, std::vector<int> &slot_param,
                   std::vector<SubRun> &subs, std::vector<FGate> &fgates)
{
    const int m = (int)order.size();
    std::vector<std::vector<int>> lists(64);
    for (int pos = 0; pos < m; pos++) {
        const PGate &g = G[order[pos]];
        for (int u = 0; u < g.k; u++) lists[g.q[u]].push_back(pos);
    }
    std::vector<int> head(64, 0);
    std::vector<char> done(m, 0);
    int ndone = 0;
    auto ready = [&](int pos) {
        const PGate &g = G[order[pos]];
        for (int u = 0; u < g.k; u++) {
            const std::vector<int> &L = lists[g.q[u]];
            for (int i = head[g.q[u]]; i < (int)L.size() && L[i] != pos; i++) {
                int j = L[i];
                if (!done[j] && !(G[order[j]].diag && g.diag)) return false;
            }
        }
        return true;
    };
    while (ndone < m) {
        int R[8], nR = 0;
        uint32_t Rmask = 0;
        std::vector<int> sub;
        for (int pos = 0; pos < m; pos++) {
            if (done[pos] || !ready(pos)) continue;
            const PGate &g = G[order[pos]];
            if (!g.diag) {
                int need[2], nn = 0;
                for (int u = 0; u < g.k; u++) {
                    int l = local_of[g.q[u]];
                    if (!((Rmask >> l) & 1)) need[nn++] = l;
                }
                if (nR + nn > NR) continue;
                for (int u = 0; u < nn; u++) {
                    R[nR++] = need[u];
                    Rmask |= 1u << need[u];
                }
            }
            sub.push_back(pos);
            done[pos] = 1;
            ndone++;
            for (int u = 0; u < g.k; u++) {
                int q = g.q[u];
                while (head[q] < (int)lists[q].size() && done[lists[q][head[q]]]) head[q]++;
            }
        }
        for (int p = 0; p < t && nR < NR; p++)
            if (!((Rmask >> p) & 1)) {
                R[nR++] = p;
                Rmask |= 1u << p;
            }
        auto slot_of = [&](int l) {
            for (int k = 0; k < NR; k++)
                if (R[k] == l) return k;
            return -1;
        };
        auto code_of = [&](int q) {  // position code of physical qubit q
            int l = local_of[q];
            if (l < 0) return -1 - q;
            int k = slot_of(l);
            return k >= 0 ? k : NR + l;
        };
        SubRun sr{};
        for (int k = 0; k < 8; k++) sr.R[k] = (int8_t)(k < NR ? R[k] : 0);
        sr.g_begin = (int)fgates.size();
        for (int pos : sub) {
            const PGate &g = G[order[pos]];
            FGate f{};
            f.type = g.ftype;
            if (g.diag) {
                f.a = code_of(g.q[0]);
                f.b = g.k == 2 ? code_of(g.q[1]) : 0;
            } else {
                f.a = slot_of(local_of[g.q[0]]);
                f.b = g.k == 2 ? slot_of(local_of[g.q[1]]) : 0;
            }
            f.rec = reverse ? g.rec_i : g.rec_f;
            f.rec2 = reverse ? g.rec_a : -1;
            f.perm = reverse ? g.perm_r : g.perm_f;
            f.gen = GEN_NONE;
            f.slot = -1;
            if (reverse && g.gen != GEN_NONE) {
                f.gen = g.gen;
                f.gpos = g.gen == GEN_Z ? code_of(g.gq) : slot_of(local_of[g.gq]);
                f.coef = g.coef;
                f.slot = slot_counter++;
                slot_param.push_back(g.param);
            }
            fgates.push_back(f);
        }
        sr.g_end = (int)fgates.size();
        subs.push_back(sr);
    }
}

}  // namespace

bool build_fused_plan(const std::vector<PGate> &G, int n, int t, int low, int nr_f, int nr_r,
                      int max_slots, FusedPlan &out, std::string &err)
{
    if (t > n) t = n;
    int nr = std::max(nr_f, nr_r);
    if (t < nr || t > 16) {
        err = "tile of " + std::to_string(t) + " qubits cannot hold " + std::to_string(nr) +
              " register qubits";
        return false;
    }
    if (low < 1) low = 1;
    if (low > t) low = t;
    out = FusedPlan();
    out.t = t;
    out.low = low;
    out.n = n;
    out.nr_f = nr_f;
    out.nr_r = nr_r;
    const int m = (int)G.size();
    std::vector<char> applied(m, 0);
    std::vector<PassBuild> passes;
    int done = 0;
    const uint64_t lowmask = (uint64_t(1) << low) - 1;
    while (done < m) {
        PassBuild pb;
        pb.S = lowmask;
        int cnt = low, slots = 0;
        uint64_t blocked = 0;
        for (int i = 0; i < m; i++) {
            if (applied[i]) continue;
            const PGate &g = G[i];
            const uint64_t qm = qmask(g);
            if (qm & blocked) {
                blocked |= qm;
                continue;
            }
            if (g.gen != GEN_NONE && slots >= max_slots) {
                blocked |= qm;
                continue;
            }
            if (!g.diag) {
                uint64_t need = qm & ~pb.S;
                int c = __builtin_popcountll(need);
                if (cnt + c > t) {
                    blocked |= qm;
                    continue;
                }
                pb.S |= need;
                cnt += c;
            }
            pb.gates.push_back(i);
            if (g.gen != GEN_NONE) slots++;
        }
        if (pb.gates.empty()) {
            err = "planner made no progress";
            return false;
        }
        for (int i : pb.gates) applied[i] = 1;
        done += (int)pb.gates.size();
        for (int q = 0; q < n && cnt < t; q++)
            if (!((pb.S >> q) & 1)) {
                pb.S |= uint64_t(1) << q;
                cnt++;
            }
        passes.push_back(pb);
    }

    int slot_counter = 0;
    out.fwd.resize(passes.size());
    out.rev.resize(passes.size());
    std::vector<std::vector<int>> local_of_pass(passes.size(), std::vector<int>(64, -1));
    for (size_t p = 0; p < passes.size(); p++) {
        PassDesc d{};
        d.t = t;
        d.n = n;
        d.low = low;
        int li = 0, ni = 0;
        for (int q = 0; q < n; q++) {
            if ((passes[p].S >> q) & 1) {
                d.S[li] = (int8_t)q;
                local_of_pass[p][q] = li++;
            } else {
                d.NS[ni++] = (int8_t)q;
            }
        }
        out.fwd[p] = d;
        out.rev[p] = d;
    }
    // forward sub-runs, pass order
    for (size_t p = 0; p < passes.size(); p++) {
        int dummy = 0;
        std::vector<int> dummy_params;
        out.fwd[p].sub_begin = (int)out.fsubs.size();
        build_subruns(passes[p].gates, G, local_of_pass[p].data(), t, nr_f, false, dummy, dummy_params,
                      out.fsubs, out.fgates);
        out.fwd[p].n_sub = (int)out.fsubs.size() - out.fwd[p].sub_begin;
    }
    // reverse sub-runs: passes and gates in reverse order; slots numbered in launch order
    for (size_t pr = 0; pr < passes.size(); pr++) {
        size_t p = passes.size() - 1 - pr;
        std::vector<int> order(passes[p].gates.rbegin(), passes[p].gates.rend());
        PassDesc &d = out.rev[p];
        d.sub_begin = (int)out.rsubs.size();
        d.slot_begin = slot_counter;
        build_subruns(order, G, local_of_pass[p].data(), t, nr_r, true, slot_counter, out.slot_param,
                      out.rsubs, out.rgates);
        d.n_sub = (int)out.rsubs.size() - d.sub_begin;
        d.n_slots = slot_counter - d.slot_begin;
        out.max_pass_slots = std::max(out.max_pass_slots, d.n_slots);
    }
    out.n_slots = slot_counter;
    return true;
}

}  // namespace gbvqc
