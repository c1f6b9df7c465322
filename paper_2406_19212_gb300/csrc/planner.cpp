// Host planner of the fused tile engine.
//
// Passes: walk the circuit in order and greedily absorb every gate that (a) does not
// touch a qubit blocked by an earlier rejected gate and (b) fits in the tile set S of t
// qubits (the lowest `low` qubits are always in S).  Diagonal gates never need to be in
// S: their phase depends on bits every thread knows.  A rejected gate blocks its qubits
// for the rest of the pass, which keeps every gate after all gates it does not commute
// with (the light-cone rule of gate fusion).  A pass also closes when its gate data
// would overflow the kernel's shared-memory budget or its gradient slots the cap.
//
// Sub-runs: inside a pass, repeatedly pick up to NR tile positions and take, in circuit
// order, every ready gate whose non-diagonal qubits fit in those positions; a gate is
// ready when every earlier gate of the pass sharing a qubit with it is done (two
// diagonal gates commute and do not order each other).  The sub-run's gates are then
// re-ordered so that diagonal gates form maximal runs (non-diagonal gates first while
// they are ready), and every run of diagonal gates (even a single one) becomes one
// phase block.  The NR
// register positions are padded to avoid shared-memory bank conflicts.
#include "planner.h"

#include <algorithm>
#include <cstdint>
#include <map>

namespace gbvqc {

namespace {

inline uint64_t qmask(const PGate &g)
{
    uint64_t m = 0;
    for (int u = 0; u < g.k; u++) m |= uint64_t(1) << g.q[u];
    return m;
}

inline bool conflicts(const PGate &x, const PGate &y)
{
    return (qmask(x) & qmask(y)) && !(x.diag && y.diag);
}

double ftype_flops(int ft)
{
    switch (ft) {
    case FT_DENSE1: return 14;
    case FT_DENSE2: return 30;
    case FT_CTRL2: return 7;
    case FT_BLOCK2: return 10;   // FT_REAL1 / FT_IMAG1 / FT_ANTI1 / FT_DIAG* / FT_RPAR2: 6
    case FT_PAR2: return 14;     // a dense 2x2 on every amplitude pair
    case FT_PROBE2: return 34;   // K Phi (dense 4x4: 30) and Re conj(Psi) . K Phi (4)
    default: return 6;
    }
}

// Shared-memory wavefronts of one warp's register gather for register positions R
// (bitmask) in a tile of t positions; elements of elem_bytes * 2 bytes, XOR swizzle of
// the kernel (bits [SB, 2SB) folded onto [0, SB)).
int gather_wavefronts(uint32_t Rmask, int t, int NR, int elem_bytes)
{
    const int SB = elem_bytes == 4 ? 4 : 3;        // 16 x 8 B or 8 x 16 B slots
    const int group = elem_bytes == 4 ? 16 : 8;     // lanes served per wavefront
    int pos[32], np = 0;
    for (int p = 0; p < t && np < 32; p++)
        if (!((Rmask >> p) & 1)) pos[np++] = p;
    const int lanes = std::min(32, 1 << std::max(0, t - NR));
    int total = 0;
    for (int g0 = 0; g0 < lanes; g0 += group) {
        int count[16] = {0}, worst = 0;
        for (int L = g0; L < std::min(lanes, g0 + group); L++) {
            int l = 0;
            for (int i = 0; i < 5 && i < np; i++)
                if ((L >> i) & 1) l |= 1 << pos[i];
            int swz = l ^ ((l >> SB) & ((1 << SB) - 1));
            int slot = swz & ((1 << SB) - 1);
            worst = std::max(worst, ++count[slot]);
        }
        total += worst;
    }
    return total;
}

struct Emitter {
    const std::vector<PGate> &G;
    const int *local_of;
    int t, NR, elem_bytes;
    bool reverse;
    int &slot_counter;
    std::vector<int> &slot_param;
    std::vector<SubRun> &subs;
    std::vector<FGate> &gates;
    std::vector<DEnt> &ents;
    std::vector<MatUnit> &units;
    std::vector<TabDesc> &tabs;
    std::vector<TabEnt> &tabents;
    bool phase_tables;
    int gate_base, ent_base, unit_base;   // pass-local indices start here
    std::map<int, int> unit_of_rec;
    double flops = 0;
    int n_blocks = 0;        // FT_DIAGB gates emitted in this pass
    bool has_2q = false;     // a non-diagonal two-qubit gate was emitted
    bool overflow = false;   // a phase block class with more than 255 entries

    // a unit of its own (no sharing): layers take runs of consecutive units
    int fresh_unit(int rec, int part = 0)
    {
        units.push_back(MatUnit{rec, part});
        return (int)units.size() - 1 - unit_base;
    }

    // the shear parameters of a rotation record (shared)
    std::map<int, int> shear_of_rec;
    int shear_unit(int rec)
    {
        auto it = shear_of_rec.find(rec);
        if (it != shear_of_rec.end()) return it->second;
        units.push_back(MatUnit{rec, kUnitShear});
        return shear_of_rec[rec] = (int)units.size() - 1 - unit_base;
    }
    bool rot_shears = false;  // PlanOptions::rot_shears

    // a register phase table over 2^NR indices from the given entries: reserves its units
    // (placeholders the gather skips) and returns the first, pass-local
    int table(const std::vector<TabEnt> &te)
    {
        const int n_units = std::max(1, (1 << NR) * 2 / 8);
        const int first = (int)units.size();
        for (int i = 0; i < n_units; i++) units.push_back(MatUnit{-1, 0});
        tabs.push_back(TabDesc{8 * first, NR, (int)tabents.size(), (int)te.size()});
        tabents.insert(tabents.end(), te.begin(), te.end());
        return first - unit_base;
    }

    int unit(int rec, int k)
    {
        auto it = unit_of_rec.find(rec);
        if (it != unit_of_rec.end()) return it->second;
        int u = (int)units.size() - unit_base;
        for (int part = 0; part < (k == 2 ? 4 : 1); part++) units.push_back(MatUnit{rec, part});
        unit_of_rec[rec] = u;
        return u;
    }
};

void build_subruns(const std::vector<int> &order, Emitter &E)
{
    const std::vector<PGate> &G = E.G;
    const int NR = E.NR, t = E.t;
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
        // 1. select the sub-run's gates
        int R[8], nR = 0;
        uint32_t Rmask = 0;
        std::vector<int> sel;
        for (int pos = 0; pos < m; pos++) {
            if (done[pos] || !ready(pos)) continue;
            const PGate &g = G[order[pos]];
            if (!g.diag) {
                int need[2], nn = 0;
                for (int u = 0; u < g.k; u++) {
                    int l = E.local_of[g.q[u]];
                    if (!((Rmask >> l) & 1)) need[nn++] = l;
                }
                if (nR + nn > NR) continue;
                for (int u = 0; u < nn; u++) {
                    R[nR++] = need[u];
                    Rmask |= 1u << need[u];
                }
            }
            sel.push_back(pos);
            done[pos] = 1;
            ndone++;
            for (int u = 0; u < g.k; u++) {
                int q = g.q[u];
                while (head[q] < (int)lists[q].size() && done[lists[q][head[q]]]) head[q]++;
            }
        }
        // 2. pad the register positions, fewest bank conflicts first
        {
            std::vector<int> cand;
            for (int p = 0; p < t; p++)
                if (!((Rmask >> p) & 1)) cand.push_back(p);
            int need = NR - nR;
            uint32_t best = 0;
            int best_score = 1 << 30;
            // exhaustive over combinations when small, else greedy
            std::vector<int> idx(need);
            long combos = 1;
            for (int i = 0; i < need; i++) combos = combos * (long)(cand.size() - i) / (i + 1);
            if (need > 0 && combos <= 400) {
                for (int i = 0; i < need; i++) idx[i] = i;
                while (true) {
                    uint32_t msk = Rmask;
                    for (int i = 0; i < need; i++) msk |= 1u << cand[idx[i]];
                    int sc = gather_wavefronts(msk, t, NR, E.elem_bytes);
                    if (sc < best_score) { best_score = sc; best = msk; }
                    int i = need - 1;
                    while (i >= 0 && idx[i] == (int)cand.size() - need + i) i--;
                    if (i < 0) break;
                    idx[i]++;
                    for (int k2 = i + 1; k2 < need; k2++) idx[k2] = idx[k2 - 1] + 1;
                }
            } else if (need > 0) {
                best = Rmask;
                for (int i = 0; i < need; i++) {
                    int bp = -1, bs = 1 << 30;
                    for (int p : cand)
                        if (!((best >> p) & 1)) {
                            int sc = gather_wavefronts(best | (1u << p), t, NR, E.elem_bytes);
                            if (sc < bs) { bs = sc; bp = p; }
                        }
                    best |= 1u << bp;
                }
            } else {
                best = Rmask;
            }
            for (int p = 0; p < t && nR < NR; p++)
                if (((best >> p) & 1) && !((Rmask >> p) & 1)) {
                    R[nR++] = p;
                    Rmask |= 1u << p;
                }
        }
        auto slot_of = [&](int l) {
            for (int k = 0; k < NR; k++)
                if (R[k] == l) return k;
            return -1;
        };
        auto code_of = [&](int q) {
            int l = E.local_of[q];
            if (l < 0) return -1 - q;
            int k = slot_of(l);
            return k >= 0 ? k : NR + l;
        };
        // 3. order: ready non-diagonal gates first, then the ready diagonal run
        std::vector<std::vector<int>> runs;   // each run: gate positions; diagonal runs flagged
        std::vector<char> run_diag;
        {
            std::vector<char> emitted(sel.size(), 0);
            size_t left = sel.size();
            auto is_ready = [&](size_t i) {
                for (size_t j = 0; j < i; j++)
                    if (!emitted[j] && conflicts(G[order[sel[j]]], G[order[sel[i]]])) return false;
                return true;
            };
            while (left > 0) {
                bool progress = true;
                std::vector<int> nd;
                while (progress) {
                    progress = false;
                    for (size_t i = 0; i < sel.size(); i++)
                        if (!emitted[i] && !G[order[sel[i]]].diag && is_ready(i)) {
                            emitted[i] = 1;
                            left--;
                            nd.push_back(sel[i]);
                            progress = true;
                        }
                }
                if (!nd.empty()) {
                    runs.push_back(nd);
                    run_diag.push_back(0);
                }
                std::vector<int> dg;
                for (size_t i = 0; i < sel.size(); i++)
                    if (!emitted[i] && G[order[sel[i]]].diag && is_ready(i)) dg.push_back((int)i);
                for (int i : dg) emitted[i] = 1;
                left -= dg.size();
                if (!dg.empty()) {
                    std::vector<int> run;
                    for (int i : dg) run.push_back(sel[i]);
                    runs.push_back(run);
                    run_diag.push_back(1);
                }
            }
        }
        // 4. emit
        SubRun sr{};
        for (int k = 0; k < 8; k++) sr.R[k] = (int8_t)(k < NR ? R[k] : 0);
        sr.g_begin = (int)E.gates.size() - E.gate_base;
        const double st = E.reverse ? 2.0 : 1.0;
        for (size_t r = 0; r < runs.size(); r++) {
            if (!run_diag[r]) {
                // one-qubit gates on distinct register slots are grouped into layers (they
                // commute; in the reverse sweep each generator may be read before or after
                // the other gates of its layer)
                std::vector<int> layer;
                auto flush_layer = [&]() {
                    if (layer.empty()) return;
                    std::sort(layer.begin(), layer.end(), [&](int x, int y) {
                        return slot_of(E.local_of[G[order[x]].q[0]]) < slot_of(E.local_of[G[order[y]].q[0]]);
                    });
                    // record: a = slot mask, b = entries, perm = per slot K the shape code
                    // (bits 2K: 0 dense, 1 real, 2 imaginary off-diagonal, 3 anti-diagonal);
                    // forward: mat = first of the entries' consecutive units (slot order)
                    FGate f{};
                    f.type = FT_LAYER1;
                    f.slot = -1;
                    f.ent = (int16_t)((int)E.ents.size() - E.ent_base);
                    int first = -1;
                    auto shear = [&](const PGate &g) { return E.rot_shears && g.rot && g.ftype == FT_REAL1; };
                    if (!E.reverse)
                        for (int pos : layer) {
                            const PGate &g = G[order[pos]];
                            const int u = E.fresh_unit(g.rec_f, shear(g) ? kUnitShear : 0);
                            if (first < 0) first = u;
                        }
                    f.mat = f.mat2 = (int16_t)first;
                    int mask = 0, codes = 0, i_ent = 0;
                    for (int pos : layer) {
                        const PGate &g = G[order[pos]];
                        DEnt d{};
                        const int k = slot_of(E.local_of[g.q[0]]);
                        mask |= 1 << k;
                        d.k = (int8_t)(shear(g)              ? SH_ROT1
                                       : g.ftype == FT_REAL1 ? SH_REAL1
                                       : g.ftype == FT_ANTI1 ? SH_ANTI1
                                       : g.ftype == FT_IMAG1 ? SH_IMAG1
                                       : g.rdiag             ? SH_RDIAG1
                                                             : SH_DENSE1);
                        codes |= (shear(g)               ? 4
                                  : g.ftype == FT_REAL1 ? 1
                                  : g.ftype == FT_IMAG1 ? 2
                                  : g.ftype == FT_ANTI1 ? 3
                                                        : 0) << (3 * k);
                        d.ca = (int8_t)k;
                        if (E.reverse && shear(g)) {
                            d.mat = (int16_t)E.shear_unit(g.rec_i);
                            d.mat2 = (int16_t)E.shear_unit(g.rec_a);
                        } else {
                            d.mat = (int16_t)(E.reverse ? E.unit(g.rec_i, 1) : first + i_ent);
                            d.mat2 = (int16_t)(E.reverse ? E.unit(g.rec_a, 1) : d.mat);
                        }
                        i_ent++;
                        d.cls = GEN_NONE;
                        d.slot = -1;
                        E.flops += st * ftype_flops(g.ftype);
                        if (E.reverse && g.gen != GEN_NONE) {
                            d.cls = (int8_t)g.gen;
                            d.coef = g.coef;
                            d.slot = E.slot_counter++;
                            E.slot_param.push_back(g.param);
                            E.flops += 4;
                        }
                        E.ents.push_back(d);
                    }
                    f.a = (int8_t)mask;
                    f.b = (int8_t)layer.size();
                    f.perm = codes;
                    f.n_ent = (int16_t)layer.size();
                    E.gates.push_back(f);
                    layer.clear();
                };
                for (int pos : runs[r]) {
                    const PGate &g = G[order[pos]];
                    if (g.k == 1) {
                        const int k = slot_of(E.local_of[g.q[0]]);
                        bool clash = false;
                        for (int x : layer) clash = clash || slot_of(E.local_of[G[order[x]].q[0]]) == k;
                        if (clash) flush_layer();
                        layer.push_back(pos);
                        continue;
                    }
                    flush_layer();
                    if (g.ftype == FT_PROBE2 && !E.reverse) continue;  // gradient reads only
                    if (g.k == 2) E.has_2q = true;
                    FGate f{};
                    f.type = (int8_t)g.ftype;
                    f.a = (int8_t)slot_of(E.local_of[g.q[0]]);
                    f.b = (int8_t)(g.k == 2 ? slot_of(E.local_of[g.q[1]]) : 0);
                    f.mat = (int16_t)E.unit(E.reverse ? g.rec_i : g.rec_f, g.k);
                    f.mat2 = (int16_t)(E.reverse ? E.unit(g.rec_a, g.k) : f.mat);
                    f.perm = E.reverse ? g.perm_r : g.perm_f;
                    f.slot = -1;
                    E.flops += st * ftype_flops(g.ftype);
                    if (E.reverse && g.gen != GEN_NONE) {
                        f.gen = (int8_t)g.gen;
                        f.gpos = (int8_t)slot_of(E.local_of[g.gq]);
                        f.coef = g.coef;
                        f.slot = E.slot_counter++;
                        E.slot_param.push_back(g.param);
                        E.flops += 4;
                    }
                    E.gates.push_back(f);
                }
                flush_layer();
                continue;
            }
            const std::vector<int> &run = runs[r];
            int nz = 0;
            for (int pos : run) nz += (E.reverse && G[order[pos]].gen == GEN_Z) ? 1 : 0;
            FGate f{};
            f.type = FT_DIAGB;
            f.slot = E.n_blocks++;
            f.nz = (int8_t)nz;
            f.ent = (int16_t)((int)E.ents.size() - E.ent_base);
            if (nz) E.flops += 2 + NR;
            for (int pos : run) {   // Z generators first: all read the states after the block
                const PGate &g = G[order[pos]];
                if (!(E.reverse && g.gen == GEN_Z)) continue;
                DEnt d{};
                d.k = 3;
                d.cls = DC_Z;
                d.ca = (int8_t)code_of(g.gq);
                d.slot = E.slot_counter++;
                d.coef = g.coef;
                E.slot_param.push_back(g.param);
                E.ents.push_back(d);
            }
            // table mode: every mixed entry (one register position, one constant) is a CZ
            bool table = E.phase_tables;
            if (table)
                for (int pos : run) {
                    const PGate &g = G[order[pos]];
                    if (g.k != 2) continue;
                    const int ca = code_of(g.q[0]), cb = code_of(g.q[1]);
                    const bool ra = ca >= 0 && ca < NR, rb = cb >= 0 && cb < NR;
                    if (ra != rb && !g.cz) table = false;
                }
            if (table) {
                std::vector<DEnt> tl[2];           // TILE, LOCAL entries
                std::vector<DEnt> mixcz;
                std::vector<TabEnt> tphi, tpsi;   // register entries: Phi (forward: U), Psi
                bool separate = false;
                for (int pos : run) {
                    const PGate &g = G[order[pos]];
                    const int rf = E.reverse ? g.rec_i : g.rec_f, ra_ = E.reverse ? g.rec_a : g.rec_f;
                    DEnt d{};
                    d.k = (int8_t)g.k;
                    d.ca = (int8_t)code_of(g.q[0]);
                    d.cb = (int8_t)(g.k == 2 ? code_of(g.q[1]) : 0);
                    d.slot = -1;
                    const bool ra = d.ca >= 0 && d.ca < NR, rb = g.k == 2 && d.cb >= 0 && d.cb < NR;
                    if (ra || rb) {
                        if (g.k == 2 && ra != rb) {   // mixed CZ: no matrix
                            d.cls = DC_REG;
                            d.mat = d.mat2 = -1;
                            mixcz.push_back(d);
                            continue;
                        }
                        tphi.push_back(TabEnt{rf, (int8_t)g.k, d.ca, d.cb, 0});
                        tpsi.push_back(TabEnt{ra_, (int8_t)g.k, d.ca, d.cb, 0});
                        if (ra_ != rf) separate = true;
                        continue;
                    }
                    d.mat = (int16_t)E.unit(rf, g.k);
                    d.mat2 = (int16_t)E.unit(ra_, g.k);
                    if (d.mat2 != d.mat) separate = true;
                    const bool tile = d.ca < 0 && (g.k == 1 || d.cb < 0);
                    d.cls = tile ? DC_TILE : DC_LOCAL;
                    tl[tile ? 0 : 1].push_back(d);
                }
                for (const DEnt &d : tl[0]) E.ents.push_back(d);
                for (const DEnt &d : tl[1]) E.ents.push_back(d);
                for (const DEnt &d : mixcz) E.ents.push_back(d);
                if (tl[0].size() > 255 || tl[1].size() > 255 || mixcz.size() > 255) E.overflow = true;
                f.perm = (int)tl[0].size() | ((int)tl[1].size() << 8) | ((int)mixcz.size() << 16);
                f.mat = (int16_t)E.table(tphi);
                f.mat2 = separate ? (int16_t)E.table(tpsi) : f.mat;
                f.flags = (int8_t)((separate ? FLAG_SEPARATE : 0) | FLAG_TABLE);
                f.n_ent = (int16_t)((int)E.ents.size() - E.ent_base - f.ent);
                // one complex product per amplitude and state
                E.flops += (separate ? 2.0 : 1.0) * 6 + st * 6;
                E.gates.push_back(f);
                continue;
            }
            // phase entries, grouped by class
            std::vector<DEnt> cls_ents[6];
            bool separate = false;
            for (int pos : run) {
                const PGate &g = G[order[pos]];
                DEnt d{};
                d.k = (int8_t)g.k;
                d.ca = (int8_t)code_of(g.q[0]);
                d.cb = (int8_t)(g.k == 2 ? code_of(g.q[1]) : 0);
                d.mat = (int16_t)E.unit(E.reverse ? g.rec_i : g.rec_f, g.k);
                d.mat2 = (int16_t)(E.reverse ? E.unit(g.rec_a, g.k) : d.mat);
                d.slot = -1;
                if (d.mat2 != d.mat) separate = true;
                auto reg = [&](int c) { return c >= 0 && c < NR; };
                auto tile = [&](int c) { return c < 0; };
                if (g.k == 1) {
                    d.cls = reg(d.ca) ? DC_REG : tile(d.ca) ? DC_TILE : DC_LOCAL;
                } else if (reg(d.ca) && reg(d.cb)) {
                    d.cls = g.cz ? DC_PAIR_CZ : DC_PAIR;
                } else if (reg(d.ca) || reg(d.cb)) {
                    d.cls = DC_REG;
                } else {
                    d.cls = (tile(d.ca) && tile(d.cb)) ? DC_TILE : DC_LOCAL;
                }
                cls_ents[(int)d.cls].push_back(d);
            }
            int cnt[6];
            for (int c = 1; c < 6; c++) {
                cnt[c] = (int)cls_ents[c].size();
                for (const DEnt &d : cls_ents[c]) E.ents.push_back(d);
            }
            const int np = cnt[DC_PAIR] + cnt[DC_PAIR_CZ];
            if (cnt[DC_TILE] > 255 || cnt[DC_LOCAL] > 255 || cnt[DC_REG] > 255 || np > 255) {
                E.overflow = true;
            }
            f.perm = cnt[DC_TILE] | (cnt[DC_LOCAL] << 8) | (cnt[DC_REG] << 16) | (np << 24);
            f.flags = separate ? FLAG_SEPARATE : 0;
            f.n_ent = (int16_t)((int)E.ents.size() - E.ent_base - f.ent);
            // per thread: the block's local factors, register pairs, two half tables and one
            // product per amplitude and state; PAIR entries add a controlled phase on a quarter
            E.flops += (separate ? 2.0 : 1.0) * (6 + 6.0 * cnt[DC_PAIR] * 0.25 + 1.5 * cnt[DC_PAIR_CZ] * 0.25) + st * 6;
            E.gates.push_back(f);
        }
        sr.g_end = (int)E.gates.size() - E.gate_base;
        E.subs.push_back(sr);
    }
}

int gate_weight(const PGate &g, int elem_bytes)
{
    int units = g.k == 2 ? 4 : 1;
    return (int)sizeof(FGate) + (g.diag ? (int)sizeof(DEnt) : 0) + 2 * units * 8 * elem_bytes;
}

}  // namespace

size_t pass_smem_bytes(const FusedPlan &plan, const PassDesc &d, bool reverse, int elem_bytes)
{
    const int nr = reverse ? plan.nr_r : plan.nr_f;
    const int threads = 1 << (d.t - nr);
    const int nwarps = (threads + 31) / 32;
    auto al = [](size_t x) { return (x + 15) & ~size_t(15); };
    size_t b = al((reverse ? 2 : 1) * (size_t(1) << d.t) * 2 * elem_bytes);
    b += al(sizeof(int64_t) * (size_t(1) << (d.t - d.low)));
    if (reverse) b += al((size_t)elem_bytes * d.n_slots * nwarps);  // per-warp partials
    b += al(sizeof(FGate) * (size_t)d.n_gates);
    b += al(sizeof(DEnt) * (size_t)d.n_ent);
    b += al((size_t)4 * elem_bytes * d.n_blocks);   // tile-constant products (Phi, Psi)
    b += al((size_t)8 * elem_bytes * d.n_units);
    return b;
}

// Greedy pass selection: scan the remaining gates in circuit order; a gate joins the pass
// if every earlier remaining gate on its qubits joined (no qubit of it is blocked), its
// non-diagonal qubits fit in the t tile qubits (the `low` lowest physical qubits are
// always in the tile), and the pass's slot and shared-memory budgets allow it.  A ready
// four-qubit gate met by an empty pass becomes a pass of its own; met later, it blocks.
bool select_passes(const std::vector<PGate> &G, int n, int t, int low, const PlanOptions &opt,
                   std::vector<PassSel> &passes, std::string &err)
{
    const int m = (int)G.size();
    std::vector<char> applied(m, 0);
    int done = 0;
    const uint64_t lowmask = (uint64_t(1) << low) - 1;
    passes.clear();
    while (done < m) {
        PassSel pb;
        pb.S = lowmask;
        int cnt = low, slots = 0, bytes = 0;
        uint64_t blocked = 0;
        for (int i = 0; i < m; i++) {
            if (applied[i]) continue;
            const PGate &g = G[i];
            const uint64_t qm = qmask(g);
            if (qm & blocked) {
                blocked |= qm;
                continue;
            }
            if (g.k == 4) {
                if (pb.gates.empty()) {
                    pb.barrier = i;
                    pb.gates.push_back(i);
                    break;
                }
                blocked |= qm;
                continue;
            }
            const int w = gate_weight(g, opt.elem_bytes);
            if ((g.gen != GEN_NONE && slots >= opt.max_slots) || (bytes + w > opt.gate_smem && !pb.gates.empty())) {
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
            bytes += w;
            if (g.gen != GEN_NONE) slots++;
        }
        if (pb.gates.empty()) {
            err = "planner made no progress";
            return false;
        }
        for (int i : pb.gates) applied[i] = 1;
        done += (int)pb.gates.size();
        if (pb.barrier >= 0) {
            passes.push_back(std::move(pb));
            continue;
        }
        for (int q = 0; q < n && cnt < t; q++)
            if (!((pb.S >> q) & 1)) {
                pb.S |= uint64_t(1) << q;
                cnt++;
            }
        passes.push_back(std::move(pb));
    }
    return true;
}

int count_passes(const std::vector<PGate> &G, int n, const PlanOptions &opt)
{
    const int t = std::min(opt.t, n);
    const int low = std::max(1, std::min(opt.low, t));
    std::vector<PassSel> passes;
    std::string err;
    if (!select_passes(G, n, t, low, opt, passes, err)) return -1;
    return (int)passes.size();
}

bool build_fused_plan(const std::vector<PGate> &G, int n, const PlanOptions &opt, FusedPlan &out,
                      std::string &err)
{
    int t = std::min(opt.t, n);
    const int nr = std::max(opt.nr_f, opt.nr_r);
    if (t < nr || t > 16) {
        err = "tile of " + std::to_string(t) + " qubits cannot hold " + std::to_string(nr) +
              " register qubits";
        return false;
    }
    int low = std::max(1, std::min(opt.low, t));
    out = FusedPlan();
    out.t = t;
    out.low = low;
    out.n = n;
    out.nr_f = opt.nr_f;
    out.nr_r = opt.nr_r;
    std::vector<PassSel> passes;
    if (!select_passes(G, n, t, low, opt, passes, err)) return false;

    int slot_counter = 0;
    std::vector<int> dummy_params;
    int dummy_counter = 0;
    const size_t P = passes.size();
    out.fwd.resize(P);
    out.rev.resize(P);
    out.fwd_flops.assign(P, 0.0);
    out.rev_flops.assign(P, 0.0);
    out.barrier.assign(P, -1);
    for (size_t p = 0; p < P; p++)
        if (passes[p].barrier >= 0) {
            out.barrier[p] = (int)out.barrier_gates.size();
            out.barrier_gates.push_back(G[passes[p].barrier]);
        }
    std::vector<std::vector<int>> local_of(P, std::vector<int>(64, -1));
    for (size_t p = 0; p < P; p++) {
        PassDesc d{};
        d.t = t;
        d.n = n;
        d.low = low;
        int li = 0, ni = 0;
        for (int q = 0; q < n; q++) {
            if ((passes[p].S >> q) & 1) {
                d.S[li] = (int8_t)q;
                local_of[p][q] = li++;
            } else {
                d.NS[ni++] = (int8_t)q;
            }
        }
        out.fwd[p] = d;
        out.rev[p] = d;
    }
    for (int dir = 0; dir < 2; dir++) {
        const bool rev = dir == 1;
        for (size_t pi = 0; pi < P; pi++) {
            const size_t p = rev ? P - 1 - pi : pi;   // reverse passes in launch order
            PassDesc &d = rev ? out.rev[p] : out.fwd[p];
            if (passes[p].barrier >= 0) {  // not a tile pass: empty ranges, no slots
                d.slot_begin = rev ? slot_counter : 0;
                continue;
            }
            std::vector<int> order = passes[p].gates;
            if (rev) std::reverse(order.begin(), order.end());
            Emitter E{G, local_of[p].data(), t, rev ? opt.nr_r : opt.nr_f, opt.elem_bytes, rev,
                      rev ? slot_counter : dummy_counter, rev ? out.slot_param : dummy_params,
                      rev ? out.rsubs : out.fsubs, rev ? out.rgates : out.fgates,
                      rev ? out.rents : out.fents, rev ? out.runits : out.funits,
                      rev ? out.rtabs : out.ftabs, rev ? out.rtabents : out.ftabents, opt.phase_tables,
                      0, 0, 0, {}, 0.0, 0, false, false};
            E.rot_shears = opt.rot_shears;
            E.gate_base = (int)E.gates.size();
            E.ent_base = (int)E.ents.size();
            E.unit_base = (int)E.units.size();
            d.sub_begin = (int)E.subs.size();
            d.gate_begin = E.gate_base;
            d.ent_begin = E.ent_base;
            d.unit_begin = E.unit_base;
            d.slot_begin = rev ? slot_counter : 0;
            build_subruns(order, E);
            if (E.overflow) {
                err = "phase block too large";
                return false;
            }
            d.n_blocks = E.n_blocks;
            d.has_2q = E.has_2q ? 1 : 0;
            d.n_sub = (int)E.subs.size() - d.sub_begin;
            d.n_gates = (int)E.gates.size() - d.gate_begin;
            d.n_ent = (int)E.ents.size() - d.ent_begin;
            d.n_units = (int)E.units.size() - d.unit_begin;
            d.n_slots = rev ? slot_counter - d.slot_begin : 0;
            if (d.n_gates > 32767 || d.n_ent > 32767 || d.n_units > 32767) {
                err = "pass too large";
                return false;
            }
            (rev ? out.rev_flops : out.fwd_flops)[p] = E.flops;
            if (rev) out.max_pass_slots = std::max(out.max_pass_slots, d.n_slots);
        }
    }
    out.n_slots = slot_counter;
    return true;
}

}  // namespace gbvqc
