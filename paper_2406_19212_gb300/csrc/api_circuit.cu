// C ABI: circuits (Sec. II.C): matrix records, the per-gate schedule, the fused tile
// schedule and its device copies, tiling options and plan queries.
#include "api_internal.h"

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
    dev_free(p->d_fwd); dev_free(p->d_rev); dev_free(p->d_fsubs); dev_free(p->d_rsubs);
    dev_free(p->d_fgates); dev_free(p->d_rgates); dev_free(p->d_fents); dev_free(p->d_rents);
    dev_free(p->d_funits); dev_free(p->d_runits); dev_free(p->d_csr_ptr); dev_free(p->d_csr_slots);
    dev_free(p->d_fimg); dev_free(p->d_rimg);
    dev_free(p->d_ftabs); dev_free(p->d_rtabs); dev_free(p->d_ftabents); dev_free(p->d_rtabents);
    if (p->jit) jit_free(*p->jit);
    p->jit.reset();
    for (cudaStream_t st : p->pf_streams) cudaStreamDestroy(st);
    for (cudaEvent_t ev : p->pf_done) cudaEventDestroy(ev);
    if (p->pf_fork) cudaEventDestroy(p->pf_fork);
    p->pf_streams.clear();
    p->pf_done.clear();
    p->pf_fork = nullptr;
}

void free_graphs(gbvqc_circuit *c)
{
    for (auto &kv : c->graphs) cudaGraphExecDestroy(kv.second);
    c->graphs.clear();
}

static void free_workspace(Workspace &w)
{
    dev_free(w.phi); dev_free(w.psi); dev_free(w.d_theta); dev_free(w.d_energy); dev_free(w.d_grad);
    dev_free(w.d_slot_grad); dev_free(w.d_slot_partials); dev_free(w.d_red); dev_free(w.d_counter);
    w = Workspace();
}

extern "C" gbvqc_status circuit_free(circuit_handle c)
{
    if (!c) return GBVQC_OK;
    free_graphs(c);
    for (auto &kv : c->plans) free_plan(kv.second.get());
    free_workspace(c->ws);
    dev_free(c->d_recs); dev_free(c->d_dyn); dev_free(c->d_plain_ptr); dev_free(c->d_plain_slots);
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    delete c;
    return GBVQC_OK;
}

gbvqc_status csr_upload(const std::vector<int> &slot_param, int n_params, int **d_ptr, int **d_slots)
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

// A general one-qubit unitary U = e^{i alpha} V with V real (SH_REAL1), with a real
// diagonal and an imaginary off-diagonal (SH_IMAG1), or with a real diagonal only (kept
// SH_DENSE1; the specialised passes apply it as SH_RDIAG1): sqrt(Y), sqrt(X) and sqrt(W)
// are of these kinds up to the phase e^{i pi/4}, and V costs 6 or 10 instead of 14 flops
// per amplitude.
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
    for (int pattern = 0; pattern < 3; pattern++) {
        double a;
        if (pattern == 0) a = std::arg(U[kmax]);  // real: any largest entry sets the phase
        else {  // imaginary off-diagonal, or (2) a real diagonal only: the diagonal does
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
            } else if (pattern == 1) {
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

// Plan-time variant of a fixed SH_BLOCK2 record, for the specialised passes (FGate.perm of
// an FT_BLOCK2 gate): BLOCK2_VARIANT | the shape of the 2x2 on {|01>, |10>} (0 general,
// 1 real diagonal and imaginary off-diagonal, 2 real) | BLOCK2_P00_ONE / BLOCK2_P11_ONE
// when the phase on |00> / |11> is exactly 1 in both precisions.  Exact comparisons: a
// variant only drops terms that are exactly zero, so results are unchanged.
static int block2_variant(const MatRec &r)
{
    auto zero = [&](int i) { return r.d[i] == 0.0 && r.f[i] == 0.0f; };
    auto one = [&](int i) { return r.d[i] == 1.0 && r.f[i] == 1.0f; };
    int v = BLOCK2_VARIANT;
    if (zero(11) && zero(13) && zero(19) && zero(21)) v |= 2;
    else if (zero(11) && zero(21) && zero(12) && zero(18)) v |= 1;
    if (one(0) && zero(1)) v |= BLOCK2_P00_ONE;
    if (one(30) && zero(31)) v |= BLOCK2_P11_ONE;
    return v;
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
    if (c->density) return;
    const double ph = std::remainder(phase, 2.0 * M_PI);
    const cd z = std::polar(1.0, ph);
    if (ph == 0.0) {
    } else if (fold >= 0) {  // shape kept: same ftype and permutation bits
        out[fold].rec_f = add_rec(c, mat_scaled(fold_f, z));
        out[fold].rec_i = out[fold].rec_a = add_rec(c, mat_scaled(fold_i, std::conj(z)));
    } else if (first_norm >= 0) {  // back to a general 2x2 on the first normalised gate
        const Mat W = mat_scaled(norm_f, z);
        out[first_norm].rec_f = add_rec(c, W);
        out[first_norm].rec_i = out[first_norm].rec_a = add_rec(c, mat_dagger(W, 2));
        out[first_norm].ftype = FT_DENSE1;
    }
    // fixed block gates (FSIM with constant angles) and dense one-qubit gates: the
    // structure of their final matrices
    std::vector<char> dynamic(c->recs.size(), 0);
    for (const DynRec &d : c->dyn) dynamic[d.rec] = 1;
    auto real_diag = [&](int rec) {
        const MatRec &r = c->recs[rec];
        return r.d[1] == 0.0 && r.d[7] == 0.0 && r.f[1] == 0.0f && r.f[7] == 0.0f;
    };
    for (PGate &g : out) {
        if (dynamic[g.rec_f] || dynamic[g.rec_i] || g.rec_a != g.rec_i) continue;
        if (g.ftype == FT_BLOCK2) {
            g.perm_f = block2_variant(c->recs[g.rec_f]);
            g.perm_r = block2_variant(c->recs[g.rec_i]);
        } else if (g.ftype == FT_DENSE1 && g.k == 1) {
            g.rdiag = real_diag(g.rec_f) && real_diag(g.rec_i);
        }
    }
    // rotations [[c, -s], [s, c]] (Ry, fixed or variational) in every direction
    auto rotation = [&](int rec) {
        const MatRec &r = c->recs[rec];
        for (int i = 1; i < 8; i += 2)
            if (r.d[i] != 0.0) return false;
        return r.d[0] == r.d[6] && r.d[2] == -r.d[4];
    };
    for (PGate &g : out)
        if (g.ftype == FT_REAL1 && g.k == 1 && g.rec_a == g.rec_i)
            g.rot = g.param >= 0 || (!dynamic[g.rec_f] && !dynamic[g.rec_i] && rotation(g.rec_f) && rotation(g.rec_i));
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
gbvqc_status ensure_device(gbvqc_circuit *c)
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
int max_tile(int dtype)
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
gbvqc_status get_host_plan(gbvqc_circuit *c, int dtype, bool grad_layout, DevPlan **out, bool batch, bool jit)
{
    int key = dtype * 2 + (grad_layout ? 1 : 0) + (batch ? 4 : 0) + (jit ? 8 : 0);
    auto it = c->plans.find(key);
    if (it != c->plans.end()) {
        *out = it->second.get();
        return GBVQC_OK;
    }
    const std::vector<PGate> &pg0 = (grad_layout && c->density) ? c->pg_grad : c->pg_std;
    PlanOptions opt;
    opt.t = c->tile_qubits ? c->tile_qubits : default_tile(dtype);
    opt.low = c->low_qubits ? c->low_qubits : default_low(dtype);
    const int64_t tiles = int64_t(1) << (c->n_phys - std::min(std::min(opt.t, max_tile(dtype)), c->n_phys));
    opt.nr_f = jit ? jit_nr(dtype, false, tiles) : fused_nr(dtype, false);
    opt.nr_r = jit ? jit_nr(dtype, true, tiles) : fused_nr(dtype, true);
    opt.t = std::min(opt.t, max_tile(dtype));
    opt.elem_bytes = dtype == GBVQC_C64 ? 4 : 8;
    opt.max_slots = batch ? 128 : 512;
    opt.gate_smem = batch ? 40 * 1024 : 64 * 1024;
    opt.phase_tables = true;  // (batch members' images: one batched gather per step)
    // a gradient ignores global phases: rotations as shears in every pure-state gradient plan
    opt.rot_shears = grad_layout && !c->density;
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
gbvqc_status get_plan(gbvqc_circuit *c, int dtype, bool grad_layout, DevPlan **out, bool batch, bool jit)
{
    DevPlan *dp = nullptr;
    ST_TRY(get_host_plan(c, dtype, grad_layout, &dp, batch, jit));
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
        ST_TRY(upload(&dp->d_ftabs, dp->p.ftabs));
        ST_TRY(upload(&dp->d_rtabs, dp->p.rtabs));
        ST_TRY(upload(&dp->d_ftabents, dp->p.ftabents));
        ST_TRY(upload(&dp->d_rtabents, dp->p.rtabents));
        const size_t eb = dtype == GBVQC_C64 ? 4 : 8;
        ST_TRY(dev_alloc((unsigned char **)&dp->d_fimg, std::max<size_t>(1, 8 * eb * dp->p.funits.size())));
        ST_TRY(dev_alloc((unsigned char **)&dp->d_rimg, std::max<size_t>(1, 8 * eb * dp->p.runits.size())));
        ST_TRY(csr_upload(dp->p.slot_param, c->n_params, &dp->d_csr_ptr, &dp->d_csr_slots));
        dp->uploaded = true;
    }
    *out = dp;
    return GBVQC_OK;
}

bool fused_supported(const gbvqc_circuit *c, int dtype)
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
    dev_free(c->ws.d_slot_partials);
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

extern "C" gbvqc_status circuit_specialize(circuit_handle c, int dtype, int for_grad, int *n_kernels, int *n_cached,
                                          double *seconds)
{
    if (!c) return fail(GBVQC_ERR_ARG, "NULL circuit");
    if (dtype != GBVQC_C64 && dtype != GBVQC_C128) return fail(GBVQC_ERR_ARG, "dtype %d", dtype);
    std::lock_guard<std::mutex> lk(c->mu);
    if (!fused_supported(c, dtype)) return fail(GBVQC_ERR_UNSUPPORTED, "too few qubits for tiles");
    DevPlan *p = nullptr;
    ST_TRY(get_host_plan(c, dtype, for_grad != 0, &p, false, true));
    std::vector<JitModule> mods;
    double secs = 0;
    std::string err;
    if (!jit_compile(p->p, dtype, for_grad != 0, mods, secs, err))
        return fail(GBVQC_ERR_CUDA, "specialising the tile passes: %s", err.c_str());
    int cached = 0;
    for (const JitModule &m : mods) cached += m.from_cache ? 1 : 0;
    if (n_kernels) *n_kernels = (int)mods.size();
    if (n_cached) *n_cached = cached;
    if (seconds) *seconds = secs;
    return GBVQC_OK;
}
