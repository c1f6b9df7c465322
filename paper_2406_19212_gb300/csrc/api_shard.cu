// C ABI: a state sharded over 2^g parts by its g global qubits, with qubit-swap exchange.
//
// The paper simulates beyond one device through distributed simulators (Introduction);
// the standard partition of a 2^n state over 2^g devices takes the g highest index bits
// as the device index.  Gates on the other (local) qubits act on every shard
// independently.  A diagonal gate on a global qubit needs no data either: every shard
// knows its global bits, so it becomes a phase of the whole shard or a diagonal gate on
// the local partner.  Any other gate on a global qubit first trades that qubit's position
// with a local qubit's: shard s and its partner s ^ 2^j exchange the half of their
// amplitudes in which the two bits differ (one all-to-all of half the state over pairs of
// shards).  The planner picks, for every such gate, the local qubit whose next
// non-diagonal use is farthest away (the classic furthest-next-use rule), which minimises
// the swaps of a lookahead-free schedule for a fixed gate order.
//
// On one GPU the shards are separate device buffers of the same device and the exchange
// is a swap kernel between two buffers; on a multi-GPU node each shard would live on its
// own device and the exchange would be a peer copy of the contiguous half (the library
// has no multi-GPU transport: the runs of this build have one GPU).
#include "api_internal.h"

namespace {

struct ShardStep {
    int kind;  // 0: ops [a, b) of the circuit; 1: swap global bit a with local bit b
    int a, b;
};

// An op with theta's values written in (param_index = -1), so gate_matrix applies.
gbvqc_op fixed_op(const gbvqc_op &op, const double *theta)
{
    gbvqc_op f = op;
    if (op.param_index >= 0 && theta) {
        if (op.kind == GBVQC_FSIM) {
            int j = 0;
            for (int k = 0; k < 5; k++)
                if ((op.param_mask >> k) & 1) f.params[k] = theta[op.param_index + j++];
            f.param_mask = 0;
        } else {
            f.params[0] = theta[op.param_index];
        }
    }
    f.param_index = -1;
    return f;
}

// Whether an op of the circuit is diagonal for every theta (no exchange needed).
bool op_diagonal(const gbvqc_op &op)
{
    if (op.kind == GBVQC_RZ) return true;
    if (op.param_index >= 0) return false;  // variational RX / RY / FSIM
    const int sh = classify(gate_matrix(op));
    return sh == SH_DIAG1 || sh == SH_DIAG2 || sh == SH_CZ;
}

bool plan_shards(const gbvqc_circuit *c, int g, std::vector<ShardStep> &steps, std::vector<int> &pos,
                 std::string &err)
{
    const int n = c->n_log, L = n - g;
    const int m = (int)c->ops.size();
    pos.resize(n);
    for (int q = 0; q < n; q++) pos[q] = q;
    // per qubit, the ops that use it non-diagonally, in order
    std::vector<std::vector<int>> uses(n);
    std::vector<char> diag(m);
    for (int i = 0; i < m; i++) {
        const gbvqc_op &op = c->ops[i];
        diag[i] = op_diagonal(op) ? 1 : 0;
        if (!diag[i])
            for (int u = 0; u < kind_qubits(op.kind); u++) uses[op.qubits[u]].push_back(i);
    }
    std::vector<size_t> head(n, 0);
    auto next_use = [&](int q, int i) {
        while (head[q] < uses[q].size() && uses[q][head[q]] < i) head[q]++;
        return head[q] < uses[q].size() ? uses[q][head[q]] : m;
    };
    steps.clear();
    int seg_begin = 0;
    for (int i = 0; i < m; i++) {
        const gbvqc_op &op = c->ops[i];
        const int k = kind_qubits(op.kind);
        if (!diag[i])
            for (int u = 0; u < k; u++) {
                const int q = op.qubits[u];
                if (pos[q] < L) continue;
                int victim = -1, best = -1;
                for (int y = 0; y < n; y++) {
                    if (pos[y] >= L) continue;
                    bool in_op = false;
                    for (int v = 0; v < k; v++) in_op = in_op || op.qubits[v] == y;
                    if (in_op) continue;
                    const int nu = next_use(y, i);
                    if (nu > best) best = nu, victim = y;
                }
                if (victim < 0) {
                    err = "not enough local qubits for op " + std::to_string(i);
                    return false;
                }
                if (i > seg_begin) steps.push_back(ShardStep{0, seg_begin, i});
                seg_begin = i;
                steps.push_back(ShardStep{1, pos[q] - L, pos[victim]});
                std::swap(pos[q], pos[victim]);
            }
    }
    if (m > seg_begin) steps.push_back(ShardStep{0, seg_begin, m});
    return true;
}

// The op for shard s (global bits of the shard fixed): non-diagonal ops (all of whose
// qubits the schedule made local) and local diagonal ops with their local positions;
// diagonal ops on global qubits reduced to the shard's phase (DENSE1 diag(f, f) on local
// qubit 0) or to a one-qubit diagonal on the local partner.
gbvqc_op shard_op(const gbvqc_op &op0, const double *theta, const std::vector<int> &pos, int L, int s)
{
    gbvqc_op f = fixed_op(op0, theta);
    const int k = kind_qubits(f.kind);
    bool global = false;
    for (int u = 0; u < k; u++) global = global || pos[f.qubits[u]] >= L;
    if (!global) {
        for (int u = 0; u < k; u++) f.qubits[u] = pos[f.qubits[u]];
        return f;
    }
    const Mat M = gate_matrix(f);
    auto bit = [&](int q) { return (s >> (pos[q] - L)) & 1; };
    cd d0, d1;
    int target = 0;
    if (k == 1) {
        d0 = d1 = M[3 * bit(f.qubits[0])];
    } else {
        const int q0 = f.qubits[0], q1 = f.qubits[1];
        const bool g0 = pos[q0] >= L, g1 = pos[q1] >= L;
        if (g0 && g1) {
            const int r = bit(q0) + 2 * bit(q1);
            d0 = d1 = M[5 * r];
        } else if (g0) {
            const int b0 = bit(q0);
            d0 = M[5 * b0];
            d1 = M[5 * (b0 + 2)];
            target = pos[q1];
        } else {
            const int b1 = bit(q1);
            d0 = M[5 * (2 * b1)];
            d1 = M[5 * (1 + 2 * b1)];
            target = pos[q0];
        }
    }
    gbvqc_op o{};
    o.kind = GBVQC_DENSE1;
    o.qubits[0] = target;
    o.param_index = -1;
    o.data[0] = d0.real();
    o.data[1] = d0.imag();
    o.data[6] = d1.real();
    o.data[7] = d1.imag();
    return o;
}

}  // namespace

struct gbvqc_sharded {
    int n = 0, g = 0, L = 0, dtype = 0;
    std::vector<sv_handle> shards;  // 2^g states of L qubits (shard index = the global bits)
    std::vector<int> pos;           // position of logical qubit q: local bit (< L) or L + global bit
    int64_t exchanges = 0, bytes = 0;
};

extern "C" gbvqc_status shard_plan(circuit_handle c, int n_global, int32_t *steps, int max_steps, int *n_steps,
                                   int *n_swaps)
{
    if (!c || !n_steps || (max_steps > 0 && !steps) || max_steps < 0) return fail(GBVQC_ERR_ARG, "bad arguments");
    if (c->density) return fail(GBVQC_ERR_UNSUPPORTED, "sharded states are pure states");
    if (n_global < 1 || n_global >= c->n_log - 1)
        return fail(GBVQC_ERR_ARG, "n_global %d for %d qubits (at least two local qubits)", n_global, c->n_log);
    std::vector<ShardStep> st;
    std::vector<int> pos;
    std::string err;
    if (!plan_shards(c, n_global, st, pos, err)) return fail(GBVQC_ERR_ARG, "%s", err.c_str());
    int swaps = 0;
    for (size_t i = 0; i < st.size(); i++) {
        swaps += st[i].kind == 1;
        if ((int)i < max_steps) {
            steps[3 * i] = st[i].kind;
            steps[3 * i + 1] = st[i].a;
            steps[3 * i + 2] = st[i].b;
        }
    }
    *n_steps = (int)st.size();
    if (n_swaps) *n_swaps = swaps;
    return GBVQC_OK;
}

extern "C" gbvqc_status sharded_free(sharded_handle h)
{
    if (!h) return GBVQC_OK;
    for (sv_handle s : h->shards) sv_free(s);
    delete h;
    return GBVQC_OK;
}

extern "C" gbvqc_status sharded_alloc(int n_qubits, int n_global, int dtype, sharded_handle *out)
{
    if (!out) return fail(GBVQC_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (dtype != GBVQC_C64 && dtype != GBVQC_C128) return fail(GBVQC_ERR_ARG, "dtype %d", dtype);
    if (n_qubits < 3 || n_qubits > 34 || n_global < 1 || n_global > 10 || n_qubits - n_global < 2)
        return fail(GBVQC_ERR_ARG, "%d qubits with %d global", n_qubits, n_global);
    gbvqc_sharded *h = new gbvqc_sharded();
    h->n = n_qubits;
    h->g = n_global;
    h->L = n_qubits - n_global;
    h->dtype = dtype;
    for (int q = 0; q < n_qubits; q++) h->pos.push_back(q);
    for (int s = 0; s < (1 << n_global); s++) {
        sv_handle sv = nullptr;
        gbvqc_status st = sv_alloc(h->L, dtype, 0, nullptr, &sv);
        if (st == GBVQC_OK && s > 0) {  // |0...0> lives in shard 0 only
            const size_t bytes = sv->bytes();
            cudaError_t e = cudaMemset(sv->data, 0, bytes);
            if (e != cudaSuccess) st = fail(GBVQC_ERR_CUDA, "cudaMemset: %s", cudaGetErrorString(e));
        }
        if (st != GBVQC_OK) {
            if (sv) sv_free(sv);
            sharded_free(h);
            return st;
        }
        h->shards.push_back(sv);
    }
    *out = h;
    return GBVQC_OK;
}

// Host copy between the logical order (index bit q = qubit q) and the shards.
static gbvqc_status sharded_copy(sharded_handle h, void *host, bool to_device)
{
    const size_t amp = amp_size(h->dtype);
    const int64_t len = int64_t(1) << h->L, dim = int64_t(1) << h->n;
    std::vector<unsigned char> buf((size_t)dim * amp);
    unsigned char *lg = static_cast<unsigned char *>(host);
    if (!to_device)
        for (int s = 0; s < (1 << h->g); s++) ST_TRY(sv_get(h->shards[s], buf.data() + (size_t)s * len * amp, len, 1));
    for (int64_t x = 0; x < dim; x++) {
        int64_t phys = 0;
        for (int q = 0; q < h->n; q++)
            if ((x >> q) & 1) phys |= int64_t(1) << h->pos[q];
        if (to_device) memcpy(buf.data() + (size_t)phys * amp, lg + (size_t)x * amp, amp);
        else memcpy(lg + (size_t)x * amp, buf.data() + (size_t)phys * amp, amp);
    }
    if (to_device)
        for (int s = 0; s < (1 << h->g); s++) ST_TRY(sv_set(h->shards[s], buf.data() + (size_t)s * len * amp, len, 1));
    return GBVQC_OK;
}

extern "C" gbvqc_status sharded_set(sharded_handle h, const void *host_src)
{
    if (!h || !host_src) return fail(GBVQC_ERR_ARG, "NULL argument");
    return sharded_copy(h, const_cast<void *>(host_src), true);
}

extern "C" gbvqc_status sharded_get(sharded_handle h, void *host_dst)
{
    if (!h || !host_dst) return fail(GBVQC_ERR_ARG, "NULL argument");
    return sharded_copy(h, host_dst, false);
}

extern "C" gbvqc_status sharded_apply(sharded_handle h, circuit_handle c, const double *theta, int n_theta)
{
    if (!h || !c || (n_theta > 0 && !theta)) return fail(GBVQC_ERR_ARG, "NULL argument");
    if (c->density) return fail(GBVQC_ERR_UNSUPPORTED, "sharded states are pure states");
    if (c->n_log != h->n) return fail(GBVQC_ERR_ARG, "circuit has %d qubits, state %d", c->n_log, h->n);
    if (n_theta != c->n_params) return fail(GBVQC_ERR_ARG, "expected %d parameters, got %d", c->n_params, n_theta);
    // plan from the state's current positions (a permuted state stays permuted)
    std::vector<ShardStep> steps;
    std::vector<int> pos_end;
    std::string err;
    gbvqc_circuit view;  // the circuit in the state's current labelling
    view.n_log = c->n_log;
    view.ops = c->ops;
    std::vector<int> inv(h->n);
    for (int q = 0; q < h->n; q++) inv[h->pos[q]] = q;
    for (gbvqc_op &op : view.ops)
        for (int u = 0; u < kind_qubits(op.kind); u++) op.qubits[u] = h->pos[op.qubits[u]];
    if (!plan_shards(&view, h->g, steps, pos_end, err)) return fail(GBVQC_ERR_ARG, "%s", err.c_str());
    // pos_end maps view labels (= current positions) to final positions
    std::vector<int> cur(h->n);
    for (int q = 0; q < h->n; q++) cur[q] = q;  // view label -> position while the schedule runs
    const int mode = h->L >= 6 ? GBVQC_MODE_FUSED : GBVQC_MODE_PLAIN;
    for (const ShardStep &st : steps) {
        if (st.kind == 1) {  // exchange: pairs of shards differing in global bit st.a
            for (int s = 0; s < (1 << h->g); s++) {
                if ((s >> st.a) & 1) continue;
                const int t = s | (1 << st.a);
                CUDA_TRY(launch_shard_swap(h->dtype, h->shards[s]->data, h->shards[t]->data, h->L, st.b, nullptr));
                h->exchanges++;
                h->bytes += 2 * (int64_t(1) << (h->L - 1)) * (int64_t)amp_size(h->dtype);
            }
            int a = -1, b = -1;
            for (int q = 0; q < h->n; q++) {
                if (cur[q] == h->L + st.a) a = q;
                if (cur[q] == st.b) b = q;
            }
            std::swap(cur[a], cur[b]);
            continue;
        }
        for (int s = 0; s < (1 << h->g); s++) {
            std::vector<gbvqc_op> ops;
            for (int i = st.a; i < st.b; i++) {
                const gbvqc_op &op = view.ops[i];
                bool global = false;
                for (int u = 0; u < kind_qubits(op.kind); u++) global = global || cur[op.qubits[u]] >= h->L;
                if (global && !op_diagonal(op))
                    return fail(GBVQC_ERR_ARG, "internal: op %d is not local in the exchange schedule", i);
                ops.push_back(shard_op(op, theta, cur, h->L, s));
            }
            circuit_handle sc = nullptr;
            ST_TRY(circuit_create(ops.data(), (int)ops.size(), h->L, 0, 0, &sc));
            gbvqc_status r = apply_circuit(h->shards[s], sc, nullptr, 0, GBVQC_PTR_HOST, mode);
            if (r == GBVQC_OK) {
                cudaError_t e = cudaStreamSynchronize(h->shards[s]->stream);
                if (e != cudaSuccess) r = fail(GBVQC_ERR_CUDA, "%s", cudaGetErrorString(e));
            }
            circuit_free(sc);
            if (r != GBVQC_OK) return r;
        }
    }
    // view label v was the logical qubit inv[v]
    for (int v = 0; v < h->n; v++) h->pos[inv[v]] = cur[v];
    (void)pos_end;
    return GBVQC_OK;
}

extern "C" gbvqc_status sharded_info(sharded_handle h, int32_t *positions, int64_t *exchanges, int64_t *bytes)
{
    if (!h) return fail(GBVQC_ERR_ARG, "NULL handle");
    if (positions)
        for (int q = 0; q < h->n; q++) positions[q] = h->pos[q];
    if (exchanges) *exchanges = h->exchanges;
    if (bytes) *bytes = h->bytes;
    return GBVQC_OK;
}
