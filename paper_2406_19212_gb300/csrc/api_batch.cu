// C ABI: batches of independent circuits evaluated by shared launches (one CUDA-graph
// replay per batch).
#include "api_internal.h"

// ------------------------------------------------------------------------ batches

struct BatchLaunch {
    bool twoq;
    int t;
    FusedBatchEntry *d_entries = nullptr;
    int n_entries = 0;
    int64_t tiles = 0;
    size_t smem = 0;
};

struct gbvqc_batch {
    std::vector<gbvqc_circuit *> circs;
    std::vector<gbvqc_obs *> obs;
    int dtype = 0, n = 0, total_params = 0;
    std::vector<int> param_off;
    void *phi_all = nullptr, *psi_all = nullptr;
    size_t state_bytes = 0;
    int64_t *d_amp_off = nullptr;
    BatchDyn *d_dyn = nullptr;
    int n_dyn = 0;
    double *d_theta = nullptr, *d_energies = nullptr, *d_grads = nullptr, *d_slot_grad = nullptr;
    double *d_slot_partials = nullptr, *d_pauli_partials = nullptr;
    std::vector<BatchLaunch> fwd, rev;
    PauliBatchEntry *d_pauli = nullptr;
    int64_t pauli_chunks = 0;
    size_t pauli_smem = 0;  // staged observables' shared memory (0: global-memory path)
    SlotBatchEntry *d_slots = nullptr;
    int64_t total_slots = 0;
    int *d_csr_ptr = nullptr, *d_csr_slots = nullptr;
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t graph = nullptr;
    bool init_in_pass = false;  // every member's first forward pass writes its |0...0> start
    GatherArgs *d_gather = nullptr;  // per member: its plan's per-step image (phase tables)
    int64_t *d_gather_off = nullptr;
    int64_t gather_total = 0;
};

// Device resources of a batch (everything batch_build makes); the member lists stay.
static void batch_release(gbvqc_batch *b)
{
    if (b->graph) cudaGraphExecDestroy(b->graph);
    if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
    for (auto *L : {&b->fwd, &b->rev})
        for (BatchLaunch &l : *L) dev_free(l.d_entries);
    dev_free(b->phi_all); dev_free(b->psi_all); dev_free(b->d_amp_off); dev_free(b->d_dyn);
    dev_free(b->d_theta); dev_free(b->d_energies); dev_free(b->d_grads); dev_free(b->d_slot_grad);
    dev_free(b->d_slot_partials); dev_free(b->d_pauli_partials); dev_free(b->d_pauli);
    dev_free(b->d_slots); dev_free(b->d_csr_ptr); dev_free(b->d_csr_slots);
    dev_free(b->d_gather); dev_free(b->d_gather_off);
    gbvqc_batch fresh;
    fresh.circs = std::move(b->circs);
    fresh.obs = std::move(b->obs);
    fresh.dtype = b->dtype;
    fresh.n = b->n;
    fresh.total_params = b->total_params;
    fresh.param_off = std::move(b->param_off);
    *b = std::move(fresh);
}

extern "C" gbvqc_status batch_free(batch_handle b)
{
    if (!b) return GBVQC_OK;
    batch_release(b);
    delete b;
    return GBVQC_OK;
}

static gbvqc_status batch_build(gbvqc_batch *b)
{
    const int n = b->n, dtype = b->dtype;
    const size_t amp = amp_size(dtype);
    std::vector<DevPlan *> plans(n);
    std::vector<int64_t> amp_off(n), slot_off(n), part_off(n), chunk_off(n);
    int64_t amps = 0, slots = 0, parts = 0, chunks = 0;
    int max_passes = 0;
    std::vector<BatchDyn> dyn;
    for (int i = 0; i < n; i++) {
        gbvqc_circuit *c = b->circs[i];
        ST_TRY(ensure_device(c));
        ST_TRY(ensure_obs(b->obs[i]));
        ST_TRY(get_plan(c, dtype, true, &plans[i], true));
        for (int bi : plans[i]->p.barrier)
            if (bi >= 0) return fail(GBVQC_ERR_UNSUPPORTED, "batch member %d holds a two-qubit channel", i);
        const FusedPlan &P = plans[i]->p;
        amp_off[i] = amps;
        amps += int64_t(1) << c->n_phys;
        slot_off[i] = slots;
        slots += P.n_slots;
        part_off[i] = parts;
        parts += (int64_t)P.n_slots << (c->n_phys - P.t);
        chunk_off[i] = chunks;
        chunks += ((int64_t(1) << c->n_phys) + (1 << kPauliChunkBits) - 1) >> kPauliChunkBits;
        max_passes = std::max(max_passes, (int)P.fwd.size());
        for (const DynRec &d : c->dyn)
            dyn.push_back(BatchDyn{c->d_recs + d.rec, b->param_off[i] + d.param, 0, d});
    }
    b->state_bytes = (size_t)amps * amp;
    ST_TRY(dev_alloc((unsigned char **)&b->phi_all, b->state_bytes));
    ST_TRY(dev_alloc((unsigned char **)&b->psi_all, b->state_bytes));
    ST_TRY(upload(&b->d_amp_off, amp_off));
    ST_TRY(upload(&b->d_dyn, dyn));
    b->n_dyn = (int)dyn.size();
    ST_TRY(dev_alloc(&b->d_theta, b->total_params + 1));
    ST_TRY(dev_alloc(&b->d_energies, n));
    ST_TRY(dev_alloc(&b->d_grads, b->total_params + 1));
    ST_TRY(dev_alloc(&b->d_slot_grad, slots + 1));
    ST_TRY(dev_alloc(&b->d_slot_partials, parts + 1));
    ST_TRY(dev_alloc(&b->d_pauli_partials, chunks + 1));
    b->total_slots = slots;
    b->pauli_chunks = chunks;
    auto state_ptr = [&](void *base, int i) { return (void *)((unsigned char *)base + amp_off[i] * amp); };
    // fused launches: pass p of every circuit that has one, grouped by tile size
    CUDA_TRY(fused_batch_prepare());
    b->init_in_pass = true;
    for (int i = 0; i < n; i++) b->init_in_pass = b->init_in_pass && !plans[i]->p.fwd.empty();
    for (int dir = 0; dir < 2; dir++) {
        const bool rev = dir == 1;
        for (int r = 0; r < max_passes; r++) {
            std::map<int, std::vector<int>> by_t;
            for (int i = 0; i < n; i++) {
                const int np = (int)plans[i]->p.fwd.size();
                const int p = rev ? np - 1 - r : r;
                if (p >= 0 && p < np) by_t[plans[i]->p.t].push_back(i);
            }
            for (auto &kv : by_t) {
                BatchLaunch L;
                L.t = kv.first;
                L.twoq = false;
                std::vector<FusedBatchEntry> ents;
                for (int i : kv.second) {
                    DevPlan *dp = plans[i];
                    const int np = (int)dp->p.fwd.size();
                    const int p = rev ? np - 1 - r : r;
                    const PassDesc &d = rev ? dp->p.rev[p] : dp->p.fwd[p];
                    FusedBatchEntry e{};
                    if (rev)
                        e.args = FusedArgs{dp->d_rev + p, dp->d_rsubs, dp->d_rgates, dp->d_rents, dp->d_runits,
                                           b->circs[i]->d_recs, dp->d_rimg, b->d_slot_partials + part_off[i],
                                           1 << (b->circs[i]->n_phys - dp->p.t)};
                    else
                        e.args = FusedArgs{dp->d_fwd + p, dp->d_fsubs, dp->d_fgates, dp->d_fents, dp->d_funits,
                                           b->circs[i]->d_recs, dp->d_fimg, nullptr, 0};
                    // the first forward pass starts from |0...0>: only the member's tile 0
                    // runs its gates, the others are written as zeros (FusedArgs::init)
                    if (!rev && p == 0 && b->init_in_pass) e.args.init = 1;
                    e.phi = state_ptr(b->phi_all, i);
                    e.psi = rev ? state_ptr(b->psi_all, i) : nullptr;
                    e.begin = L.tiles;
                    L.tiles += int64_t(1) << (b->circs[i]->n_phys - dp->p.t);
                    L.twoq = L.twoq || d.has_2q;
                    L.smem = std::max(L.smem, rev ? dp->rev_smem[p] : dp->fwd_smem[p]);
                    ents.push_back(e);
                }
                L.n_entries = (int)ents.size();
                ST_TRY(upload(&L.d_entries, ents));
                (rev ? b->rev : b->fwd).push_back(L);
            }
        }
    }
    std::vector<PauliBatchEntry> pe(n);
    std::vector<SlotBatchEntry> se(n);
    std::vector<int> gslot_param(slots, -1);
    for (int i = 0; i < n; i++) {
        ObsDev od;
        ST_TRY(obs_dev_perm(b->obs[i], plans[i]->perm, &od));
        pe[i] = PauliBatchEntry{state_ptr(b->phi_all, i), state_ptr(b->psi_all, i), od,
                                b->d_pauli_partials + chunk_off[i], b->circs[i]->n_phys, 0, chunk_off[i]};
        se[i] = SlotBatchEntry{b->d_slot_partials + part_off[i], 1 << (b->circs[i]->n_phys - plans[i]->p.t), 0,
                               slot_off[i]};
        for (int s = 0; s < plans[i]->p.n_slots; s++)
            gslot_param[slot_off[i] + s] = b->param_off[i] + plans[i]->p.slot_param[s];
    }
    bool staged = true;
    for (int i = 0; i < n; i++) {
        ObsDev od;
        ST_TRY(obs_dev_perm(b->obs[i], plans[i]->perm, &od));
        staged = staged && obs_stageable(od, b->dtype);
        b->pauli_smem = std::max(b->pauli_smem, obs_smem_bytes(od, b->dtype));
    }
    if (!staged) b->pauli_smem = 0;
    // per-step matrix images of every member (their phase tables), one launch
    std::vector<GatherArgs> ga(n);
    std::vector<int64_t> goff(n + 1, 0);
    for (int i = 0; i < n; i++) {
        DevPlan *p = plans[i];
        ga[i] = GatherArgs{p->d_funits, (int)p->p.funits.size(), p->d_runits, (int)p->p.runits.size(), p->d_fimg,
                           p->d_rimg, b->circs[i]->d_recs, p->d_ftabs, p->d_rtabs, p->d_ftabents, p->d_rtabents,
                           (int)p->p.ftabs.size(), (int)p->p.rtabs.size(), p->p.nr_f, p->p.nr_r};
        goff[i + 1] = goff[i] + gather_items(ga[i]);
    }
    b->gather_total = goff[n];
    ST_TRY(upload(&b->d_gather, ga));
    ST_TRY(upload(&b->d_gather_off, goff));
    ST_TRY(upload(&b->d_pauli, pe));
    ST_TRY(upload(&b->d_slots, se));
    ST_TRY(csr_upload(gslot_param, b->total_params, &b->d_csr_ptr, &b->d_csr_slots));
    CUDA_TRY(cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking));
    return GBVQC_OK;
}

static gbvqc_status batch_enqueue(gbvqc_batch *b, cudaStream_t s)
{
    CUDA_TRY(launch_batch_init(b->d_dyn, b->n_dyn, b->d_theta, b->dtype, b->phi_all, b->state_bytes, b->d_amp_off,
                               b->n, s, !b->init_in_pass));
    CUDA_TRY(launch_gather_batch(b->dtype, b->d_gather, b->d_gather_off, b->n, b->gather_total, s));
    for (const BatchLaunch &L : b->fwd)
        CUDA_TRY(launch_fused_batch(b->dtype, false, L.twoq, L.t, L.d_entries, L.n_entries, L.tiles, L.smem, s));
    CUDA_TRY(launch_pauli_batch(b->dtype, b->d_pauli, b->n, b->pauli_chunks, b->pauli_smem, b->d_energies, s));
    for (const BatchLaunch &L : b->rev)
        CUDA_TRY(launch_fused_batch(b->dtype, true, L.twoq, L.t, L.d_entries, L.n_entries, L.tiles, L.smem, s));
    CUDA_TRY(launch_slots_batch(b->d_slots, b->n, b->total_slots, b->d_slot_grad, s));
    CUDA_TRY(launch_accumulate(b->d_slot_grad, b->d_csr_ptr, b->d_csr_slots, b->total_params, b->d_grads, s));
    return GBVQC_OK;
}

extern "C" gbvqc_status batch_create(const circuit_handle *circuits, const obs_handle *observables, int n_circuits,
                                     int dtype, batch_handle *out)
{
    if (!out || !circuits || !observables || n_circuits < 1) return fail(GBVQC_ERR_ARG, "bad arguments");
    *out = nullptr;
    if (dtype != GBVQC_C64 && dtype != GBVQC_C128) return fail(GBVQC_ERR_ARG, "dtype %d", dtype);
    gbvqc_batch *b = new gbvqc_batch();
    b->dtype = dtype;
    b->n = n_circuits;
    for (int i = 0; i < n_circuits; i++) {
        gbvqc_circuit *c = circuits[i];
        gbvqc_obs *h = observables[i];
        if (!c || !h) { batch_free(b); return fail(GBVQC_ERR_ARG, "circuit or observable %d is NULL", i); }
        if (c->density) { batch_free(b); return fail(GBVQC_ERR_ARG, "circuit %d is a density circuit", i); }
        if (h->n_qubits != c->n_log) { batch_free(b); return fail(GBVQC_ERR_ARG, "observable %d qubit count", i); }
        if (!fused_supported(c, dtype)) { batch_free(b); return fail(GBVQC_ERR_UNSUPPORTED, "circuit %d: too few qubits", i); }
        b->circs.push_back(c);
        b->obs.push_back(h);
        b->param_off.push_back(b->total_params);
        b->total_params += c->n_params;
    }
    gbvqc_status st = batch_build(b);
    if (st != GBVQC_OK) {
        batch_free(b);
        return st;
    }
    *out = b;
    return GBVQC_OK;
}

extern "C" gbvqc_status batch_grad(batch_handle b, const double *theta_all, int n_theta_total, int ptr_loc,
                                   void *stream, double *energies, double *grads)
{
    if (!b || !energies || (!grads && b->total_params > 0)) return fail(GBVQC_ERR_ARG, "NULL argument");
    if (n_theta_total != b->total_params)
        return fail(GBVQC_ERR_ARG, "expected %d parameters, got %d", b->total_params, n_theta_total);
    if (n_theta_total > 0 && !theta_all) return fail(GBVQC_ERR_ARG, "theta is NULL");
    if (ptr_loc != GBVQC_PTR_HOST && ptr_loc != GBVQC_PTR_DEVICE) return fail(GBVQC_ERR_ARG, "ptr_loc %d", ptr_loc);
    cudaStream_t s = (cudaStream_t)stream;
    const cudaMemcpyKind in = ptr_loc == GBVQC_PTR_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    const cudaMemcpyKind outk = ptr_loc == GBVQC_PTR_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (n_theta_total > 0) CUDA_TRY(cudaMemcpyAsync(b->d_theta, theta_all, sizeof(double) * n_theta_total, in, s));
    if (!b->graph) {
        cudaGraph_t graph = nullptr;
        CUDA_TRY(cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal));
        gbvqc_status st = batch_enqueue(b, b->cap_stream);
        cudaError_t e = cudaStreamEndCapture(b->cap_stream, &graph);
        if (st != GBVQC_OK) {
            if (graph) cudaGraphDestroy(graph);
            return st;
        }
        CUDA_TRY(e);
        e = cudaGraphInstantiate(&b->graph, graph, 0);
        cudaGraphDestroy(graph);
        CUDA_TRY(e);
    }
    CUDA_TRY(cudaGraphLaunch(b->graph, s));
    CUDA_TRY(cudaMemcpyAsync(energies, b->d_energies, sizeof(double) * b->n, outk, s));
    if (b->total_params > 0)
        CUDA_TRY(cudaMemcpyAsync(grads, b->d_grads, sizeof(double) * b->total_params, outk, s));
    if (ptr_loc == GBVQC_PTR_HOST) CUDA_TRY(cudaStreamSynchronize(s));
    return GBVQC_OK;
}

extern "C" gbvqc_status grad_batch(const circuit_handle *circuits, const obs_handle *observables, int n_circuits,
                                   const double *theta_all, void *stream, double *energies, double *grads)
{
    batch_handle b = nullptr;
    ST_TRY(batch_create(circuits, observables, n_circuits, GBVQC_C64, &b));
    gbvqc_status st = batch_grad(b, theta_all, b->total_params, GBVQC_PTR_HOST, stream, energies, grads);
    batch_free(b);
    return st;
}

// Rebuild the batch after its members' tilings changed.
static gbvqc_status batch_rebuild(gbvqc_batch *b)
{
    batch_release(b);
    return batch_build(b);
}

extern "C" gbvqc_status batch_autotune(batch_handle b, const double *theta_all, int n_theta_total, void *stream,
                                       int *tiles, double *best_ms)
{
    if (!b || !best_ms || (n_theta_total > 0 && !theta_all)) return fail(GBVQC_ERR_ARG, "NULL argument");
    if (n_theta_total != b->total_params)
        return fail(GBVQC_ERR_ARG, "expected %d parameters, got %d", b->total_params, n_theta_total);
    const int n = b->n, tmax = max_tile(b->dtype);
    std::vector<double> e(n), g(std::max(1, b->total_params));
    cudaEvent_t e0, e1;
    CUDA_TRY(cudaEventCreate(&e0));
    CUDA_TRY(cudaEventCreate(&e1));
    // member i's tile for a requested size: within [8, 12] and the member's qubits
    auto clamp_tile = [&](int i, int t) { return std::max(6, std::min({t, tmax, b->circs[i]->n_phys})); };
    auto evaluate = [&](const std::vector<int> &t, double *ms) -> gbvqc_status {
        for (int i = 0; i < n; i++)
            if (b->circs[i]->tile_qubits != t[i]) ST_TRY(circuit_set_tiling(b->circs[i], t[i], b->circs[i]->low_qubits));
        ST_TRY(batch_rebuild(b));
        // one call captures the graph; then the median of three timed calls
        ST_TRY(batch_grad(b, theta_all, n_theta_total, GBVQC_PTR_HOST, stream, e.data(), g.data()));
        std::vector<double> runs;
        for (int r = 0; r < 3; r++) {
            CUDA_TRY(cudaEventRecord(e0, (cudaStream_t)stream));
            ST_TRY(batch_grad(b, theta_all, n_theta_total, GBVQC_PTR_HOST, stream, e.data(), g.data()));
            CUDA_TRY(cudaEventRecord(e1, (cudaStream_t)stream));
            CUDA_TRY(cudaEventSynchronize(e1));
            float f = 0;
            CUDA_TRY(cudaEventElapsedTime(&f, e0, e1));
            runs.push_back(f);
        }
        std::sort(runs.begin(), runs.end());
        *ms = runs[1];
        return GBVQC_OK;
    };
    gbvqc_status st = GBVQC_OK;
    std::vector<int> best(n), cur(n);
    double best_t = 1e30;
    // one tile size for every member (clamped to its qubits) ...
    for (int T = 8; T <= 12 && st == GBVQC_OK; T++) {
        for (int i = 0; i < n; i++) cur[i] = clamp_tile(i, T);
        double ms = 0;
        st = evaluate(cur, &ms);
        if (st == GBVQC_OK && ms < best_t) best_t = ms, best = cur;
    }
    // ... then per qubit-count class, the classes with the most amplitudes first
    std::map<int, double> weight;
    for (int i = 0; i < n; i++) weight[b->circs[i]->n_phys] += std::ldexp(1.0, b->circs[i]->n_phys);
    std::vector<std::pair<double, int>> classes;
    for (auto &kv : weight) classes.push_back({-kv.second, kv.first});
    std::sort(classes.begin(), classes.end());
    for (size_t ci = 0; ci < classes.size() && ci < 4 && st == GBVQC_OK; ci++) {
        const int nq = classes[ci].second;
        for (int T = 8; T <= 12 && st == GBVQC_OK; T++) {
            cur = best;
            bool changed = false;
            for (int i = 0; i < n; i++)
                if (b->circs[i]->n_phys == nq && cur[i] != clamp_tile(i, T)) cur[i] = clamp_tile(i, T), changed = true;
            if (!changed) continue;
            double ms = 0;
            st = evaluate(cur, &ms);
            if (st == GBVQC_OK && ms < best_t) best_t = ms, best = cur;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != GBVQC_OK) return st;
    for (int i = 0; i < n; i++)
        if (b->circs[i]->tile_qubits != best[i]) ST_TRY(circuit_set_tiling(b->circs[i], best[i], b->circs[i]->low_qubits));
    ST_TRY(batch_rebuild(b));
    if (tiles)
        for (int i = 0; i < n; i++) tiles[i] = best[i];
    *best_ms = best_t;
    return GBVQC_OK;
}
