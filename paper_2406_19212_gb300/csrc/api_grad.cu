// C ABI: apply_circuit (Eq. circuitevolve) and the gradient of Algorithm 2, with
// CUDA-graph replay of the launch sequence and per-launch profiling.
#include "api_internal.h"

// ------------------------------------------------------------------- execution

static gbvqc_status ensure_theta(gbvqc_circuit *c)
{
    if (!c->ws.d_theta) ST_TRY(dev_alloc(&c->ws.d_theta, c->n_params + 1));
    return GBVQC_OK;
}

static gbvqc_status stage_theta(gbvqc_circuit *c, const double *theta, int n_theta, int loc, cudaStream_t s)
{
    if (n_theta != c->n_params) return fail(GBVQC_ERR_ARG, "expected %d parameters, got %d", c->n_params, n_theta);
    if (n_theta > 0 && !theta) return fail(GBVQC_ERR_ARG, "theta is NULL");
    ST_TRY(ensure_theta(c));
    if (n_theta > 0)
        CUDA_TRY(cudaMemcpyAsync(c->ws.d_theta, theta, sizeof(double) * n_theta,
                                 loc == GBVQC_PTR_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
    return GBVQC_OK;
}

double state_bytes(const gbvqc_circuit *c, int dtype) { return double(size_t(1) << c->n_phys) * amp_size(dtype); }

// Four-qubit superoperator (16 rows from record rec) on physical qubits q[0..3].
static gbvqc_status gate4(gbvqc_circuit *c, int dtype, void *psi, const int *q, int rec, cudaStream_t s)
{
    const double amps = double(size_t(1) << c->n_phys), sb = state_bytes(c, dtype);
    return run_k("gate4q", shape_flops(SH_DENSE4) * amps, 2.0 * sb, s, [&] {
        return launch_gate4(dtype, psi, c->n_phys, q[0], q[1], q[2], q[3], c->d_recs + rec, s);
    });
}

static gbvqc_status plain_gate(gbvqc_circuit *c, int dtype, void *psi, const PlainGate &g, int rec, cudaStream_t s)
{
    const double amps = double(size_t(1) << c->n_phys), sb = state_bytes(c, dtype);
    if (g.shape == SH_DENSE4) {
        const int q[4] = {g.q0, g.q1, g.q2, g.q3};
        return gate4(c, dtype, psi, q, rec, s);
    }
    const bool one = shape_qubits(g.shape) == 1;
    // complex64 runs CNOT through the controlled-2x2 kernel (launch_gate)
    const int fsh = g.shape == SH_CX && dtype == GBVQC_C64 ? SH_CTRL2 : g.shape;
    return run_k(one ? "gate1q" : "gate2q", shape_flops(fsh) * amps, (g.shape == SH_CTRL2 || g.shape == SH_CX ? 1.0 : g.shape == SH_CZ ? 0.5 : 2.0) * sb, s,
                 [&] { return launch_gate(dtype, psi, c->n_phys, g.shape, g.q0, g.q1, c->d_recs + rec, s); });
}

static gbvqc_status run_plain_forward(gbvqc_circuit *c, int dtype, void *psi, cudaStream_t s)
{
    for (const PlainGate &g : c->plain) ST_TRY(plain_gate(c, dtype, psi, g, g.rec_f, s));
    return GBVQC_OK;
}

// Matrix images of the plan's forward (and reverse) unit lists from this step's records.
static gbvqc_status gather_images(gbvqc_circuit *c, DevPlan *p, int dtype, bool with_rev, cudaStream_t s)
{
    GatherArgs g{p->d_funits, (int)p->p.funits.size(), p->d_runits, with_rev ? (int)p->p.runits.size() : 0,
                 p->d_fimg, p->d_rimg, c->d_recs, p->d_ftabs, p->d_rtabs, p->d_ftabents, p->d_rtabents,
                 (int)p->p.ftabs.size(), with_rev ? (int)p->p.rtabs.size() : 0, p->p.nr_f, p->p.nr_r};
    return run_k("gather_units", 0, 0, s, [&] { return launch_gather_units(dtype, g, s); });
}

// Specialised passes of plan p (GBVQC_MODE_JIT): compiled, or loaded from the cache, on
// first use; with_rev adds the reverse sweep's passes.  Call outside stream capture.
static gbvqc_status ensure_jit(DevPlan *p, int dtype, bool with_rev)
{
    if (p->jit && (!with_rev || !p->jit->rev.empty())) return GBVQC_OK;
    if (p->jit) jit_free(*p->jit);
    p->jit.reset(new JitPlan());
    std::string err;
    if (!jit_build(p->p, dtype, with_rev, *p->jit, err)) {
        p->jit.reset();
        return fail(GBVQC_ERR_CUDA, "specialising the tile passes: %s", err.c_str());
    }
    if (with_rev) {  // side streams of the gradient's code prefetch (made outside any capture)
        size_t n = 0;
        for (size_t i = 0; i < p->p.fwd.size(); i++) n += p->p.barrier[i] >= 0 ? 0 : 2;
        CUDA_TRY(cudaEventCreateWithFlags(&p->pf_fork, cudaEventDisableTiming));
        for (size_t i = 0; i < n; i++) {
            cudaStream_t st = nullptr;
            cudaEvent_t ev = nullptr;
            CUDA_TRY(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
            p->pf_streams.push_back(st);
            CUDA_TRY(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
            p->pf_done.push_back(ev);
        }
    }
    return GBVQC_OK;
}

// Code prefetch of the specialised passes of a gradient evaluation.  Straight-line passes
// are hundreds of kilobytes of instructions each; when the caches are cold (another
// workload ran in between) every SM would stream them from HBM at the pace of its
// instruction fetch.  A dry launch of every pass (one CTA per sub-run, each walking its
// own sub-run's code on tile 0, no global stores) is forked onto its own side stream:
// they pull the passes' code into L2 concurrently, in a few microseconds, before the real
// launches reach it.  Phase 0 forks the forward passes' prefetch at the start of the
// evaluation, phase 1 the reverse passes' after the forward sweep (so that their CTAs do
// not take SM slots from the forward passes; the expectation kernel between the sweeps
// gives them time), phase 2 makes s wait for all of them.
static gbvqc_status jit_prefetch(gbvqc_circuit *c, DevPlan *p, int phase, cudaStream_t s)
{
    if (g_prof || !p->jit || p->pf_streams.empty()) return GBVQC_OK;  // profiles time the passes alone
    if (phase == 2) {
        for (cudaEvent_t ev : p->pf_done) CUDA_TRY(cudaStreamWaitEvent(s, ev, 0));
        return GBVQC_OK;
    }
    CUDA_TRY(cudaEventRecord(p->pf_fork, s));
    Workspace &w = c->ws;
    const int tiles = 1 << (c->n_phys - p->p.t);
    size_t k = 0;
    for (int dir = 0; dir < 2; dir++)
        for (size_t i = 0; i < p->p.fwd.size(); i++) {
            if (p->p.barrier[i] >= 0) continue;
            if (dir != phase) {  // the other sweep's stream and event, left alone
                k++;
                continue;
            }
            cudaStream_t st = p->pf_streams[k];
            CUDA_TRY(cudaStreamWaitEvent(st, p->pf_fork, 0));
            const bool rev = dir == 1;
            const PassDesc &d = rev ? p->p.rev[i] : p->p.fwd[i];
            const FusedArgs args = rev ? FusedArgs{p->d_rev + i, p->d_rsubs, p->d_rgates, p->d_rents, p->d_runits,
                                                   c->d_recs, p->d_rimg, w.d_slot_partials, tiles}
                                       : FusedArgs{p->d_fwd + i, p->d_fsubs, p->d_fgates, p->d_fents, p->d_funits,
                                                   c->d_recs, p->d_fimg, nullptr, 0};
            CUDA_TRY(jit_launch(rev ? p->jit->rev[i] : p->jit->fwd[i], w.phi, w.psi, args, (unsigned)d.n_sub,
                                1 << (d.t - (rev ? p->p.nr_r : p->p.nr_f)), rev ? p->rev_smem[i] : p->fwd_smem[i],
                                st, true));
            CUDA_TRY(cudaEventRecord(p->pf_done[k], st));
            k++;
        }
    return GBVQC_OK;
}

// Forward tile passes of plan p on psi.  init: psi is not read, the sweep starts from
// |0...0> (the first pass must be a tile pass: init_in_first_pass).
static bool init_in_first_pass(const DevPlan *p) { return !p->p.fwd.empty() && p->p.barrier[0] < 0; }

static gbvqc_status run_fused_forward(gbvqc_circuit *c, DevPlan *p, int dtype, void *psi, cudaStream_t s,
                                      bool jit = false, bool init = false)
{
    const double amps = double(size_t(1) << c->n_phys), sb = state_bytes(c, dtype);
    const FusedDev fd{p->d_fwd, p->d_fsubs, p->d_fgates, p->d_fents, p->d_funits, c->d_recs, p->d_fimg};
    for (size_t i = 0; i < p->p.fwd.size(); i++) {
        if (p->p.barrier[i] >= 0) {  // two-qubit channel between the tile passes
            const PGate &g = p->p.barrier_gates[p->p.barrier[i]];
            ST_TRY(gate4(c, dtype, psi, g.q, g.rec_f, s));
            continue;
        }
        if (jit) {
            const PassDesc &d = p->p.fwd[i];
            FusedArgs args{p->d_fwd + i, p->d_fsubs, p->d_fgates, p->d_fents, p->d_funits, c->d_recs,
                           p->d_fimg, nullptr, 0};
            args.init = init && i == 0;
            ST_TRY(run_k("fused_forward", p->p.fwd_flops[i] * amps, 2 * sb, s, [&] {
                return jit_launch(p->jit->fwd[i], psi, nullptr, args, 1u << (d.n - d.t), 1 << (d.t - p->p.nr_f),
                                  p->fwd_smem[i], s);
            }));
            continue;
        }
        ST_TRY(run_k("fused_forward", p->p.fwd_flops[i] * amps, 2 * sb, s, [&] {
            return launch_fused_forward(dtype, psi, fd, (int)i, p->p.fwd[i], p->fwd_smem[i], s, init && i == 0);
        }));
    }
    return GBVQC_OK;
}

extern "C" gbvqc_status apply_circuit(sv_handle sv, circuit_handle c, const double *theta, int n_theta, int theta_loc,
                                      int mode)
{
    if (!sv || !c) return fail(GBVQC_ERR_ARG, "NULL argument");
    if (sv->n_log != c->n_log || sv->density != c->density)
        return fail(GBVQC_ERR_ARG, "state (%d qubits, density %d) does not match circuit (%d, %d)", sv->n_log,
                    sv->density, c->n_log, c->density);
    if (mode != GBVQC_MODE_PLAIN && mode != GBVQC_MODE_FUSED && mode != GBVQC_MODE_JIT)
        return fail(GBVQC_ERR_ARG, "mode %d", mode);
    std::lock_guard<std::mutex> lk(c->mu);
    cudaStream_t s = sv->stream;
    ST_TRY(ensure_device(c));
    ST_TRY(stage_theta(c, theta, n_theta, theta_loc, s));
    CUDA_TRY(launch_materialize(c->d_dyn, (int)c->dyn.size(), c->ws.d_theta, c->d_recs, s));
    if (mode != GBVQC_MODE_PLAIN && fused_supported(c, sv->dtype)) {
        DevPlan *p = nullptr;
        ST_TRY(get_plan(c, sv->dtype, false, &p, false, mode == GBVQC_MODE_JIT));
        if (mode == GBVQC_MODE_JIT) ST_TRY(ensure_jit(p, sv->dtype, false));
        ST_TRY(gather_images(c, p, sv->dtype, false, s));
        return run_fused_forward(c, p, sv->dtype, sv->data, s, mode == GBVQC_MODE_JIT);
    }
    return run_plain_forward(c, sv->dtype, sv->data, s);
}

// ------------------------------------------------------------------------ gradient

static gbvqc_status ensure_workspace(gbvqc_circuit *c, int dtype)
{
    Workspace &w = c->ws;
    if (w.dtype != dtype) {
        free_graphs(c);
        dev_free(w.phi);
        dev_free(w.psi);
        w.phi = w.psi = nullptr;
        size_t bytes = (size_t(1) << c->n_phys) * amp_size(dtype);
        ST_TRY(dev_alloc((unsigned char **)&w.phi, bytes));
        ST_TRY(dev_alloc((unsigned char **)&w.psi, bytes));
        w.dtype = dtype;
    }
    ST_TRY(ensure_theta(c));
    if (!w.d_energy) ST_TRY(dev_alloc(&w.d_energy, 1));
    if (!w.d_grad) ST_TRY(dev_alloc(&w.d_grad, c->n_params + 1));
    if (!w.d_red) ST_TRY(dev_alloc(&w.d_red, kMaxRedBlocks));
    if (!w.d_counter) {
        ST_TRY(dev_alloc(&w.d_counter, 1));
        CUDA_TRY(cudaMemset(w.d_counter, 0, sizeof(unsigned)));
    }
    return GBVQC_OK;
}

// The whole gradient evaluation as a stream-ordered launch sequence (capturable).
static gbvqc_status enqueue_grad(gbvqc_circuit *c, obs_handle h, int dtype, int mode, DevPlan *p, cudaStream_t s)
{
    Workspace &w = c->ws;
    RedScratch red{w.d_red, w.d_counter};
    const bool fused = mode != GBVQC_MODE_PLAIN && p, jit = mode == GBVQC_MODE_JIT && p;
    const double amps = double(size_t(1) << c->n_phys), sb = state_bytes(c, dtype);
    if (jit) ST_TRY(jit_prefetch(c, p, 0, s));  // first: overlaps the whole sequence
    ST_TRY(run_k("materialize", 0, 0, s, [&] {
        return launch_materialize(c->d_dyn, (int)c->dyn.size(), w.d_theta, c->d_recs, s);
    }));
    if (fused) ST_TRY(gather_images(c, p, dtype, true, s));
    // Phi starts as |0...0>: written by the first tile pass where the plan starts with one
    const bool init = fused && init_in_first_pass(p);
    if (!init) ST_TRY(run_k("zero_state", 0, sb, s, [&] { return launch_zero_state(dtype, w.phi, c->n_phys, s); }));
    if (fused) {
        ST_TRY(run_fused_forward(c, p, dtype, w.phi, s, jit, init));
        if (jit) ST_TRY(jit_prefetch(c, p, 1, s));
    } else {
        ST_TRY(run_plain_forward(c, dtype, w.phi, s));
    }
    // energy and adjoint seed
    if (c->density) {
        const DensMap &m = fused ? c->map_grad : c->map_std;
        ST_TRY(run_k("density_expect", 0, 0, s, [&] {
            return launch_density_expect(dtype, w.phi, c->n_log, m, h->dev(), red, w.d_energy, s);
        }));
        ST_TRY(run_k("density_seed", 0, sb, s, [&] {
            return launch_density_seed(dtype, w.psi, c->n_log, m, h->dev(), s);
        }));
    } else {
        ObsDev od;  // in the plan's gradient layout (copies made before any capture)
        ST_TRY(obs_dev_perm(h, fused ? p->perm : std::vector<int8_t>(), &od));
        ST_TRY(run_k("pauli_expect_seed", (8.0 * h->groups.size() + 4) * amps, 2 * sb, s, [&] {
            return launch_pauli_expect(dtype, w.phi, w.psi, c->n_phys, od, red, w.d_energy, s);
        }));
    }
    if (fused) {
        const int tiles = 1 << (c->n_phys - p->p.t);
        const FusedDev fd{p->d_rev, p->d_rsubs, p->d_rgates, p->d_rents, p->d_runits, c->d_recs, p->d_rimg};
        for (int i = (int)p->p.rev.size() - 1; i >= 0; i--) {
            if (p->p.barrier[i] >= 0) {  // Phi <- S^-1 Phi, Psi <- S^dag Psi (no parameters)
                const PGate &g = p->p.barrier_gates[p->p.barrier[i]];
                ST_TRY(gate4(c, dtype, w.phi, g.q, g.rec_i, s));
                ST_TRY(gate4(c, dtype, w.psi, g.q, g.rec_a, s));
                continue;
            }
            if (jit) {
                const PassDesc &d = p->p.rev[i];
                const FusedArgs args{p->d_rev + i, p->d_rsubs, p->d_rgates, p->d_rents, p->d_runits, c->d_recs,
                                     p->d_rimg, w.d_slot_partials, tiles};
                ST_TRY(run_k("fused_reverse", p->p.rev_flops[i] * amps, 4 * sb, s, [&] {
                    return jit_launch(p->jit->rev[i], w.phi, w.psi, args, 1u << (d.n - d.t), 1 << (d.t - p->p.nr_r),
                                      p->rev_smem[i], s);
                }));
                continue;
            }
            ST_TRY(run_k("fused_reverse", p->p.rev_flops[i] * amps, 4 * sb, s, [&] {
                return launch_fused_reverse(dtype, w.phi, w.psi, fd, i, p->p.rev[i], p->rev_smem[i],
                                            w.d_slot_partials, tiles, s);
            }));
        }
        ST_TRY(run_k("reduce_grad", 0, 0, s, [&] {
            return launch_reduce_grad(w.d_slot_partials, tiles, tiles, p->d_csr_ptr, p->d_csr_slots, c->n_params,
                                      w.d_grad, s);
        }));
        if (jit) ST_TRY(jit_prefetch(c, p, 2, s));
    } else {
        // Algorithm 2: Phi <- Q^-1 Phi; g = scale Re <Psi|dQ|Phi>; Psi <- Q^-1 Psi (Q^dag for channels)
        for (int j = (int)c->plain.size() - 1; j >= 0; j--) {
            const PlainGate &g = c->plain[j];
            ST_TRY(plain_gate(c, dtype, w.phi, g, g.rec_i, s));
            if (g.slot >= 0)
                ST_TRY(run_k("dot_derivative", (shape_flops(g.der_k == 1 ? SH_DENSE1 : SH_DENSE2) + 4) * amps, 2 * sb, s,
                             [&] {
                                 return launch_dot_matrix(dtype, w.psi, w.phi, c->n_phys, g.der_k, g.dq0, g.dq1,
                                                          c->d_recs + g.rec_d, g.gscale, red, w.d_slot_grad + g.slot, s);
                             }));
            for (int e = 0; e < g.n_extra; e++)
                ST_TRY(run_k("dot_derivative", (shape_flops(SH_DENSE2) + 4) * amps, 2 * sb, s, [&] {
                    return launch_dot_matrix(dtype, w.psi, w.phi, c->n_phys, g.der_k, g.dq0, g.dq1,
                                             c->d_recs + g.ex_rec[e], g.gscale, red, w.d_slot_grad + g.ex_slot[e], s);
                }));
            ST_TRY(plain_gate(c, dtype, w.psi, g, g.rec_a, s));
        }
        ST_TRY(run_k("accumulate", 0, 0, s, [&] {
            return launch_accumulate(w.d_slot_grad, c->d_plain_ptr, c->d_plain_slots, c->n_params, w.d_grad, s);
        }));
    }
    return GBVQC_OK;
}

extern "C" gbvqc_status grad(circuit_handle c, const double *theta, int n_theta, obs_handle h, int dtype, int mode,
                             int ptr_loc, void *stream, double *energy, double *grad_out)
{
    if (!c || !h || !energy || (!grad_out && c->n_params > 0)) return fail(GBVQC_ERR_ARG, "NULL argument");
    if (dtype != GBVQC_C64 && dtype != GBVQC_C128) return fail(GBVQC_ERR_ARG, "dtype %d", dtype);
    if (mode != GBVQC_MODE_PLAIN && mode != GBVQC_MODE_FUSED && mode != GBVQC_MODE_JIT)
        return fail(GBVQC_ERR_ARG, "mode %d", mode);
    if (ptr_loc != GBVQC_PTR_HOST && ptr_loc != GBVQC_PTR_DEVICE) return fail(GBVQC_ERR_ARG, "ptr_loc %d", ptr_loc);
    if (h->n_qubits != c->n_log) return fail(GBVQC_ERR_ARG, "observable has %d qubits, circuit %d", h->n_qubits, c->n_log);
    std::lock_guard<std::mutex> lk(c->mu);
    cudaStream_t s = (cudaStream_t)stream;
    ST_TRY(ensure_device(c));
    ST_TRY(ensure_obs(h));
    DevPlan *p = nullptr;
    if (mode != GBVQC_MODE_PLAIN && fused_supported(c, dtype)) {
        ST_TRY(get_plan(c, dtype, true, &p, false, mode == GBVQC_MODE_JIT));
        if (mode == GBVQC_MODE_JIT) ST_TRY(ensure_jit(p, dtype, true));
    } else {
        mode = GBVQC_MODE_PLAIN;
    }
    if (p && !c->density) {
        ObsDev od;
        ST_TRY(obs_dev_perm(h, p->perm, &od));
    }
    ST_TRY(ensure_workspace(c, dtype));
    Workspace &w = c->ws;
    // a gradient slot per variational physical gate: at most two per op (ket and bra)
    if (!w.d_slot_grad) ST_TRY(dev_alloc(&w.d_slot_grad, (size_t)2 * c->n_param_ops + 1));
    if (p) {
        size_t need = (size_t)p->p.n_slots * (size_t(1) << (c->n_phys - p->p.t));
        if (need > c->partials_cap) {
            free_graphs(c);
            dev_free(w.d_slot_partials);
            w.d_slot_partials = nullptr;
            ST_TRY(dev_alloc(&w.d_slot_partials, std::max<size_t>(need, 1)));
            c->partials_cap = std::max<size_t>(need, 1);
        }
    }
    ST_TRY(stage_theta(c, theta, n_theta, ptr_loc, s));
    if (g_prof) {  // grad_profile: plain stream launches with events
        ST_TRY(enqueue_grad(c, h, dtype, mode, p, s));
        cudaMemcpyKind k = ptr_loc == GBVQC_PTR_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
        CUDA_TRY(cudaMemcpyAsync(energy, w.d_energy, sizeof(double), k, s));
        if (c->n_params > 0) CUDA_TRY(cudaMemcpyAsync(grad_out, w.d_grad, sizeof(double) * c->n_params, k, s));
        CUDA_TRY(cudaStreamSynchronize(s));
        return GBVQC_OK;
    }
    // replay the captured launch sequence
    if ((const void *)h != c->graph_obs) {
        free_graphs(c);
        c->graph_obs = h;
    }
    const int gkey = dtype * 4 + mode;
    auto it = c->graphs.find(gkey);
    if (it == c->graphs.end()) {
        cudaGraph_t graph = nullptr;
        CUDA_TRY(cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
        gbvqc_status st = enqueue_grad(c, h, dtype, mode, p, c->cap_stream);
        cudaError_t e = cudaStreamEndCapture(c->cap_stream, &graph);
        if (st != GBVQC_OK) {
            if (graph) cudaGraphDestroy(graph);
            return st;
        }
        CUDA_TRY(e);
        cudaGraphExec_t exec = nullptr;
        e = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        CUDA_TRY(e);
        it = c->graphs.emplace(gkey, exec).first;
    }
    CUDA_TRY(cudaGraphLaunch(it->second, s));
    cudaMemcpyKind kind = ptr_loc == GBVQC_PTR_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    CUDA_TRY(cudaMemcpyAsync(energy, w.d_energy, sizeof(double), kind, s));
    if (c->n_params > 0) CUDA_TRY(cudaMemcpyAsync(grad_out, w.d_grad, sizeof(double) * c->n_params, kind, s));
    if (ptr_loc == GBVQC_PTR_HOST) CUDA_TRY(cudaStreamSynchronize(s));
    return GBVQC_OK;
}

extern "C" gbvqc_status grad_profile(circuit_handle c, const double *theta, int n_theta, obs_handle h, int dtype,
                                     int mode, void *stream, gbvqc_kernel_stat *stats, int max_stats, int *n_stats)
{
    if (!stats || !n_stats || max_stats < 0) return fail(GBVQC_ERR_ARG, "NULL argument");
    std::vector<ProfRec> recs;
    std::vector<double> g(c ? std::max(c->n_params, 1) : 1);
    double e = 0;
    g_prof = &recs;
    gbvqc_status st = grad(c, theta, n_theta, h, dtype, mode, GBVQC_PTR_HOST, stream, &e, g.data());
    g_prof = nullptr;
    std::vector<gbvqc_kernel_stat> agg;
    for (ProfRec &r : recs) {
        float ms = 0;
        if (st == GBVQC_OK && cudaEventElapsedTime(&ms, r.a, r.b) != cudaSuccess)
            st = fail(GBVQC_ERR_CUDA, "event timing failed");
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
        size_t i = 0;
        while (i < agg.size() && r.name != agg[i].name) i++;
        if (i == agg.size()) {
            gbvqc_kernel_stat k{};
            snprintf(k.name, sizeof k.name, "%s", r.name.c_str());
            agg.push_back(k);
        }
        agg[i].launches++;
        agg[i].ms += ms;
        agg[i].alg_flops += r.flops;
        agg[i].alg_bytes += r.bytes;
    }
    if (st != GBVQC_OK) return st;
    *n_stats = (int)std::min<size_t>(agg.size(), (size_t)max_stats);
    for (int i = 0; i < *n_stats; i++) stats[i] = agg[i];
    return GBVQC_OK;
}
