/*
 * gbvqc.h -- C ABI of the GB300 variational-circuit simulator core (libgbvqc.so).
 *
 * The library applies gates and noise channels to a 2^n complex amplitude vector
 * on one GPU, evaluates Pauli-sum expectation values, and computes exact gradients
 * with the memory-efficient reverse sweep, following JuliVQC (arXiv 2406.19212).
 *
 * Conventions (paper Sec. II.A-B):
 *   - qubits are 0-based; qubit q is bit q of the amplitude index (the paper's
 *     column-major order with its qubit 1 varying fastest);
 *   - a k-qubit matrix acting on the ordered qubits (q_0 .. q_{k-1}) is indexed by
 *     sum_t bit(q_t) 2^t (first listed qubit = least significant bit), and is passed
 *     ROW-MAJOR as interleaved (re, im) doubles: M[row][col] at data[2*(row*2^k+col)];
 *   - a density matrix of n qubits is the 2n-qubit vector |rho>> with rho_ab stored at
 *     index a + 2^n b (ket bits low, bra bits high; Sec. II.A and Sec. III.D);
 *   - amplitudes are interleaved complex: complex64 = {float re, im},
 *     complex128 = {double re, im}, the layout of torch.complex64 / complex128.
 *
 * Errors: every call returns a gbvqc_status; no call throws or aborts.  On failure
 * gbvqc_last_error() returns a message for the calling thread.  A CUDA error inside a
 * call is reported as GBVQC_ERR_CUDA.  No kernel of the library waits on another, so no
 * call has a bounded device wait: GBVQC_ERR_TIMEOUT is reserved and no call returns it.
 *
 * Streams: `stream` arguments are cudaStream_t values passed as void* (NULL = the
 * legacy default stream).  Calls enqueue work on that stream; calls that return a
 * host value (expect, grad with host outputs, sv_get to host) synchronise it.
 */
#ifndef GBVQC_API_H_
#define GBVQC_API_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    GBVQC_OK = 0,
    GBVQC_ERR_ARG = 1,          /* bad handle, size, qubit index or option          */
    GBVQC_ERR_OOM = 2,          /* device allocation failed                         */
    GBVQC_ERR_CUDA = 3,         /* a CUDA runtime call or kernel launch failed      */
    GBVQC_ERR_TIMEOUT = 4,      /* reserved: a bounded device wait ran out (unused)  */
    GBVQC_ERR_NOT_DENSITY = 5,  /* channel applied to a pure state                  */
    GBVQC_ERR_UNSUPPORTED = 6   /* valid request the library does not implement     */
} gbvqc_status;

enum { GBVQC_C64 = 0, GBVQC_C128 = 1 };            /* amplitude dtype                */
enum { GBVQC_MODE_PLAIN = 0,  /* one launch per gate                                     */
       GBVQC_MODE_FUSED = 1,  /* tile passes run by the record interpreter                */
       GBVQC_MODE_JIT = 2     /* tile passes specialised to the circuit: the first call per
                                 circuit, dtype and tiling compiles them (NVRTC, seconds;
                                 cached on disk, see grad), later calls only launch      */
};
enum { GBVQC_PTR_HOST = 0, GBVQC_PTR_DEVICE = 1 };   /* where theta/outputs live      */

/* Operation kinds (paper Sec. II.B).  Rotations: Rx = [[c,-is],[-is,c]],
 * Ry = [[c,-s],[s,c]], Rz = diag(e^{-it/2}, e^{it/2}), c = cos(t/2), s = sin(t/2).
 * SX/SY/SW = ((1+i)I + (1-i)G)/2 for G = X, Y, W=(X+Y)/sqrt2.  CNOT and CONTROL list
 * (control, target).  FSIM takes params (theta, phi, d_plus, d_minus, d_minus_off) as
 * in Eq. (FSIM).  Channels act on one logical qubit of a density matrix:
 * DEPOL(p): K0 = sqrt(1-3p/4) I, K1..3 = sqrt(p/4) X, Y, Z;  AMPDAMP(g), PHASEDAMP(g)
 * as printed in Sec. II.B;  KRAUS: n_kraus (1..4) 2x2 operators in data[]. */
enum {
    GBVQC_X = 0, GBVQC_Y, GBVQC_Z, GBVQC_H, GBVQC_S, GBVQC_T, GBVQC_SX, GBVQC_SY,
    GBVQC_SW, GBVQC_RX, GBVQC_RY, GBVQC_RZ, GBVQC_CNOT, GBVQC_CZ, GBVQC_SWAP,
    GBVQC_ISWAP, GBVQC_FSIM, GBVQC_CONTROL, GBVQC_DENSE1, GBVQC_DENSE2,
    GBVQC_DEPOL, GBVQC_AMPDAMP, GBVQC_PHASEDAMP, GBVQC_KRAUS,
    GBVQC_DEPOL2,          /* two-qubit depolarising: sqrt(1 - 15p/16) I and sqrt(p/16) for
                              the 15 other two-qubit Paulis, i.e. (1-p) rho + p/4 Tr(rho) I */
    GBVQC_KRAUS2,          /* two-qubit QuantumMap: n_kraus 4x4 operators in `kraus`      */
    GBVQC_NUM_KINDS
};

/* One circuit element (QuantumGate / QuantumMap, Sec. II.B-C). */
typedef struct gbvqc_op {
    int32_t kind;          /* GBVQC_X .. GBVQC_KRAUS                                    */
    int32_t qubits[2];     /* logical qubits; qubits[1] unused for one-qubit kinds      */
    int32_t param_index;   /* RX/RY/RZ: index into theta (the paper's isparas=true);
                              -1 = fixed angle params[0].  FSIM: index of the first
                              variational parameter (see param_mask).  Must be -1 for
                              other kinds.                                              */
    int32_t n_kraus;       /* KRAUS only: number of 2x2 operators in data (1..4)        */
    int32_t param_mask;    /* FSIM with param_index >= 0: bit k set
                              = parameter k of (theta, phi, d_plus, d_minus, d_minus_off)
                              is variational (the paper's isparas array, Sec. II.B); the
                              variational ones read theta[param_index], [param_index + 1],
                              ... in increasing k, the others params[k].  Ignored by
                              other kinds.                                              */
    double  params[5];     /* fixed angle / FSIM angles / channel strength              */
    double  data[32];      /* DENSE1 (2x2), DENSE2 (4x4), CONTROL (2x2 target block),
                              KRAUS (n_kraus 2x2 blocks): row-major (re, im) pairs      */
    const double *kraus;   /* KRAUS2 only: n_kraus (1..16) 4x4 operators, row-major (re, im)
                              pairs, 32 doubles each, host memory, copied by
                              circuit_create; NULL for every other kind                 */
} gbvqc_op;

/* One Pauli term coeff * P (Sec. II.E, QubitsTerm): qubit q carries X if only bit q of
 * x_mask is set, Z if only bit q of z_mask, Y if both (Y = i X Z), I if neither. */
typedef struct gbvqc_pauli {
    double   coeff;
    uint64_t x_mask;
    uint64_t z_mask;
} gbvqc_pauli;

typedef struct gbvqc_sv *sv_handle;
typedef struct gbvqc_circuit *circuit_handle;
typedef struct gbvqc_obs *obs_handle;

/* Message describing the last failure on the calling thread ("" if none). */
const char *gbvqc_last_error(void);
/* Library version: major*10000 + minor*100 + patch. */
int gbvqc_version(void);

/* The library's own device memory (a diagnostic, not a paper operation): bytes it holds
 * now (states, plans, work buffers, scratch of handles) and the number of device
 * allocations it has made since the process started (either pointer may be NULL).  Every
 * allocation of the library is counted; memory of sv_wrap'ed states is the caller's and
 * is not.  The environment variable GBVQC_DEVICE_ALLOC_LIMIT (read once, a byte count)
 * caps the live bytes: a request that would exceed it fails with GBVQC_ERR_OOM as a
 * failed cudaMalloc does (host-side fault injection).  Never fails. */
gbvqc_status gbvqc_mem_info(int64_t *live_bytes, int64_t *allocations);

/* ---------------------------------------------------------------- states (Sec. II.A) */

/* Allocate a state of n_qubits logical qubits (a density matrix holds 2^(2n) amplitudes)
 * in device memory owned by the library, initialised to |0...0> (or |0..0><0..0|,
 * Listing 1).  dtype GBVQC_C64 or GBVQC_C128.  1 <= n (2n for density) <= 34.
 * Errors: ERR_ARG, ERR_OOM, ERR_CUDA.  Free with sv_free. */
gbvqc_status sv_alloc(int n_qubits, int dtype, int is_density, void *stream, sv_handle *out);

/* Wrap caller-owned device memory (e.g. a torch tensor's data_ptr) of 2^n (or 2^(2n))
 * amplitudes; the library never frees it.  The pointer must be 16-byte aligned. */
gbvqc_status sv_wrap(void *device_ptr, int n_qubits, int dtype, int is_density, void *stream,
                     sv_handle *out);

/* Release a handle (and its memory if the library allocated it).  NULL is accepted. */
gbvqc_status sv_free(sv_handle sv);

/* Reset to |0...0> (density: |0><0|). */
gbvqc_status sv_reset(sv_handle sv);

/* Copy n_amps amplitudes (must equal the state size) from src, in the state's dtype,
 * from host (src_is_host = 1) or device memory (StateVector(T, data), Listing 1). */
gbvqc_status sv_set(sv_handle sv, const void *src, size_t n_amps, int src_is_host);

/* Copy the amplitudes out to host (dst_is_host = 1) or device memory; synchronous. */
gbvqc_status sv_get(sv_handle sv, void *dst, size_t n_amps, int dst_is_host);

/* Query a state: logical qubits, dtype, density flag, device pointer (any may be NULL). */
gbvqc_status sv_info(sv_handle sv, int *n_qubits, int *dtype, int *is_density, void **device_ptr);

/* ------------------------------------------------------------- circuits (Sec. II.C) */

/* Build a circuit over n_qubits logical qubits from n_ops operations (copied; the caller
 * keeps ownership of ops).  n_params = length of the theta vectors passed later; every
 * param_index must lie in [0, n_params) (a variational FSIM: all of its parameter
 * indices).  is_density = 1 allows channels and makes every unitary act as U rho U^dag
 * (Sec. III.D).  Builds and caches the execution plans (per-gate records and the fused
 * tile schedule).  Errors: ERR_ARG (bad kind, qubit, param index, FSIM param_mask outside
 * [1, 31], Kraus count), ERR_NOT_DENSITY (channel with is_density = 0). */
gbvqc_status circuit_create(const gbvqc_op *ops, int n_ops, int n_qubits, int n_params,
                            int is_density, circuit_handle *out);
gbvqc_status circuit_free(circuit_handle c);

/* Tile-engine options: tile_qubits in [6, 13] (0 = autotune/default) and the number of
 * contiguous low qubits every tile keeps for coalescing, low_qubits in [1, 6] (0 = default).
 * Replaces the cached fused schedule. */
gbvqc_status circuit_set_tiling(circuit_handle c, int tile_qubits, int low_qubits);

/* Autotuner: time `grad` (fused mode, dtype) on this circuit for tile sizes 8..12 (within
 * the kernel's limits) and 2..4 contiguous low qubits, keep the fastest tiling in the
 * circuit (as circuit_set_tiling would), and return it with its time per evaluation.
 * Results are cached on disk, keyed by the circuit's structure, dtype and GPU name, in
 * the file named by the environment variable GBVQC_TUNE_CACHE (default
 * $HOME/.cache/gbvqc/autotune.txt; set it to "off" to disable); a cached circuit is not
 * re-timed (*best_ms is then the cached time).  theta (host) only feeds the timing runs. */
gbvqc_status circuit_autotune(circuit_handle c, const double *theta, int n_theta, obs_handle h, int dtype,
                              void *stream, int *best_tile, int *best_low, double *best_ms);

/* Specialise the fused tile passes of the circuit to its structure (GBVQC_MODE_JIT) ahead
 * of time: generate the CUDA source of every pass of the plan for dtype (the gradient plan
 * and both sweeps with for_grad = 1, else the forward passes of apply_circuit's plan) and
 * compile it with NVRTC for sm_103a into the on-disk cache, so that the first JIT-mode call
 * only loads the modules.  Host only: needs no GPU.  The cache is the directory named by
 * GBVQC_JIT_CACHE (default $HOME/.cache/gbvqc/jit; "off" disables it, and then this call
 * only checks that the sources compile).  *n_kernels = passes specialised, *n_cached = of
 * them found in the cache, *seconds = compile wall time (any pointer may be NULL).
 * Errors: ERR_ARG; ERR_UNSUPPORTED (too few qubits for tiles); ERR_CUDA if NVRTC cannot be
 * loaded or a source fails to compile (the message carries NVRTC's log). */
gbvqc_status circuit_specialize(circuit_handle c, int dtype, int for_grad, int *n_kernels, int *n_cached,
                                double *seconds);

/* Report the fused schedule: number of tile passes and of gate records it holds. */
gbvqc_status circuit_plan_info(circuit_handle c, int *n_passes, int *n_gates, int *tile_qubits);

/* Host-only statistics of the fused schedule for dtype (the reverse layout of grad if
 * for_grad = 1); needs no GPU.  stats[0..9] = tile qubits, passes, forward sub-runs,
 * forward gate records, forward phase blocks, reverse sub-runs, gradient slots,
 * largest per-pass shared memory in bytes (forward, reverse), gates in the circuit's
 * physical gate list.  Fills min(n_stats, 10) entries. */
gbvqc_status circuit_plan_stats(circuit_handle c, int dtype, int for_grad, int64_t *stats, int n_stats);

/* Kernel structure the library uses for a one- or two-qubit matrix (a diagnostic query:
 * host only, needs no GPU).  matrix: dim x dim complex entries, row-major, interleaved
 * (re, im) doubles, dim 2 or 4 (first qubit = matrix bit 0).  *shape receives one of the
 * GBVQC_SHAPE_* codes: which sweep a gate or a one-qubit channel's superoperator takes
 * (exact zeros, ones and real parts decide; no tolerance).  Errors: ERR_ARG (NULL
 * pointer, dim not 2 or 4). */
enum {
    GBVQC_SHAPE_DENSE1 = 0,  /* general 2x2 */
    GBVQC_SHAPE_DIAG1 = 1,   /* diagonal 2x2 */
    GBVQC_SHAPE_ANTI1 = 2,   /* anti-diagonal 2x2 */
    GBVQC_SHAPE_REAL1 = 3,   /* real 2x2 */
    GBVQC_SHAPE_DENSE2 = 4,  /* general 4x4 */
    GBVQC_SHAPE_DIAG2 = 5,   /* diagonal 4x4 */
    GBVQC_SHAPE_PERM2 = 6,   /* one non-zero per row and column */
    GBVQC_SHAPE_CTRL2 = 7,   /* identity unless the first qubit is 1 */
    GBVQC_SHAPE_BLOCK2 = 8,  /* phases on |00>, |11> and a 2x2 on |01>, |10> (FSIM) */
    GBVQC_SHAPE_IMAG1 = 9,   /* real diagonal, imaginary off-diagonal 2x2 (Rx) */
    GBVQC_SHAPE_PAR2 = 11,   /* a 2x2 on |00>, |11> and a 2x2 on |01>, |10> */
    GBVQC_SHAPE_RPAR2 = 12,  /* the same with real entries */
    GBVQC_SHAPE_CX = 13,     /* exactly CNOT, the first qubit the control */
    GBVQC_SHAPE_CZ = 14      /* exactly CZ */
};
gbvqc_status gate_shape(const double *matrix, int dim, int *shape);

/* ------------------------------------------------------------ execution (Sec. II.D) */

/* psi <- C(theta) psi in place (apply!, Eq. circuitevolve; Eq. channel for density
 * states).  theta: n_theta doubles on host or device (theta_loc).  mode PLAIN runs one
 * kernel per gate (Eq. 3 / Eq. twoqubitgate); FUSED runs the tile passes.  The state's
 * qubit count and density flag must match the circuit's.  Enqueued on the state's
 * stream; returns without synchronising. */
gbvqc_status apply_circuit(sv_handle sv, circuit_handle c, const double *theta, int n_theta,
                           int theta_loc, int mode);

/* Apply one single-qubit channel (Sec. II.B, Eq. channel / channel2) to a density state:
 * kind GBVQC_DEPOL / AMPDAMP / PHASEDAMP with strength, or GBVQC_KRAUS with n_kraus 2x2
 * operators in kraus (row-major (re,im), host memory).  Pure state: ERR_NOT_DENSITY. */
gbvqc_status apply_channel(sv_handle sv, int kind, int qubit, double strength,
                           const double *kraus, int n_kraus);

/* measure!(state, qubit) of Sec. II.D (Listing 4): measures one qubit and collapses the
 * state in place.  P(k) = w_k / (w_0 + w_1) with w_k the FP64 sum of |psi_a|^2 (pure) or
 * rho_aa (density) over the indices a whose bit `qubit` is k.  The random draw is the
 * caller's: u must lie in [0, 1); the outcome is 0 if u < P(0), else 1.  The state is
 * projected on the outcome and renormalised (pure: divided by sqrt(w_k); density:
 * P rho P divided by w_k).  Writes *outcome and *prob (its probability, host memory).
 * Synchronises the state's stream before returning the outcome; the collapse is then
 * enqueued on that stream.  Errors: ERR_ARG for a NULL pointer, qubit outside
 * [0, n_qubits), u outside [0, 1) or a state of zero norm; ERR_CUDA if a launch fails. */
gbvqc_status measure(sv_handle sv, int qubit, double u, int *outcome, double *prob);

/* Sampling: measurement of every qubit on n_shots fresh copies of the state (the state is
 * not changed).  With weights w_a = |psi_a|^2 (pure) or rho_aa (density) and their total
 * W, shot s returns in out[s] the least basis index a with u[s] W < w_0 + ... + w_a (FP64
 * partial sums over chunks of the index range, then within the chunk).  u: n_shots
 * uniform draws in [0, 1) (host), out: n_shots int64 (host).  Synchronises the state's
 * stream; allocates and frees scratch of about 2^(n-cbits) doubles.  Errors: ERR_ARG for
 * NULL pointers or u outside [0, 1); ERR_OOM; ERR_CUDA. */
gbvqc_status sample(sv_handle sv, const double *u, int n_shots, int64_t *out);

/* ---------------------------------------------------------- observables (Sec. II.E) */

/* Pauli sum H = sum_t terms[t].coeff P_t over n_qubits logical qubits (QubitsOperator).
 * Terms are copied to the device; masks must not touch qubits >= n_qubits. */
gbvqc_status obs_create(const gbvqc_pauli *terms, int n_terms, int n_qubits, obs_handle *out);
gbvqc_status obs_free(obs_handle h);

/* <psi|H|psi> (pure) or tr(H rho) (density), reduced in FP64 (expectation, Sec. II.E;
 * Eq. loss_mixed).  Synchronises the state's stream and writes *out_energy (host). */
gbvqc_status expect(sv_handle sv, obs_handle h, double *out_energy);

/* ------------------------------------------------------ gradients (Sec. III.C, III.E) */

/* Energy L(theta) = <0|C^dag H C|0> (Eq. loss_pure) or <<I|H C|0>> (Eq. loss_mixed) and
 * its exact gradient dL/dtheta (n_params values; gates sharing a parameter add up) by
 * the reverse sweep of Algorithm 2: two live states, no checkpoints.  dtype selects
 * complex64 sweeps (FP64 reductions) or complex128.  mode PLAIN = per-gate kernels;
 * FUSED = tile passes.  ptr_loc says whether theta, energy and grad_out are host or
 * device pointers; with host pointers the call synchronises `stream`.  Work buffers are
 * cached in the circuit handle (one grad call per circuit handle at a time).
 * Errors: ERR_ARG, ERR_OOM, ERR_CUDA. */
gbvqc_status grad(circuit_handle c, const double *theta, int n_theta, obs_handle h,
                  int dtype, int mode, int ptr_loc, void *stream, double *energy,
                  double *grad_out);

/* Per-kernel timing of one gradient evaluation.  Runs the same launch sequence as grad
 * (host theta), without graph replay, with CUDA events around every launch on `stream`,
 * and aggregates by kernel name: launches, total milliseconds, and the algorithmic
 * floating-point operations and bytes those launches must perform (flops: complex
 * arithmetic of the applied matrices and generator inner products over 2^n amplitudes;
 * bytes: one read and one write of every state a launch sweeps).  Fills at most
 * max_stats entries and sets *n_stats.  Synchronises `stream`. */
typedef struct gbvqc_kernel_stat {
    char   name[32];
    int    launches;
    double ms;
    double alg_flops;
    double alg_bytes;
} gbvqc_kernel_stat;

gbvqc_status grad_profile(circuit_handle c, const double *theta, int n_theta, obs_handle h,
                          int dtype, int mode, void *stream, gbvqc_kernel_stat *stats,
                          int max_stats, int *n_stats);

/* ------------------------------------------------ batched gradients (many circuits) */

typedef struct gbvqc_batch *batch_handle;

/* A batch of independent pure-state circuits (each with its own qubit count >= 6, gates,
 * parameters and observable) evaluated together: every step of the gradient sequence
 * (materialisation, state init, fused pass p of every circuit, expectation, reverse
 * pass p, gradient reduction) is one launch over all circuits, and the whole sequence
 * is captured once into a CUDA graph that batch_grad replays.  dtype GBVQC_C64 (FP32
 * sweeps, FP64 reductions) or GBVQC_C128.  The batch keeps pointers to the circuit and
 * observable handles: free the batch before them, and do not run the member circuits
 * elsewhere while batch_grad runs (they share matrix records).  Work buffers: two states
 * per circuit plus per-slot partials, owned by the batch.
 * Errors: ERR_ARG (NULL, empty batch, density circuit, observable/circuit qubit
 * mismatch), ERR_UNSUPPORTED (fewer than 6 qubits), ERR_OOM, ERR_CUDA. */
gbvqc_status batch_create(const circuit_handle *circuits, const obs_handle *observables, int n_circuits,
                          int dtype, batch_handle *out);
gbvqc_status batch_free(batch_handle b);

/* Energies (one per circuit) and gradients (concatenated in circuit order, n_params of
 * each) for theta_all (all circuits' parameters concatenated, n_theta_total values).
 * ptr_loc: theta_all, energies and grads are host or device pointers; host pointers
 * synchronise `stream`. */
gbvqc_status batch_grad(batch_handle b, const double *theta_all, int n_theta_total, int ptr_loc,
                        void *stream, double *energies, double *grads);

/* Autotuner of a batch: times batch_grad (theta_all on the host, n_theta_total values)
 * with every member's tile size set to T = 8 .. 12 (clamped to the member's qubit count),
 * then, for the four qubit-count classes holding the most amplitudes, each T for that
 * class alone; keeps the fastest assignment (set on the member circuits, as
 * circuit_set_tiling would, and the batch rebuilt) and returns the members' tile sizes in
 * tiles[0 .. n_circuits) (may be NULL) and its time per batch_grad in *best_ms.  Takes
 * up to about 25 batch rebuilds and four timed calls each.  Errors: those of batch_grad. */
gbvqc_status batch_autotune(batch_handle b, const double *theta_all, int n_theta_total, void *stream, int *tiles,
                            double *best_ms);

/* One-shot convenience: batch_create (complex64), batch_grad with host pointers,
 * batch_free. */
gbvqc_status grad_batch(const circuit_handle *circuits, const obs_handle *observables,
                        int n_circuits, const double *theta_all, void *stream,
                        double *energies, double *grads);

/* ------------------------------------------- sharded states with qubit-swap exchange */

/* A pure state of n_qubits split into 2^n_global shards by its n_global global qubits
 * (the standard partition of a state over devices, each shard holding 2^(n - n_global)
 * amplitudes; the paper simulates beyond one device with distributed simulators,
 * Introduction).  Gates on local qubits act on every shard alone; diagonal gates on
 * global qubits become per-shard phases or one-qubit diagonals on the local partner;
 * any other gate on a global qubit is preceded by a qubit swap that trades its position
 * with a local qubit's, exchanging half of every shard with its partner shard.  In this
 * library the shards are buffers on the calling thread's current GPU and the exchange a
 * swap kernel between them (one GPU per process); the schedule is the one a multi-device
 * run would execute. */
typedef struct gbvqc_sharded *sharded_handle;

/* The exchange schedule of a pure circuit for n_global global qubits (host only, no GPU):
 * steps[3 i .. 3 i + 2] = {0, op_begin, op_end} (apply ops [op_begin, op_end) of the
 * circuit on every shard) or {1, j, l} (swap global qubit position j with local qubit
 * position l).  Positions start as the identity (qubit q at position q; positions
 * >= n - n_global are global, bit position - (n - n_global) of the shard index).  The
 * local qubit given up is the one whose next non-diagonal use is farthest away.  Fills
 * min(max_steps, total) steps, sets *n_steps = total and *n_swaps (may be NULL).
 * Errors: ERR_ARG (NULL, n_global outside [1, n - 2]), ERR_UNSUPPORTED (density circuit). */
gbvqc_status shard_plan(circuit_handle c, int n_global, int32_t *steps, int max_steps, int *n_steps, int *n_swaps);

/* A sharded state |0...0> of n_qubits (3 .. 34) with n_global (1 .. 10, leaving at least
 * two local qubits) global qubits, dtype GBVQC_C64 / GBVQC_C128.  Errors: ERR_ARG,
 * ERR_OOM, ERR_CUDA. */
gbvqc_status sharded_alloc(int n_qubits, int n_global, int dtype, sharded_handle *out);
gbvqc_status sharded_free(sharded_handle h);

/* Copy the full state (2^n amplitudes in the logical order, index bit q = qubit q, host
 * memory) into / out of the shards, through the state's current qubit positions.
 * Synchronous. */
gbvqc_status sharded_set(sharded_handle h, const void *host_src);
gbvqc_status sharded_get(sharded_handle h, void *host_dst);

/* psi <- C(theta) psi for a pure circuit of the same qubit count (theta on the host): the
 * exchange schedule from the state's current positions, local segments run as tile passes
 * on every shard (per-gate kernels below 6 local qubits), exchanges between the shard
 * pairs.  The positions the schedule leaves are kept (sharded_get reads through them).
 * Synchronous.  Errors: ERR_ARG, ERR_UNSUPPORTED (density circuit), ERR_OOM, ERR_CUDA. */
gbvqc_status sharded_apply(sharded_handle h, circuit_handle c, const double *theta, int n_theta);

/* The current position of every qubit (n_qubits entries), and the exchanges made so far
 * (shard-pair swaps) with their bytes moved (each pair swaps half of both shards); any
 * pointer may be NULL. */
gbvqc_status sharded_info(sharded_handle h, int32_t *positions, int64_t *exchanges, int64_t *bytes);

/* ------------------------------------------------------ allocation-free expectation */

/* <psi|H|psi> of a pure state for callers that cannot allocate device memory.  The
 * paper has no counterpart: this exists for code that runs while a stream is being
 * captured into a CUDA graph (where cudaMalloc is refused or unsafe), for applications
 * whose framework owns the device memory budget through its own pool, and for loops
 * that cannot take an allocation's implicit synchronisation.  Unlike `expect`, which
 * reduces through scratch owned by a state handle (sv_alloc / sv_wrap allocate it),
 * this call needs no handle and allocates nothing: it calls no cudaMalloc, cudaFree or
 * allocating library routine.
 *
 * psi_device: 2^n_qubits amplitudes of dtype GBVQC_C64 / GBVQC_C128 in device memory,
 * 16-byte aligned, owned by the caller.  terms: at most 64 Pauli terms in host memory
 * (they are passed to the kernel as parameters).  energy_device: one double in device
 * memory, written by the kernel.  The call only enqueues work on `stream` and returns.
 *
 * Scratch: a fixed 5120-byte array (256-byte arrival counter + 608 FP64 block partials)
 * in the library's device memory, present on every GPU that loads the library until the
 * process exits.  All calls share it: calls whose kernels overlap on the GPU race, so
 * order them on one stream (or with events).  The counter is cleared before every
 * launch.  The first call on a device looks up the array's device address with that
 * device current; make that first call before any stream capture.
 * Errors: ERR_ARG for NULL pointers, a bad dtype or qubit count, a term on a qubit
 * >= n_qubits, or more than 64 terms (the no-allocation maximum); ERR_CUDA if the
 * launch fails. */
gbvqc_status expect_noalloc(const void *psi_device, int n_qubits, int dtype,
                            const gbvqc_pauli *terms, int n_terms, void *stream,
                            double *energy_device);

#ifdef __cplusplus
}
#endif
#endif /* GBVQC_API_H_ */
