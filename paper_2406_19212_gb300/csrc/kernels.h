// Host-side launchers of the CUDA kernels (implemented in kernels_*.cu).
#pragma once

#include "common.cuh"

#ifndef __CUDACC_RTC__  // (runtime compilation: NVRTC's built-in definitions)
#include <cuda_runtime.h>
#include <stdint.h>
#endif

namespace gbvqc {

// Pauli sum on the device, terms grouped by X mask: for group g with mask x_g,
// c_g(b) = sum_{k in g} coeff_k i^{ph_k} (-1)^{popcount(b & z_k)}, and
// (H psi)_a = sum_g c_g(a ^ x_g) psi_{a ^ x_g}.
struct ObsTerm {
    double coeff;
    uint64_t z;
    int32_t ph;   // number of Y factors mod 4
    float coeff_f;  // coeff rounded once to FP32 (complex64 sweeps never convert per amplitude)
};
struct ObsGroup {
    uint64_t x;
    int32_t t_begin, t_end;
};
struct ObsDev {
    const ObsGroup *groups;
    const ObsTerm *terms;
    int n_groups;
    int n_terms;
    const unsigned char *chunk = nullptr;  // staging image of the chunked kernels (chunk_image)
};

// Chunked Pauli-sum kernels (k_pauli_chunk): a CTA of 2^kPauliTB threads stages 2^kPauliC
// amplitudes, kPauliPV per thread (a = hi | r << kPauliTB | thread).  The observable is
// staged from a host-built image: the groups, then the terms in the sweep's precision
// with the group's sign (-1)^{x_g . z} folded into the coefficient (the sign of a term at
// amplitude a ^ x_g is then read from a itself) and rpat = bit r set where the term's
// Z mask has odd overlap with r << kPauliTB.
constexpr int kPauliPV = 4, kPauliTB = 8, kPauliC = 10;
enum : uint32_t { CG_REAL = 1, CG_SELF = 2, CG_CHUNK = 4, CG_CONST = 8 };
struct ChunkGroup {
    uint32_t xlo, xhi;
    uint16_t t_begin, t_end;
    uint32_t flags;  // CG_*: real coefficients, X mask 0, X mask inside the chunk, every Z mask 0
};
struct ChunkTermF {
    uint32_t zlo, zhi, rpat;
    float cr, ci;
    uint32_t pad;
};
struct ChunkTermD {
    uint32_t zlo, zhi, rpat, pad;
    double cr, ci;
};
// Byte offsets in the image: groups (16 * even count), complex64 terms, complex128 terms.
__host__ __device__ inline size_t chunk_terms_f_offset(int n_groups) { return 16 * (size_t)((n_groups + 1) & ~1); }
__host__ __device__ inline size_t chunk_terms_d_offset(int n_groups, int n_terms)
{
    return chunk_terms_f_offset(n_groups) + ((sizeof(ChunkTermF) * (size_t)n_terms + 15) & ~size_t(15));
}
inline size_t chunk_image_bytes(int n_groups, int n_terms)
{
    return chunk_terms_d_offset(n_groups, n_terms) + sizeof(ChunkTermD) * (size_t)n_terms;
}

// Shared memory of the staged observable in the expectation kernels; observables
// larger than kObsStageMax (or with 65536 terms or more) are read from global memory.
constexpr size_t kObsStageMax = 160 * 1024;
inline size_t obs_smem_bytes(const ObsDev &obs, int dtype)
{
    const size_t g = 16 * (size_t)((obs.n_groups + 1) & ~1);
    return g + (size_t)obs.n_terms * (dtype == 0 ? 16 : 24);
}
inline bool obs_stageable(const ObsDev &obs, int dtype)
{
    return obs.n_terms < 65536 && obs_smem_bytes(obs, dtype) <= kObsStageMax;
}
cudaError_t pauli_prepare();  // shared-memory opt-in of the staged kernels, outside capture
cudaError_t pauli_batch_prepare();

// Scratch of a grid reduction: one double per block plus an arrival counter that the
// last block resets to zero.
struct RedScratch {
    double *partials;   // kMaxRedBlocks doubles
    unsigned *counter;  // one counter, zero between launches
};
constexpr int kMaxRedBlocks = 1024;

// ---- per-gate kernels (kernels_plain.cu)
cudaError_t launch_gate(int dtype, void *psi, int n, int shape, int q0, int q1,
                        const MatRec *rec, cudaStream_t s);
cudaError_t launch_zero_state(int dtype, void *psi, int n, cudaStream_t s);
// Qubit-swap exchange between two shards of 2^local_qubits amplitudes (see k_shard_swap).
cudaError_t launch_shard_swap(int dtype, void *a, void *b, int local_qubits, int l, cudaStream_t s);
// Four-qubit gate: psi <- M psi on physical qubits q0..q3 (matrix bits 0..3), M = 16 x 16
// complex in 16 consecutive records (record r = row r).
cudaError_t launch_gate4(int dtype, void *psi, int n, int q0, int q1, int q2, int q3, const MatRec *rows,
                         cudaStream_t s);
cudaError_t launch_materialize(const DynRec *dyn, int n_dyn, const double *theta,
                               MatRec *recs, cudaStream_t s);
cudaError_t launch_accumulate(const double *slot_grad, const int *csr_ptr, const int *csr_slots,
                              int n_params, double *grad, cudaStream_t s);

// ---- reductions (kernels_reduce.cu)
// out[0] = scale * Re sum conj(psi) (D phi), D a 2x2 (k=1) or 4x4 (k=2) on (q0, q1).
cudaError_t launch_dot_matrix(int dtype, const void *psi, const void *phi, int n, int k,
                              int q0, int q1, const MatRec *rec, double scale,
                              RedScratch red, double *out, cudaStream_t s);
// Pure state: out[0] = Re <psi|H|psi>; if lam != nullptr also writes lam = H psi.
cudaError_t launch_pauli_expect(int dtype, const void *psi, void *lam, int n, ObsDev obs,
                                RedScratch red, double *out, cudaStream_t s);
// Physical layout of a density matrix of n logical qubits: ket bit q of rho_ab sits at
// physical bit ket[q], bra bit q at bra[q] (standard layout: ket[q] = q, bra[q] = q + n).
struct DensMap {
    int8_t ket[32];
    int8_t bra[32];
};
// out[0] = Re tr(H rho).
cudaError_t launch_density_expect(int dtype, const void *rho, int n, DensMap map, ObsDev obs,
                                  RedScratch red, double *out, cudaStream_t s);
// Density adjoint seed psi = vec(H) (psi_ab = H_ab) in the layout `map`; the whole
// vector is written (zeros off the Pauli support).
// measure!: out[k] = weight of outcome k of qubit q (FP64, fixed order; scratch holds
// 2 * max_blocks doubles), and the projection + renormalisation on outcome k.
cudaError_t launch_measure_sums(int dtype, const void *st, int n, int density, int q, double *scratch,
                                int max_blocks, double *out, cudaStream_t s);
cudaError_t launch_collapse(int dtype, void *st, int n, int density, int q, int k, double scale,
                            cudaStream_t s);
// Sampling: chunk sums (2^(n - cbits) doubles), their inclusive prefix, then out[s] = the
// least index a with u[s] * total < w_0 + ... + w_a (device buffers; 5 <= cbits <= n).
cudaError_t launch_sample(int dtype, const void *st, int n, int density, int cbits, double *chunk_sum,
                          double *incl, const double *u, int n_shots, int64_t *out, cudaStream_t s);
cudaError_t launch_density_seed(int dtype, void *psi, int n, DensMap map, ObsDev obs,
                                cudaStream_t s);

// ---- fused tile passes (kernels_fused.cu)
// Device arrays of one direction (forward or reverse) of a fused plan.
struct FusedDev {
    const PassDesc *passes;
    const SubRun *subs;
    const FGate *gates;
    const DEnt *ents;
    const MatUnit *units;
    const MatRec *recs;
    const void *img;  // matrix image (8 reals per unit, unit order) or null
};
// Arguments of one tile pass of one circuit.
struct FusedArgs {
    const PassDesc *pd;
    const SubRun *subs;
    const FGate *gates;
    const DEnt *ents;
    const MatUnit *units;
    const MatRec *recs;
    const void *img;  // 8 reals of every unit in unit order (the staged matrices of pass p
                      // are one contiguous run), or null to gather them through units/recs
    double *slot_partials;
    int tiles_stride;
    int dry;  // 1: a code-prefetch launch (specialised passes): runs tile 0 of the pass and
              // writes nothing to global memory; it only pulls the kernel's instructions
              // into L2 ahead of the pass's real launch
    int init;  // 1 (first forward pass of a gradient): the pass starts from |0...0> instead of
               // reading phi.  Tile 0 holds the one nonzero amplitude and runs the gates;
               // every other tile stays zero under the pass's linear maps and is written as
               // zeros without running them.
};
// img_f / img_r [8 u + e] = element e of unit u of the forward / reverse unit list, in the
// state's precision (after the step's matrices are materialised).
struct GatherArgs {
    const MatUnit *fu;          // forward unit list (nf units) -> img_f
    int nf;
    const MatUnit *ru;          // reverse unit list (nr units) -> img_r
    int nr;
    void *img_f, *img_r;
    const MatRec *recs;
    const TabDesc *ftabs, *rtabs;   // register phase tables written into img_f / img_r
    const TabEnt *ftabents, *rtabents;
    int n_ftabs, n_rtabs, fbits, rbits;
};
// Items of a plan's image (one thread each).
inline __host__ __device__ int64_t gather_items(const GatherArgs &g)
{
    return 8 * (int64_t)(g.nf + g.nr) + ((int64_t)g.n_ftabs << g.fbits) + ((int64_t)g.n_rtabs << g.rbits);
}
cudaError_t launch_gather_units(int dtype, const GatherArgs &g, cudaStream_t s);
// The same for n plans at once (batched gradients): args[k] of plan k, item_off[k] its
// first item (8 per unit, one per table entry), item_off[n] = total items.
cudaError_t launch_gather_batch(int dtype, const GatherArgs *args, const int64_t *item_off, int n, int64_t total,
                                cudaStream_t s);
int fused_nr(int dtype, bool reverse);           // register qubits per sub-run
// Threads per CTA the fused kernels are compiled for (launch bounds): 2^(t - NR) must
// not exceed it.  Two CTAs per SM for the reverse kernels, three for the forward ones.
constexpr int fused_max_threads(int nr, bool reverse) { return reverse && nr < 5 ? 256 : 128; }
constexpr int fused_min_blocks(bool reverse) { return reverse ? 2 : 3; }
cudaError_t fused_prepare();                     // shared-memory opt-in, outside capture
// init: the pass starts from |0...0> and writes psi without reading it (FusedArgs::init).
cudaError_t launch_fused_forward(int dtype, void *psi, const FusedDev &fd, int pass,
                                 const PassDesc &pass_host, size_t smem, cudaStream_t s, bool init = false);
cudaError_t launch_fused_reverse(int dtype, void *phi, void *psi, const FusedDev &fd, int pass,
                                 const PassDesc &pass_host, size_t smem, double *slot_partials,
                                 int n_tiles_stride, cudaStream_t s);
// grad[p] = sum over slots[ptr[p] .. ptr[p+1]) of sum_tile slot_partials[slot * stride + tile]
// (tiles and slots in index order, one fixed reduction tree per slot).
cudaError_t launch_reduce_grad(const double *slot_partials, int n_tiles, int stride, const int *csr_ptr,
                               const int *csr_slots, int n_params, double *grad, cudaStream_t s);

// ---- batched kernels (kernels_batch.cu): one launch covers many circuits; CTA c
// belongs to the last entry whose `begin` is <= c.
struct FusedBatchEntry {
    FusedArgs args;
    void *phi, *psi;
    int64_t begin;           // first CTA (tile) of this circuit in the launch
};
constexpr int kPauliChunkBits = 12;  // amplitudes per CTA of the batched expectation
struct PauliBatchEntry {
    const void *psi;
    void *lam;
    ObsDev obs;
    double *partials;        // one per chunk
    int n;                   // qubits
    int pad;
    int64_t begin;           // first CTA (chunk)
};
struct SlotBatchEntry {
    const double *partials;  // [slot][tile]
    int n_tiles;
    int pad;
    int64_t begin;           // first global slot of this circuit
};
struct BatchDyn {            // theta-dependent record of a batch member
    MatRec *rec;
    int theta_index;         // into the concatenated parameter vector
    int pad;
    DynRec r;                // the member's record description (r.param unused)
};
cudaError_t fused_batch_prepare();
cudaError_t launch_fused_batch(int dtype, bool reverse, bool two_q, int t, const FusedBatchEntry *entries,
                               int n_entries, int64_t total_tiles, size_t smem, cudaStream_t s);
// smem: the largest obs_smem_bytes of the batch, or 0 to read every observable from
// global memory.
cudaError_t launch_pauli_batch(int dtype, const PauliBatchEntry *entries, int n_entries, int64_t total_chunks,
                               size_t smem, double *energies, cudaStream_t s);
cudaError_t launch_slots_batch(const SlotBatchEntry *entries, int n_entries, int64_t total_slots,
                               double *slot_grad, cudaStream_t s);
// Materialise the batch's rotation records and, with zero_states, set every instance to
// |0...0> (without it the first forward passes write the initial states: FusedArgs::init).
cudaError_t launch_batch_init(const BatchDyn *dyn, int n_dyn, const double *theta, int dtype, void *phi_all,
                              size_t phi_bytes, const int64_t *offsets, int n_inst, cudaStream_t s,
                              bool zero_states = true);

}  // namespace gbvqc
