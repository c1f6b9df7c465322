// Device helpers of Pauli-sum observables (shared by the single and batched kernels).
#pragma once

#include "kernels.h"

namespace gbvqc {

// c_g(b) = sum_{k in g} coeff_k i^{ph_k} (-1)^{popcount(b & z_k)}
template <typename R>
__device__ __forceinline__ void group_coeff(const ObsTerm *__restrict__ terms, int t0, int t1,
                                            uint64_t b, R &cr, R &ci)
{
    cr = 0;
    ci = 0;
    for (int k = t0; k < t1; k++) {
        const ObsTerm t = terms[k];
        R c;
        if constexpr (sizeof(R) == 4) c = t.coeff_f;
        else c = t.coeff;
        if (__popcll(b & t.z) & 1) c = -c;
        switch (t.ph & 3) {
        case 0: cr += c; break;
        case 1: ci += c; break;
        case 2: cr -= c; break;
        default: ci -= c; break;
        }
    }
}

// (H psi)_a = sum_g c_g(a ^ x_g) psi_{a ^ x_g} for one amplitude index a.
template <typename R, typename T>
__device__ __forceinline__ void pauli_apply_amp(const T *__restrict__ psi, uint64_t a, const T pa, const ObsDev &obs,
                                                R &lr, R &li)
{
    lr = 0;
    li = 0;
    for (int g = 0; g < obs.n_groups; g++) {
        const ObsGroup gr = obs.groups[g];
        const uint64_t b = a ^ gr.x;
        const T pb = gr.x ? psi[b] : pa;
        R cr, ci;
        group_coeff<R>(obs.terms, gr.t_begin, gr.t_end, b, cr, ci);
        lr += cr * pb.x - ci * pb.y;
        li += cr * pb.y + ci * pb.x;
    }
}

// Compact form of a Pauli sum staged in shared memory by the expectation kernels: per
// term the Z mask halves and coeff * i^{ph} in the sweep's precision; per group the X
// mask halves, the term range and whether every term of the group is real.  The
// per-term work is then an AND (two for more than 32 qubits), a popcount whose low bit
// flips the sign bit of the coefficient, and one or two adds.
template <typename R>
struct PTerm {
    uint32_t zlo, zhi;
    R cr, ci;
};
struct PGroup {
    uint32_t xlo, xhi;
    uint16_t t_begin, t_end;
    uint32_t real;
};

__device__ __forceinline__ float sign_flip(float c, uint32_t p)
{
    return __int_as_float(__float_as_int(c) ^ (int)(p << 31));
}
__device__ __forceinline__ double sign_flip(double c, uint32_t p)
{
    return __hiloint2double(__double2hiint(c) ^ (int)(p << 31), __double2loint(c));
}

// Stage obs into shared memory (sg: obs.n_groups rounded up to even, then the terms);
// returns after a __syncthreads.
template <typename R>
__device__ __forceinline__ void stage_obs(const ObsDev &obs, unsigned char *smem, const PGroup *&sg,
                                          const PTerm<R> *&st)
{
    PGroup *g_out = reinterpret_cast<PGroup *>(smem);
    PTerm<R> *t_out = reinterpret_cast<PTerm<R> *>(smem + sizeof(PGroup) * ((obs.n_groups + 1) & ~1));
    for (int k = threadIdx.x; k < obs.n_terms; k += blockDim.x) {
        const ObsTerm t = obs.terms[k];
        R c;
        if constexpr (sizeof(R) == 4) c = t.coeff_f;
        else c = t.coeff;
        const int ph = t.ph & 3;
        PTerm<R> p;
        p.zlo = (uint32_t)t.z;
        p.zhi = (uint32_t)(t.z >> 32);
        p.cr = ph == 0 ? c : ph == 2 ? -c : R(0);
        p.ci = ph == 1 ? c : ph == 3 ? -c : R(0);
        t_out[k] = p;
    }
    for (int g = threadIdx.x; g < obs.n_groups; g += blockDim.x) {
        const ObsGroup gr = obs.groups[g];
        uint32_t real = 1;
        for (int k = gr.t_begin; k < gr.t_end; k++) real &= (obs.terms[k].ph & 1) == 0;
        g_out[g] = PGroup{(uint32_t)gr.x, (uint32_t)(gr.x >> 32), (uint16_t)gr.t_begin, (uint16_t)gr.t_end, real};
    }
    __syncthreads();
    sg = g_out;
    st = t_out;
}

// (H psi)_a for V amplitudes a[0..V) at once from the staged form (WIDE: more than 32
// qubits).  Groups run in the outer loop so the V partner loads of a group are in
// flight together and every staged term is read once per V amplitudes.  Entries with
// ok[j] false are left at zero and read nothing.
template <typename R, bool WIDE, int V, typename T>
__device__ __forceinline__ void pauli_apply_staged(const T *__restrict__ psi, const uint64_t (&a)[V],
                                                   const bool (&ok)[V], const T (&pa)[V], const PGroup *sg,
                                                   const PTerm<R> *st, int n_groups, R (&lr)[V], R (&li)[V])
{
#pragma unroll
    for (int j = 0; j < V; j++) lr[j] = li[j] = 0;
    for (int g = 0; g < n_groups; g++) {
        const PGroup gr = sg[g];
        const bool flipped = WIDE ? (gr.xlo | gr.xhi) != 0 : gr.xlo != 0;
        uint32_t blo[V], bhi[V];
        T pb[V];
#pragma unroll
        for (int j = 0; j < V; j++) {
            blo[j] = (uint32_t)a[j] ^ gr.xlo;
            bhi[j] = WIDE ? (uint32_t)(a[j] >> 32) ^ gr.xhi : 0u;
            pb[j] = pa[j];
            if (flipped && ok[j]) pb[j] = psi[WIDE ? (((uint64_t)bhi[j] << 32) | blo[j]) : (uint64_t)blo[j]];
        }
        R cr[V], ci[V];
#pragma unroll
        for (int j = 0; j < V; j++) cr[j] = ci[j] = 0;
        if (gr.real) {
            for (int k = gr.t_begin; k < gr.t_end; k++) {
                const uint32_t zl = st[k].zlo, zh = WIDE ? st[k].zhi : 0u;
                const R c = st[k].cr;
#pragma unroll
                for (int j = 0; j < V; j++) {
                    const uint32_t m = WIDE ? (blo[j] & zl) ^ (bhi[j] & zh) : blo[j] & zl;
                    cr[j] += sign_flip(c, __popc(m));
                }
            }
#pragma unroll
            for (int j = 0; j < V; j++) {
                lr[j] += cr[j] * pb[j].x;
                li[j] += cr[j] * pb[j].y;
            }
        } else {
            for (int k = gr.t_begin; k < gr.t_end; k++) {
                const uint32_t zl = st[k].zlo, zh = WIDE ? st[k].zhi : 0u;
                const R c0 = st[k].cr, c1 = st[k].ci;
#pragma unroll
                for (int j = 0; j < V; j++) {
                    const uint32_t m = WIDE ? (blo[j] & zl) ^ (bhi[j] & zh) : blo[j] & zl;
                    const uint32_t p = __popc(m);
                    cr[j] += sign_flip(c0, p);
                    ci[j] += sign_flip(c1, p);
                }
            }
#pragma unroll
            for (int j = 0; j < V; j++) {
                lr[j] += cr[j] * pb[j].x - ci[j] * pb[j].y;
                li[j] += cr[j] * pb[j].y + ci[j] * pb[j].x;
            }
        }
    }
}

}  // namespace gbvqc
