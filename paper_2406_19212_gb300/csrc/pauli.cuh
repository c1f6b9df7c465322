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
        ObsTerm t = terms[k];
        R c = (R)t.coeff;
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

}  // namespace gbvqc
