// Shared definitions of the GB300 library: matrix records, structural shapes of gate
// kernels, and materialisation of the theta-dependent rotation matrices (host + device).
#pragma once

#ifdef __CUDACC_RTC__
// runtime compilation of specialised tile passes (NVRTC): no host headers
typedef signed char int8_t;
typedef short int16_t;
typedef int int32_t;
typedef long long int64_t;
typedef unsigned char uint8_t;
typedef unsigned short uint16_t;
typedef unsigned int uint32_t;
typedef unsigned long long uint64_t;
#else
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#endif

namespace gbvqc {

// One gate matrix (up to 4x4 complex, row-major, interleaved re/im) kept in both
// precisions so that complex64 and complex128 sweeps read the same record.
struct alignas(16) MatRec {
    double d[32];
    float f[32];
};

// Structural specialisation of a gate kernel (paper Sec. II.B: predefined gates run
// faster than the general QuantumGate by exploiting their structure).
enum Shape : int32_t {
    SH_DENSE1 = 0,  // general 2x2
    SH_DIAG1 = 1,   // diagonal 2x2 (Z, S, T, Rz)
    SH_ANTI1 = 2,   // anti-diagonal 2x2 (X, Y)
    SH_REAL1 = 3,   // real 2x2 (Ry, H)
    SH_DENSE2 = 4,  // general 4x4
    SH_DIAG2 = 5,   // diagonal 4x4 (CZ, superoperators of Rz)
    SH_PERM2 = 6,   // one non-zero per row (SWAP, iSWAP)
    SH_CTRL2 = 7,   // identity unless the first qubit is 1, then a 2x2 on the second
    SH_BLOCK2 = 8,  // phase on |00>, a 2x2 on {|01>, |10>}, phase on |11> (FSIM, iSWAP-like)
    SH_IMAG1 = 9,   // real diagonal, imaginary off-diagonal 2x2 (Rx; sqrt(X) up to a phase)
    SH_DENSE4 = 10, // general 16x16 (two-qubit channel superoperator), 16 records of one row
    SH_PAR2 = 11,   // parity-preserving 4x4: a 2x2 on {|00>, |11>} and a 2x2 on {|01>, |10>}
                    // (superoperator of a phase-covariant one-qubit channel on (ket, bra))
    SH_RPAR2 = 12,  // SH_PAR2 with real entries (depolarising, amplitude and phase damping)
    SH_CX = 13,     // exactly CNOT (control = first qubit): a swap, no arithmetic
    SH_CZ = 14,     // exactly CZ: the sign of |11>, no arithmetic
    SH_RDIAG1 = 15, // real diagonal, general off-diagonal 2x2 (a fixed gate such as sqrt(W)
                    // after phase normalisation); one-qubit layer entries only
    SH_ROT1 = 16    // a rotation [[c, -s], [s, c]] applied as three shears (unit entries:
                    // alpha, beta; kUnitShear); up to a global sign, so gradient plans only
};

inline __host__ __device__ bool shape_is_diag(int sh) { return sh == SH_DIAG1 || sh == SH_DIAG2 || sh == SH_CZ; }
inline __host__ __device__ int shape_qubits(int sh)
{
    return sh == SH_DENSE4 ? 4 : (sh >= SH_DENSE2 && sh <= SH_BLOCK2) || (sh >= SH_PAR2 && sh <= SH_CZ) ? 2 : 1;
}

// Row-major re/im offsets of the 2x2 block of an SH_BLOCK2 matrix (rows/columns 1 and 2)
// and of its two diagonal phases (rows 0 and 3).
#define GBVQC_BLOCK2_U(m) {(m)[10], (m)[11], (m)[12], (m)[13], (m)[18], (m)[19], (m)[20], (m)[21]}
// ... and of the 2x2 on rows/columns 0 and 3 (the other block of an SH_PAR2 matrix).
#define GBVQC_OUTER_U(m) {(m)[0], (m)[1], (m)[6], (m)[7], (m)[24], (m)[25], (m)[30], (m)[31]}

enum Rot : int32_t { ROT_X = 0, ROT_Y = 1, ROT_Z = 2, ROT_FSIM = 3 };
// FWD: U; INV: U^-1 (= U^dag); DER: dU/dp; GEN: (dU/dp) U^dag, the derivative read from
// the state after the gate (FSIM parameter p = comp).
enum Variant : int32_t { VAR_FWD = 0, VAR_INV = 1, VAR_DER = 2, VAR_GEN = 3 };
// KET: U on the ket (or pure) qubit; BRA: conj(U) on the bra qubit q+n;
// SUPER: the 4x4 U (x) conj(U) on (q, q+n) of the vectorised density matrix (Eq. channel2).
enum Domain : int32_t { DOM_KET = 0, DOM_BRA = 1, DOM_SUPER = 2 };

// A matrix record whose entries depend on theta[param] (FSIM: on theta[param + j] for
// the j-th set bit of mask; the parameters outside mask take their values from fixed).
struct DynRec {
    int32_t rec, param, rot, variant, domain, comp;
    int32_t mask, pad;
    double fixed[5];
};

// 2x2 rotation exp(-i t P / 2) for P = X, Y, Z (Sec. II.B: Rx, Ry with the unitary sign,
// Rz), its inverse R(-t) and its derivative dR/dt; row-major (re, im).
inline __host__ __device__ void rot2(int rot, int variant, double t, double *m)
{
    double s, c;
#ifdef __CUDA_ARCH__
    sincos(0.5 * t, &s, &c);
#else
    s = sin(0.5 * t);
    c = cos(0.5 * t);
#endif
    for (int i = 0; i < 8; i++) m[i] = 0.0;
    if (variant == VAR_INV) s = -s;  // R(-t) = R(t)^dag
    if (variant == VAR_DER) {
        if (rot == ROT_X) {        // [[-s/2, -i c/2], [-i c/2, -s/2]]
            m[0] = -0.5 * s; m[3] = -0.5 * c; m[5] = -0.5 * c; m[6] = -0.5 * s;
        } else if (rot == ROT_Y) { // [[-s/2, -c/2], [c/2, -s/2]]
            m[0] = -0.5 * s; m[2] = -0.5 * c; m[4] = 0.5 * c; m[6] = -0.5 * s;
        } else {                   // diag(-s/2 - i c/2, -s/2 + i c/2)
            m[0] = -0.5 * s; m[1] = -0.5 * c; m[6] = -0.5 * s; m[7] = 0.5 * c;
        }
        return;
    }
    if (rot == ROT_X) {            // [[c, -i s], [-i s, c]]
        m[0] = c; m[3] = -s; m[5] = -s; m[6] = c;
    } else if (rot == ROT_Y) {     // [[c, -s], [s, c]]
        m[0] = c; m[2] = -s; m[4] = s; m[6] = c;
    } else {                       // diag(c - i s, c + i s)
        m[0] = c; m[1] = -s; m[6] = c; m[7] = s;
    }
}

// S[(a + 2b), (c + 2d)] = A[a][c] * conj(B[b][d]) (4x4 from two 2x2, row-major re/im).
inline __host__ __device__ void kron_conj(const double *A, const double *B, double *S, bool add)
{
    for (int a = 0; a < 2; a++)
        for (int b = 0; b < 2; b++)
            for (int c = 0; c < 2; c++)
                for (int d = 0; d < 2; d++) {
                    double ar = A[2 * (2 * a + c)], ai = A[2 * (2 * a + c) + 1];
                    double br = B[2 * (2 * b + d)], bi = -B[2 * (2 * b + d) + 1];
                    int o = 2 * ((a + 2 * b) * 4 + (c + 2 * d));
                    double re = ar * br - ai * bi, im = ar * bi + ai * br;
                    if (add) { S[o] += re; S[o + 1] += im; }
                    else { S[o] = re; S[o + 1] = im; }
                }
}

inline __host__ __device__ void cis(double a, double &c, double &s)
{
#ifdef __CUDA_ARCH__
    sincos(a, &s, &c);
#else
    s = sin(a);
    c = cos(a);
#endif
}

// FSIM of Eq. (FSIM) with v = (theta, phi, d_plus, d_minus, d_minus_off), row-major re/im
// (first qubit = matrix bit 0; the 2x2 block sits on rows/columns 1 and 2), or with
// comp >= 0 its derivative with respect to v[comp]: d/dtheta turns cos into -sin and sin
// into cos; a phase parameter multiplies each entry by i times its coefficient.
inline __host__ __device__ void fsim_matrix(const double *v, int comp, double *m)
{
    double ct, st, c11, s11, c12, s12, c21, s21, c22, s22, c33, s33;
    cis(v[0], ct, st);
    cis(v[2] + v[3], c11, s11);
    cis(v[2] - v[4], c12, s12);
    cis(v[2] + v[4], c21, s21);
    cis(v[2] - v[3], c22, s22);
    cis(2.0 * v[2] - v[1], c33, s33);
    for (int i = 0; i < 32; i++) m[i] = 0.0;
    // entries as (amplitude a, phase cis(x)): 11 = cos(th) cis, 12 = -i sin(th) cis,
    // 21 = -i sin(th) cis, 22 = cos(th) cis, 33 = cis
    double a11 = ct, a12 = st, a22 = ct;           // real amplitudes (12, 21 carry the -i)
    double f00 = 1, f11 = 1, f12 = 1, f21 = 1, f22 = 1, f33 = 1;  // i-multipliers (real part)
    double g11 = 0, g12 = 0, g21 = 0, g22 = 0, g33 = 0;            // (imaginary part)
    if (comp == 0) {
        a11 = -st; a12 = ct; a22 = -st;
        f33 = 0; f00 = 0;
    } else if (comp >= 1) {
        // d/dv_k: entry * (i * coefficient of v_k in the entry's exponent)
        const double k11 = comp == 2 ? 1 : comp == 3 ? 1 : 0;
        const double k12 = comp == 2 ? 1 : comp == 4 ? -1 : 0;
        const double k21 = comp == 2 ? 1 : comp == 4 ? 1 : 0;
        const double k22 = comp == 2 ? 1 : comp == 3 ? -1 : 0;
        const double k33 = comp == 2 ? 2 : comp == 1 ? -1 : 0;
        f00 = 0;
        f11 = 0; g11 = k11;
        f12 = 0; g12 = k12;
        f21 = 0; g21 = k21;
        f22 = 0; g22 = k22;
        f33 = 0; g33 = k33;
    }
    // z = (f + i g) * amplitude * cis; the -i of entries 12 and 21 applied last
    auto put = [&](int idx, double amp, double c, double s, double f, double g, bool minus_i) {
        double re = amp * (f * c - g * s), im = amp * (f * s + g * c);
        if (minus_i) {
            const double t = re;
            re = im;
            im = -t;
        }
        m[2 * idx] = re;
        m[2 * idx + 1] = im;
    };
    m[0] = f00;
    put(5, a11, c11, s11, f11, g11, false);
    put(6, a12, c12, s12, f12, g12, true);
    put(9, a12, c21, s21, f21, g21, true);
    put(10, a22, c22, s22, f22, g22, false);
    put(15, 1.0, c33, s33, f33, g33, false);
}

// c = a * b^dag for 4x4 complex row-major re/im matrices.
inline __host__ __device__ void mul_dag4(const double *a, const double *b, double *c)
{
    for (int r = 0; r < 4; r++)
        for (int col = 0; col < 4; col++) {
            double re = 0, im = 0;
            for (int k = 0; k < 4; k++) {
                const double ar = a[2 * (4 * r + k)], ai = a[2 * (4 * r + k) + 1];
                const double br = b[2 * (4 * col + k)], bi = -b[2 * (4 * col + k) + 1];  // conj(b[col][k])
                re += ar * br - ai * bi;
                im += ar * bi + ai * br;
            }
            c[2 * (4 * r + col)] = re;
            c[2 * (4 * r + col) + 1] = im;
        }
}

// Fill a record for a theta-dependent matrix; th points at theta[r.param].
inline __host__ __device__ void materialize(const DynRec &r, const double *th, MatRec *out)
{
    double m[32];
    for (int i = 0; i < 32; i++) m[i] = 0.0;
    if (r.rot == ROT_FSIM) {
        double v[5];
        for (int k = 0, j = 0; k < 5; k++) v[k] = ((r.mask >> k) & 1) ? th[j++] : r.fixed[k];
        if (r.variant == VAR_FWD) {
            fsim_matrix(v, -1, m);
        } else if (r.variant == VAR_DER) {
            fsim_matrix(v, r.comp, m);
        } else {
            double u[32];
            fsim_matrix(v, -1, u);
            if (r.variant == VAR_INV) {  // U^dag
                for (int a = 0; a < 4; a++)
                    for (int b = 0; b < 4; b++) {
                        m[2 * (4 * a + b)] = u[2 * (4 * b + a)];
                        m[2 * (4 * a + b) + 1] = -u[2 * (4 * b + a) + 1];
                    }
            } else {  // VAR_GEN: (dU/dv) U^dag
                double d[32];
                fsim_matrix(v, r.comp, d);
                mul_dag4(d, u, m);
            }
        }
        if (r.domain == DOM_BRA)  // conj(U), and correspondingly conjugated inverse / derivatives
            for (int i = 1; i < 32; i += 2) m[i] = -m[i];
        for (int i = 0; i < 32; i++) {
            out->d[i] = m[i];
            out->f[i] = (float)m[i];
        }
        return;
    }
    const double t = th[0];
    if (r.domain == DOM_SUPER) {
        double U[8], dU[8];
        if (r.variant == VAR_DER) {
            rot2(r.rot, VAR_FWD, t, U);
            rot2(r.rot, VAR_DER, t, dU);
            kron_conj(dU, U, m, false);
            kron_conj(U, dU, m, true);
        } else {
            rot2(r.rot, r.variant, t, U);
            kron_conj(U, U, m, false);
        }
    } else {
        rot2(r.rot, r.variant, t, m);
        if (r.domain == DOM_BRA)
            for (int i = 1; i < 8; i += 2) m[i] = -m[i];
    }
    // a 2x2 fills the first 8 entries; the rest of the record stays zero
    const int used = r.domain == DOM_SUPER ? 32 : 8;
    for (int i = 0; i < used; i++) {
        out->d[i] = m[i];
        out->f[i] = (float)m[i];
    }
}

// ------------------------------------------------------------------ fused tile plan

// Gate of a fused pass.  Non-diagonal gates name register slots (0..NR-1) of their
// sub-run.  Diagonal gates and Z generators name a position code c: c < NR is a
// register slot, NR <= c is local tile position c - NR (not held in registers), and
// c < 0 is the tile-index bit of physical qubit -1 - c (constant over the tile).
enum FType : int32_t {
    FT_DENSE1 = 0, FT_REAL1 = 1, FT_ANTI1 = 2, FT_DIAG1 = 3,
    FT_DENSE2 = 4, FT_DIAG2 = 5, FT_PERM2 = 6, FT_CTRL2 = 7,
    FT_DIAGB = 8,  // a run of commuting diagonal gates (DEnt list) fused into one phase table
    FT_LAYER1 = 9,  // one-qubit non-diagonal gates on distinct register slots: a = slot
                    // mask, b = entries, perm = per-slot shape code, forward: mat = first
                    // of the entries' consecutive units; DEnt list (slot order): entry =
                    // Shape, ca = slot, cls = GenType, mat / mat2, gradient slot and weight
    FT_BLOCK2 = 10,  // SH_BLOCK2 on two register slots
    FT_IMAG1 = 11,   // SH_IMAG1 on one register slot
    FT_PROBE2 = 12,  // reverse only: gradient read 2 Re <Psi| K |Phi> with the 4x4 K on two
                     // register slots; the states are not changed
    FT_DENSE4 = 13,  // a two-qubit channel's superoperator: never in a tile pass (the planner
                     // makes it a pass of its own, run by the per-gate kernel)
    FT_PAR2 = 14,    // SH_PAR2 on two register slots
    FT_RPAR2 = 15    // SH_RPAR2 on two register slots
};
// FGate.perm of an FT_BLOCK2 gate with a fixed matrix (set at plan time, read by the
// specialised passes only): BLOCK2_VARIANT | inner shape (bits 0-1: 0 general, 1 real
// diagonal with imaginary off-diagonal, 2 real) | P00 / P11 = 1 flags.
enum : int32_t { BLOCK2_VARIANT = 0x100, BLOCK2_P00_ONE = 4, BLOCK2_P11_ONE = 8 };
// Generator of a variational gate for the fused reverse sweep: the gradient term is
// coef * Im <Psi| P |Phi> with both states taken right after the gate.
enum GenType : int32_t { GEN_NONE = 0, GEN_X = 1, GEN_Y = 2, GEN_Z = 3, GEN_M2 = 4 /* FT_PROBE2 */ };

// Matrices of a pass are staged in shared memory in units of 8 elements (a 2x2 matrix is
// one unit, a 4x4 matrix four); unit u copies elements 8*part .. 8*part+7 of record rec.
struct MatUnit {
    int32_t rec, part;
};
// MatUnit.part of a unit holding a rotation record's shear parameters (alpha, beta, 0...):
// for c >= 0, alpha = -s / (1 + c), beta = s; for c < 0 the shears of -R, alpha = s / (1 - c),
// beta = -s (|alpha| <= 1 both ways; the dropped sign is a global phase).
constexpr int32_t kUnitShear = 8;

struct FGate {               // 32 bytes, staged in shared memory
    int8_t type;             // FType
    int8_t a, b;             // register slots (non-diagonal) or position codes (FT_DIAG1/2)
    int8_t gen;              // GEN_X / GEN_Y generator of a variational non-diagonal gate
    int8_t gpos;             // its register slot
    int8_t flags;            // FT_DIAGB: bit 0 = Psi uses separate phases (non-unitary block)
    int8_t nz;               // FT_DIAGB: number of Z-generator entries (listed first)
    int8_t pad0;
    int16_t mat, mat2;       // pass-local matrix units: Phi (forward: U) / Psi (reverse)
    int16_t ent, n_ent;      // FT_DIAGB: first pass-local DEnt and count (incl. Z entries)
    int32_t slot;            // X/Y generator: gradient slot (-1 if none); FT_DIAGB: pass-local
                             // block index (its tile-constant phase product in shared memory)
    float coef;              // gradient weight
    int32_t perm;            // FT_DIAGB: entry counts per class after the Z entries:
                             // tile | local << 8 | register << 16 | pair << 24
                             // (table mode: tile | local << 8 | mixed CZ << 16);
                             // FT_PERM2: source column of output row r in bits 2r, 2r+1
    int32_t pad1;
};

// Classes of diagonal entries inside a phase block, listed in this order after the Z
// generators: TILE (every position is a tile-index bit: one product per CTA), LOCAL (no
// register position: one factor per thread), REG (one register position, the other
// constant: a factor pair on that register bit), PAIR (two register positions: factor
// pairs plus a controlled phase on |11>), PAIR_CZ (the |11> sign flip of CZ).
enum DClass : int8_t { DC_Z = 0, DC_TILE = 1, DC_LOCAL = 2, DC_REG = 3, DC_PAIR = 4, DC_PAIR_CZ = 5 };

// Table mode of a phase block (FGate.flags bit 1): every entry on register positions
// only (one-qubit phases on a register bit, two-qubit diagonals on two register bits) is
// multiplied into one table over the 2^NR register indices, the same for every thread
// of every tile; it is computed once per step (k_phase_tables, FP64 products of the FP64
// records rounded once) into the pass's matrix image at unit FGate.mat (Psi: mat2), and
// the kernel multiplies amplitude j by table[j].  The block's DEnt list after its Z
// entries is then TILE, LOCAL, and MIXCZ entries: CZ between a register position and a
// constant one, a sign flip of the amplitudes whose register bit is 1 in the threads
// whose constant bit is 1.  Blocks with any other mixed entry keep the factor-pair form.
constexpr int FLAG_SEPARATE = 1;  // Psi takes its own phases (a non-unitary block)
constexpr int FLAG_TABLE = 2;     // table mode

// One register phase table: 2^nbits complex entries at img[off .. off + 2^(nbits+1)) (reals)
// of the direction's matrix image, the product of TabEnt [ent_begin, ent_begin + n_ent).
struct TabDesc {
    int32_t off, nbits, ent_begin, n_ent;
};
struct TabEnt {
    int32_t rec;             // matrix record (its FP64 entries)
    int8_t k;                // 1: diagonal 2x2 on register bit ca; 2: diagonal 4x4 on (ca, cb)
    int8_t ca, cb;
    int8_t pad;
};

struct DEnt {                // 16 bytes: one diagonal gate or Z generator of an FT_DIAGB
    int8_t k;                // 1 or 2 positions with phases; 3 = Z generator only
    int8_t ca, cb;           // position codes
    int8_t cls;              // DClass
    int16_t mat, mat2;       // pass-local matrix units of the Phi / Psi phases
    int32_t slot;            // Z generator: gradient slot
    float coef;              // Z generator: gradient weight
};

struct SubRun {
    int8_t R[8];             // local positions held in registers (NR of them)
    int32_t g_begin, g_end;  // pass-local gate range
};

struct PassDesc {
    int32_t t;               // tile qubits
    int32_t n;               // physical qubits of the state
    int32_t sub_begin, n_sub;
    int32_t slot_begin, n_slots;    // gradient slots touched by this pass (reverse sweep)
    int32_t gate_begin, n_gates;    // FGate range (global array)
    int32_t ent_begin, n_ent;       // DEnt range
    int32_t unit_begin, n_units;    // MatUnit range
    int8_t S[16];            // local position -> physical qubit (ascending)
    int8_t NS[64];           // tile-index bit -> physical qubit (ascending)
    int32_t low;             // S[0..low-1] = 0..low-1 (contiguous in memory)
    int32_t n_blocks;        // FT_DIAGB gates in the pass
    int32_t has_2q;          // the pass holds non-diagonal two-qubit gates (kernel flavour)
    int32_t pad2;
};

}  // namespace gbvqc
