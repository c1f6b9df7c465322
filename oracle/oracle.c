/*
 * Oracle: a plain, slow, FP64 CPU reference for the variational circuit simulator.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the CUDA library links, includes or calls this
 * file; only the tests, the smoke check and the CPU-baseline leg of the benchmark load
 * it.  It shares no code with the GPU path: its own gate matrices, its own index
 * arithmetic, its own reductions.
 *
 * What it computes (JuliVQC, arXiv 2406.19212):
 *   - gate matrices of Sec. II.B (Rx/Ry/Rz, FSIM, named gates, Kraus operators);
 *   - the Schroedinger update of Eq. (3) and Eq. (twoqubitgate): for every assignment
 *     of the untouched qubits, gather the 2^k amplitudes of the gate's qubits, multiply
 *     by the 2^k x 2^k matrix, scatter back (Algorithm 1, generalised to k qubits);
 *   - circuit evolution Eq. (circuitevolve): gates applied in order;
 *   - expectation of a Pauli sum (Sec. II.E): sum_k c_k <psi|P_k psi>, with P_k psi
 *     formed by applying each single-qubit Pauli matrix as a gate;
 *   - the memory-efficient adjoint gradient, Algorithm 2 (Sec. III.C);
 *   - density matrices (Sec. III.D): rho -> sum_s K_s rho K_s^dag on the 2^n x 2^n
 *     matrix (Eq. channel), and tr(H rho);
 *   - the noisy adjoint gradient of Sec. III.E on the vectorised |rho>> with
 *     superoperators M = sum_s K_s (x) conj(K_s) (Eq. channel2, read with the
 *     conjugate on the bra index);
 *   - measure!(state, i) of Sec. II.D: the probability of each outcome of qubit i, the
 *     outcome picked by a caller-supplied uniform u (0 if u < P(0)), and the collapsed,
 *     renormalised state (pure or density); and sampling of all qubits (the index where
 *     the cumulative probability first exceeds u times the total).
 *
 * Readings of the paper taken here (each also listed in the design notes):
 *   - the printed Ry matrix [[c,-s],[-s,c]] is not unitary: Ry = [[c,-s],[s,c]];
 *   - the third rotation printed as "Rx" is Rz = diag(e^{-i t/2}, e^{i t/2});
 *   - Depolarizing: K0 = sqrt(1-3p/4) I, K1..3 = sqrt(p/4) X, Y, Z (the printed
 *     sqrt(p/2) breaks completeness);
 *   - sqrt(G) for G in {X, Y, W=(X+Y)/sqrt2} is the principal root ((1+i)I+(1-i)G)/2;
 *   - in the noisy Algorithm 2 the state Phi is uncomputed with S^{-1} and the adjoint
 *     state Psi with S^dag (for unitary S these agree).
 *
 * Layout: qubit q is bit q of the amplitude index; the first listed qubit of a gate is
 * the least significant bit of the gate-matrix index; matrices are row-major; a density
 * matrix element rho_ab sits at index a + 2^n b.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

enum {
    O_X, O_Y, O_Z, O_H, O_S, O_T, O_SX, O_SY, O_SW, O_RX, O_RY, O_RZ,
    O_CNOT, O_CZ, O_SWAP, O_ISWAP, O_FSIM, O_CONTROL, O_DENSE1, O_DENSE2,
    O_DEPOL, O_AMPDAMP, O_PHASEDAMP, O_KRAUS, O_DEPOL2, O_KRAUS2
};

typedef struct {
    int32_t kind;
    int32_t nq;
    int32_t q[2];
    int32_t param;     /* index into theta, -1 = fixed */
    int32_t n_kraus;
    int32_t pmask;     /* FSIM: bit k set = parameter k is variational (theta[param + rank]) */
    double fixed[5];
    double data[32];   /* complex (re, im) pairs, row-major; KRAUS: n_kraus 2x2 blocks */
    const double *kraus; /* KRAUS2: n_kraus 4x4 blocks, (re, im) row-major */
} orc_op;

static int is_channel(int kind) { return kind >= O_DEPOL; }

/* ----------------------------------------------------------------- gate matrices */

static double op_angle(const orc_op *op, const double *theta)
{
    return op->param >= 0 ? theta[op->param] : op->fixed[0];
}

/* The five FSIM parameters (theta, phi, d_plus, d_minus, d_minus_off): the variational
 * ones (bits of pmask, in increasing k) read consecutive entries of theta from param. */
static void fsim_values(const orc_op *op, const double *theta, double v[5])
{
    int k, r = 0;
    for (k = 0; k < 5; k++) {
        v[k] = op->fixed[k];
        if (op->param >= 0 && ((op->pmask >> k) & 1)) v[k] = theta[op->param + r++];
    }
}

/* Fill the row-major matrix of a unitary op; returns its qubit count k. */
static int gate_matrix(const orc_op *op, const double *theta, cplx *M)
{
    const double r2 = 1.0 / sqrt(2.0);
    double t, c, s;
    int i;
    for (i = 0; i < 16; i++) M[i] = 0;
    switch (op->kind) {
    case O_X: M[1] = 1; M[2] = 1; return 1;
    case O_Y: M[1] = -I; M[2] = I; return 1;
    case O_Z: M[0] = 1; M[3] = -1; return 1;
    case O_H: M[0] = r2; M[1] = r2; M[2] = r2; M[3] = -r2; return 1;
    case O_S: M[0] = 1; M[3] = I; return 1;
    case O_T: M[0] = 1; M[3] = cexp(I * M_PI / 4); return 1;
    case O_SX: /* ((1+i) I + (1-i) X) / 2 */
        M[0] = (1 + I) / 2; M[1] = (1 - I) / 2; M[2] = (1 - I) / 2; M[3] = (1 + I) / 2;
        return 1;
    case O_SY: /* ((1+i) I + (1-i) Y) / 2, Y = [[0,-i],[i,0]] */
        M[0] = (1 + I) / 2; M[1] = (1 - I) / 2 * (-I); M[2] = (1 - I) / 2 * I;
        M[3] = (1 + I) / 2;
        return 1;
    case O_SW: /* ((1+i) I + (1-i) W) / 2, W = (X+Y)/sqrt2 = [[0,(1-i)/r],[(1+i)/r,0]] */
        M[0] = (1 + I) / 2; M[1] = (1 - I) / 2 * ((1 - I) * r2);
        M[2] = (1 - I) / 2 * ((1 + I) * r2); M[3] = (1 + I) / 2;
        return 1;
    case O_RX: /* Sec. II.B, Rx */
        t = op_angle(op, theta); c = cos(t / 2); s = sin(t / 2);
        M[0] = c; M[1] = -I * s; M[2] = -I * s; M[3] = c;
        return 1;
    case O_RY: /* Sec. II.B, Ry (sign of the lower-left entry read as +) */
        t = op_angle(op, theta); c = cos(t / 2); s = sin(t / 2);
        M[0] = c; M[1] = -s; M[2] = s; M[3] = c;
        return 1;
    case O_RZ: /* Sec. II.B, third rotation (printed label "Rx") */
        t = op_angle(op, theta);
        M[0] = cexp(-I * t / 2); M[3] = cexp(I * t / 2);
        return 1;
    case O_DENSE1:
        for (i = 0; i < 4; i++) M[i] = op->data[2 * i] + I * op->data[2 * i + 1];
        return 1;
    /* two-qubit gates: matrix index = bit(q[0]) + 2 bit(q[1]) */
    case O_CNOT: /* control q[0], target q[1] */
        M[0 * 4 + 0] = 1; M[2 * 4 + 2] = 1; M[1 * 4 + 3] = 1; M[3 * 4 + 1] = 1;
        return 2;
    case O_CZ: M[0] = 1; M[5] = 1; M[10] = 1; M[15] = -1; return 2;
    case O_SWAP: M[0] = 1; M[1 * 4 + 2] = 1; M[2 * 4 + 1] = 1; M[15] = 1; return 2;
    case O_ISWAP: M[0] = 1; M[1 * 4 + 2] = I; M[2 * 4 + 1] = I; M[15] = 1; return 2;
    case O_FSIM: { /* Eq. (FSIM): (theta, phi, d_plus, d_minus, d_minus_off) */
        double v[5];
        fsim_values(op, theta, v);
        double th = v[0], ph = v[1], dp = v[2], dm = v[3], dmo = v[4];
        M[0] = 1;
        M[1 * 4 + 1] = cexp(I * (dp + dm)) * cos(th);
        M[1 * 4 + 2] = -I * cexp(I * (dp - dmo)) * sin(th);
        M[2 * 4 + 1] = -I * cexp(I * (dp + dmo)) * sin(th);
        M[2 * 4 + 2] = cexp(I * (dp - dm)) * cos(th);
        M[3 * 4 + 3] = cexp(I * (2 * dp - ph));
        return 2;
    }
    case O_CONTROL: { /* control q[0]; target block U (2x2) on q[1] when control = 1 */
        int a, b;
        M[0] = 1; M[2 * 4 + 2] = 1;
        for (a = 0; a < 2; a++)
            for (b = 0; b < 2; b++)
                M[(1 + 2 * a) * 4 + (1 + 2 * b)] =
                    op->data[2 * (2 * a + b)] + I * op->data[2 * (2 * a + b) + 1];
        return 2;
    }
    case O_DENSE2:
        for (i = 0; i < 16; i++) M[i] = op->data[2 * i] + I * op->data[2 * i + 1];
        return 2;
    default:
        return -1;
    }
}

/* Derivative of a variational rotation's matrix with respect to its angle. */
static int gate_derivative(const orc_op *op, const double *theta, cplx *D)
{
    double t = op_angle(op, theta), c = cos(t / 2), s = sin(t / 2);
    int i;
    for (i = 0; i < 4; i++) D[i] = 0;
    switch (op->kind) {
    case O_RX: D[0] = -s / 2; D[1] = -I * c / 2; D[2] = -I * c / 2; D[3] = -s / 2; return 1;
    case O_RY: D[0] = -s / 2; D[1] = -c / 2; D[2] = c / 2; D[3] = -s / 2; return 1;
    case O_RZ: D[0] = -I / 2 * cexp(-I * t / 2); D[3] = I / 2 * cexp(I * t / 2); return 1;
    default: return -1;
    }
}

/* Derivative of the FSIM matrix of Eq. (FSIM) with respect to its parameter k (entry by
 * entry: d/dtheta turns cos into -sin and sin into cos; a phase parameter multiplies each
 * entry by i times its coefficient in that entry's exponent). */
static void fsim_derivative(const orc_op *op, const double *theta, int k, cplx *D)
{
    double v[5];
    cplx M[16];
    int i;
    fsim_values(op, theta, v);
    gate_matrix(op, theta, M);
    for (i = 0; i < 16; i++) D[i] = 0;
    switch (k) {
    case 0: {
        const double th = v[0], dp = v[2], dm = v[3], dmo = v[4];
        D[1 * 4 + 1] = -cexp(I * (dp + dm)) * sin(th);
        D[1 * 4 + 2] = -I * cexp(I * (dp - dmo)) * cos(th);
        D[2 * 4 + 1] = -I * cexp(I * (dp + dmo)) * cos(th);
        D[2 * 4 + 2] = -cexp(I * (dp - dm)) * sin(th);
        break;
    }
    case 1: D[15] = -I * M[15]; break;
    case 2:
        D[5] = I * M[5]; D[6] = I * M[6]; D[9] = I * M[9]; D[10] = I * M[10];
        D[15] = 2 * I * M[15];
        break;
    case 3: D[5] = I * M[5]; D[10] = -I * M[10]; break;
    default: D[6] = -I * M[6]; D[9] = I * M[9]; break;
    }
}

/* Kraus operators of a channel (Sec. II.B, QuantumMap): returns their count and sets *k
 * to the channel's qubit count (K holds count blocks of 2^k x 2^k entries). */
static int channel_kraus_k(const orc_op *op, cplx *K /* up to 256 entries */, int *k)
{
    double g = op->fixed[0];
    int i;
    for (i = 0; i < 256; i++) K[i] = 0;
    *k = 1;
    switch (op->kind) {
    case O_DEPOL2: { /* sqrt(1 - 15p/16) I, sqrt(p/16) s_a (x) s_b for the 15 other Paulis */
        const cplx P[4][4] = {{1, 0, 0, 1}, {0, 1, 1, 0}, {0, -I, I, 0}, {1, 0, 0, -1}};
        int a, b, r0, r1, c0, c1;
        *k = 2;
        for (a = 0; a < 4; a++)       /* Pauli on the first qubit (matrix bit 0) */
            for (b = 0; b < 4; b++) { /* Pauli on the second qubit (matrix bit 1) */
                const double w = (a == 0 && b == 0) ? sqrt(1 - 15 * g / 16) : sqrt(g / 16);
                cplx *M = K + 16 * (4 * b + a);
                for (r0 = 0; r0 < 2; r0++)
                    for (r1 = 0; r1 < 2; r1++)
                        for (c0 = 0; c0 < 2; c0++)
                            for (c1 = 0; c1 < 2; c1++)
                                M[(r0 + 2 * r1) * 4 + (c0 + 2 * c1)] = w * P[a][2 * r0 + c0] * P[b][2 * r1 + c1];
            }
        return 16;
    }
    case O_KRAUS2:
        *k = 2;
        for (i = 0; i < 16 * op->n_kraus; i++) K[i] = op->kraus[2 * i] + I * op->kraus[2 * i + 1];
        return op->n_kraus;
    case O_AMPDAMP:
        K[0] = 1; K[3] = sqrt(1 - g);
        K[4 + 1] = sqrt(g);
        return 2;
    case O_PHASEDAMP:
        K[0] = 1; K[3] = sqrt(1 - g);
        K[4 + 3] = sqrt(g);
        return 2;
    case O_DEPOL: {
        double a = sqrt(1 - 3 * g / 4), b = sqrt(g / 4);
        K[0] = a; K[3] = a;
        K[4 + 1] = b; K[4 + 2] = b;             /* X */
        K[8 + 1] = -I * b; K[8 + 2] = I * b;    /* Y */
        K[12 + 0] = b; K[12 + 3] = -b;          /* Z */
        return 4;
    }
    case O_KRAUS:
        for (i = 0; i < 4 * op->n_kraus; i++) K[i] = op->data[2 * i] + I * op->data[2 * i + 1];
        return op->n_kraus;
    default:
        return -1;
    }
}

/* ------------------------------------------------------------ state evolution */

/* Eq. (3) / Eq. (twoqubitgate) / Algorithm 1 for k qubits: psi <- M acting on qs. */
static void apply_k(cplx *psi, int n, int k, const int *qs, const cplx *M)
{
    int sorted[8], t, a, b;
    int64_t g, ngroups = (int64_t)1 << (n - k);
    for (t = 0; t < k; t++) sorted[t] = qs[t];
    for (a = 0; a < k; a++)                       /* insertion sort of bit positions */
        for (b = a + 1; b < k; b++)
            if (sorted[b] < sorted[a]) { int x = sorted[a]; sorted[a] = sorted[b]; sorted[b] = x; }
#pragma omp parallel for schedule(static) if (ngroups > 8192)
    for (g = 0; g < ngroups; g++) {
        int64_t base = g, idx[16];
        cplx v[16], w[16];
        int l, r, c, u;
        for (u = 0; u < k; u++) {                 /* insert a 0 bit at each gate qubit */
            int64_t low = base & (((int64_t)1 << sorted[u]) - 1);
            base = ((base >> sorted[u]) << (sorted[u] + 1)) | low;
        }
        for (l = 0; l < (1 << k); l++) {
            int64_t ix = base;
            for (u = 0; u < k; u++)
                if ((l >> u) & 1) ix |= (int64_t)1 << qs[u];
            idx[l] = ix;
            v[l] = psi[ix];
        }
        for (r = 0; r < (1 << k); r++) {
            cplx acc = 0;
            for (c = 0; c < (1 << k); c++) acc += M[r * (1 << k) + c] * v[c];
            w[r] = acc;
        }
        for (l = 0; l < (1 << k); l++) psi[idx[l]] = w[l];
    }
}

/* Blocked FP64 sum of conj(a) * b: fixed 4096-element blocks, blocks summed in order,
 * so the result does not depend on the thread count. */
static cplx inner(const cplx *a, const cplx *b, int64_t len)
{
    int64_t nb = (len + 4095) / 4096, blk;
    cplx *part = (cplx *)malloc(sizeof(cplx) * (size_t)nb), tot = 0;
#pragma omp parallel for schedule(static) if (nb > 4)
    for (blk = 0; blk < nb; blk++) {
        int64_t i, lo = blk * 4096, hi = lo + 4096 < len ? lo + 4096 : len;
        cplx s = 0;
        for (i = lo; i < hi; i++) s += conj(a[i]) * b[i];
        part[blk] = s;
    }
    for (blk = 0; blk < nb; blk++) tot += part[blk];
    free(part);
    return tot;
}

/* Gauss-Jordan inverse with partial pivoting of a d x d complex matrix (d <= 16). */
static int invert(int d, const cplx *A, cplx *Ainv)
{
    cplx m[16 * 32];
    int r, c, k;
    for (r = 0; r < d; r++)
        for (c = 0; c < 2 * d; c++)
            m[r * 2 * d + c] = c < d ? A[r * d + c] : (c - d == r ? 1 : 0);
    for (k = 0; k < d; k++) {
        int piv = k;
        for (r = k + 1; r < d; r++)
            if (cabs(m[r * 2 * d + k]) > cabs(m[piv * 2 * d + k])) piv = r;
        if (cabs(m[piv * 2 * d + k]) < 1e-300) return -1;
        if (piv != k)
            for (c = 0; c < 2 * d; c++) {
                cplx x = m[k * 2 * d + c]; m[k * 2 * d + c] = m[piv * 2 * d + c]; m[piv * 2 * d + c] = x;
            }
        {
            cplx p = m[k * 2 * d + k];
            for (c = 0; c < 2 * d; c++) m[k * 2 * d + c] /= p;
        }
        for (r = 0; r < d; r++)
            if (r != k) {
                cplx f = m[r * 2 * d + k];
                for (c = 0; c < 2 * d; c++) m[r * 2 * d + c] -= f * m[k * 2 * d + c];
            }
    }
    for (r = 0; r < d; r++)
        for (c = 0; c < d; c++) Ainv[r * d + c] = m[r * 2 * d + d + c];
    return 0;
}

/* ----------------------------------------------------------------- public: pure */

int orc_gate_matrix(const orc_op *op, const double *theta, double *out /* 32 doubles */)
{
    cplx M[16];
    int k = gate_matrix(op, theta, M), i;
    if (k < 0) return -1;
    for (i = 0; i < (1 << (2 * k)); i++) { out[2 * i] = creal(M[i]); out[2 * i + 1] = cimag(M[i]); }
    return k;
}

/* Kraus operators of a channel op: count returned, *k = its qubit count, out = count
 * blocks of 2^k x 2^k (re, im) entries, row-major (up to 512 doubles). */
int orc_kraus(const orc_op *op, double *out, int *k)
{
    cplx K[256];
    int m = channel_kraus_k(op, K, k), i;
    if (m < 0) return -1;
    for (i = 0; i < (1 << (2 * *k)) * m; i++) { out[2 * i] = creal(K[i]); out[2 * i + 1] = cimag(K[i]); }
    return m;
}

int orc_apply_matrix(double *psi, int n, int k, const int *qs, const double *mat)
{
    cplx M[256];
    int i;
    if (k < 1 || k > 4) return -1;
    for (i = 0; i < (1 << (2 * k)); i++) M[i] = mat[2 * i] + I * mat[2 * i + 1];
    apply_k((cplx *)psi, n, k, qs, M);
    return 0;
}

/* Eq. (circuitevolve): psi <- Q^M ... Q^1 psi, unitary ops only. */
int orc_apply_circuit(double *psi_, int n, const orc_op *ops, int n_ops, const double *theta)
{
    cplx *psi = (cplx *)psi_, M[16];
    int j;
    for (j = 0; j < n_ops; j++) {
        int k;
        if (is_channel(ops[j].kind)) return -2;
        k = gate_matrix(&ops[j], theta, M);
        if (k < 0) return -1;
        apply_k(psi, n, k, ops[j].q, M);
    }
    return 0;
}

/* out = P psi for one Pauli string (paulis[q] in 'I','X','Y','Z'), gate by gate. */
static void pauli_string_apply(cplx *out, const cplx *psi, int n, const char *paulis)
{
    static const cplx PX[4] = {0, 1, 1, 0}, PY[4] = {0, -I, I, 0}, PZ[4] = {1, 0, 0, -1};
    int q;
    memcpy(out, psi, sizeof(cplx) * ((size_t)1 << n));
    for (q = 0; q < n; q++) {
        const cplx *P = paulis[q] == 'X' ? PX : paulis[q] == 'Y' ? PY : paulis[q] == 'Z' ? PZ : 0;
        if (P) apply_k(out, n, 1, &q, P);
    }
}

/* out = H psi, H = sum_k coeff[k] P_k; pauli strings packed n chars per term. */
int orc_apply_hamiltonian(double *out_, const double *psi_, int n, const double *coeff,
                          const char *paulis, int n_terms)
{
    int64_t dim = (int64_t)1 << n, i;
    cplx *out = (cplx *)out_, *tmp = (cplx *)malloc(sizeof(cplx) * (size_t)dim);
    int t;
    for (i = 0; i < dim; i++) out[i] = 0;
    for (t = 0; t < n_terms; t++) {
        pauli_string_apply(tmp, (const cplx *)psi_, n, paulis + (size_t)t * n);
        for (i = 0; i < dim; i++) out[i] += coeff[t] * tmp[i];
    }
    free(tmp);
    return 0;
}

/* Sec. II.E: <psi|H|psi> = sum_k c_k <psi|P_k psi>; returns real and imaginary parts. */
int orc_expect(const double *psi_, int n, const double *coeff, const char *paulis,
               int n_terms, double *re_im)
{
    int64_t dim = (int64_t)1 << n;
    cplx *tmp = (cplx *)malloc(sizeof(cplx) * (size_t)dim), e = 0;
    int t;
    for (t = 0; t < n_terms; t++) {
        pauli_string_apply(tmp, (const cplx *)psi_, n, paulis + (size_t)t * n);
        e += coeff[t] * inner((const cplx *)psi_, tmp, dim);
    }
    free(tmp);
    re_im[0] = creal(e);
    re_im[1] = cimag(e);
    return 0;
}

/* Algorithm 2 (Sec. III.C).  Runs the circuit from |0...0>, then
 *   Phi = psi, Psi = H psi; for j = M..1: Phi <- Q_j^{-1} Phi;
 *   grads[j] = 2 Re <Psi| dQ_j |Phi>; Psi <- Q_j^{-1} Psi.
 * Gradients of gates sharing a parameter are summed into grad[param]. */
int orc_adjoint_grad(int n, const orc_op *ops, int n_ops, const double *theta, int n_params,
                     const double *coeff, const char *paulis, int n_terms,
                     double *energy, double *grad)
{
    int64_t dim = (int64_t)1 << n;
    cplx *phi = (cplx *)calloc((size_t)dim, sizeof(cplx));
    cplx *psi = (cplx *)malloc(sizeof(cplx) * (size_t)dim);
    cplx *tmp = (cplx *)malloc(sizeof(cplx) * (size_t)dim);
    cplx M[16], Minv[16], D[16];
    double e[2];
    int j, rc = 0;
    phi[0] = 1;
    if (orc_apply_circuit((double *)phi, n, ops, n_ops, theta) != 0) { rc = -1; goto done; }
    orc_expect((double *)phi, n, coeff, paulis, n_terms, e);
    *energy = e[0];
    orc_apply_hamiltonian((double *)psi, (const double *)phi, n, coeff, paulis, n_terms);
    for (j = 0; j < n_params; j++) grad[j] = 0;
    for (j = n_ops - 1; j >= 0; j--) {
        int k = gate_matrix(&ops[j], theta, M);
        if (invert(1 << k, M, Minv) != 0) { rc = -3; goto done; }
        apply_k(phi, n, k, ops[j].q, Minv);
        if (ops[j].param >= 0 && ops[j].kind == O_FSIM) {  /* one term per variational parameter */
            int b, r = 0;
            for (b = 0; b < 5; b++) {
                if (!((ops[j].pmask >> b) & 1)) continue;
                fsim_derivative(&ops[j], theta, b, D);
                memcpy(tmp, phi, sizeof(cplx) * (size_t)dim);
                apply_k(tmp, n, 2, ops[j].q, D);
                grad[ops[j].param + r++] += 2 * creal(inner(psi, tmp, dim));
            }
        } else if (ops[j].param >= 0) {
            int kd = gate_derivative(&ops[j], theta, D);
            if (kd < 0) { rc = -4; goto done; }
            memcpy(tmp, phi, sizeof(cplx) * (size_t)dim);
            apply_k(tmp, n, kd, ops[j].q, D);
            grad[ops[j].param] += 2 * creal(inner(psi, tmp, dim));
        }
        apply_k(psi, n, k, ops[j].q, Minv);
    }
done:
    free(phi); free(psi); free(tmp);
    return rc;
}

/* -------------------------------------------------------------- public: density */

/* rho <- K rho K^dag on the 2^n x 2^n matrix (rho_ab at a + 2^n b): K acts on every
 * column (ket index) and conj(K) on every row (bra index). */
static void rho_sandwich(cplx *rho, int n, int k, const int *qs, const cplx *K)
{
    int64_t dim = (int64_t)1 << n, a, b;
    cplx Kc[16];
    int i;
    for (i = 0; i < (1 << (2 * k)); i++) Kc[i] = conj(K[i]);
    for (b = 0; b < dim; b++) apply_k(rho + b * dim, n, k, qs, K);
    {
        cplx *row = (cplx *)malloc(sizeof(cplx) * (size_t)dim);
        for (a = 0; a < dim; a++) {
            for (b = 0; b < dim; b++) row[b] = rho[a + b * dim];
            apply_k(row, n, k, qs, Kc);
            for (b = 0; b < dim; b++) rho[a + b * dim] = row[b];
        }
        free(row);
    }
}

/* Eq. (channel): unitary gates as rho -> U rho U^dag, channels as sum_s K_s rho K_s^dag. */
int orc_rho_apply_circuit(double *rho_, int n, const orc_op *ops, int n_ops, const double *theta)
{
    cplx *rho = (cplx *)rho_, M[16];
    int64_t len = (int64_t)1 << (2 * n), i;
    int j;
    for (j = 0; j < n_ops; j++) {
        if (!is_channel(ops[j].kind)) {
            int k = gate_matrix(&ops[j], theta, M);
            if (k < 0) return -1;
            rho_sandwich(rho, n, k, ops[j].q, M);
        } else {
            cplx K[256];
            int kq, m = channel_kraus_k(&ops[j], K, &kq), s;
            cplx *acc = (cplx *)calloc((size_t)len, sizeof(cplx));
            cplx *tmp = (cplx *)malloc(sizeof(cplx) * (size_t)len);
            if (m < 0) { free(acc); free(tmp); return -1; }
            for (s = 0; s < m; s++) {
                memcpy(tmp, rho, sizeof(cplx) * (size_t)len);
                rho_sandwich(tmp, n, kq, ops[j].q, K + (1 << (2 * kq)) * s);
                for (i = 0; i < len; i++) acc[i] += tmp[i];
            }
            memcpy(rho, acc, sizeof(cplx) * (size_t)len);
            free(acc); free(tmp);
        }
    }
    return 0;
}

/* tr(H rho) = sum_k c_k tr(P_k rho): P_k applied to every column, then the trace. */
int orc_rho_expect(const double *rho_, int n, const double *coeff, const char *paulis,
                   int n_terms, double *re_im)
{
    int64_t dim = (int64_t)1 << n, a, b;
    const cplx *rho = (const cplx *)rho_;
    cplx *col = (cplx *)malloc(sizeof(cplx) * (size_t)dim), *pc = (cplx *)malloc(sizeof(cplx) * (size_t)dim);
    cplx e = 0;
    int t;
    for (t = 0; t < n_terms; t++) {
        cplx tr = 0;
        for (b = 0; b < dim; b++) {
            for (a = 0; a < dim; a++) col[a] = rho[a + b * dim];
            pauli_string_apply(pc, col, n, paulis + (size_t)t * n);
            tr += pc[b];
        }
        e += coeff[t] * tr;
    }
    free(col); free(pc);
    re_im[0] = creal(e);
    re_im[1] = cimag(e);
    return 0;
}

/* Superoperator of an op on the vectorised density matrix (Eq. channel2):
 * S[(r_ket + 2^k r_bra), (c_ket + 2^k c_bra)] = sum_s K_s[r_ket][c_ket] conj(K_s[r_bra][c_bra]),
 * acting on the 2k physical qubits (q..., q+n...).  A unitary has the single K = U. */
static int superop(const orc_op *op, const double *theta, int n, cplx *S, int *pq)
{
    cplx K[256];
    int m, k, s, a, b, c, d;
    if (is_channel(op->kind)) {
        m = channel_kraus_k(op, K, &k);
    } else {
        k = gate_matrix(op, theta, K);
        m = 1;
    }
    if (m < 0 || k < 0) return -1;
    {
        int dk = 1 << k, D = dk * dk;
        for (a = 0; a < D * D; a++) S[a] = 0;
        for (s = 0; s < m; s++)
            for (a = 0; a < dk; a++)          /* r_ket */
                for (b = 0; b < dk; b++)      /* r_bra */
                    for (c = 0; c < dk; c++)  /* c_ket */
                        for (d = 0; d < dk; d++)
                            S[(a + dk * b) * D + (c + dk * d)] +=
                                K[s * dk * dk + a * dk + c] * conj(K[s * dk * dk + b * dk + d]);
    }
    for (a = 0; a < k; a++) { pq[a] = op->q[a]; pq[a + k] = op->q[a] + n; }
    return 2 * k;
}

/* Derivative of the superoperator U (x) conj(U) of a variational FSIM with respect to
 * its parameter comp: dS = dU (x) conj(U) + U (x) conj(dU), 16 x 16 on (ket q0, ket q1,
 * bra q0, bra q1). */
static int superop_derivative_fsim(const orc_op *op, const double *theta, int n, int comp, cplx *dS, int *pq)
{
    cplx U[16], dU[16];
    int a, b, c, d;
    gate_matrix(op, theta, U);
    fsim_derivative(op, theta, comp, dU);
    for (a = 0; a < 4; a++)
        for (b = 0; b < 4; b++)
            for (c = 0; c < 4; c++)
                for (d = 0; d < 4; d++)
                    dS[(a + 4 * b) * 16 + (c + 4 * d)] =
                        dU[a * 4 + c] * conj(U[b * 4 + d]) + U[a * 4 + c] * conj(dU[b * 4 + d]);
    pq[0] = op->q[0];
    pq[1] = op->q[1];
    pq[2] = op->q[0] + n;
    pq[3] = op->q[1] + n;
    return 4;
}

/* Derivative of U (x) conj(U) for a variational single-qubit rotation:
 * dS = dU (x) conj(U) + U (x) conj(dU). */
static int superop_derivative(const orc_op *op, const double *theta, int n, cplx *dS, int *pq)
{
    cplx U[16], dU[16];
    int a, b, c, d;
    if (gate_matrix(op, theta, U) != 1 || gate_derivative(op, theta, dU) != 1) return -1;
    for (a = 0; a < 2; a++)
        for (b = 0; b < 2; b++)
            for (c = 0; c < 2; c++)
                for (d = 0; d < 2; d++)
                    dS[(a + 2 * b) * 4 + (c + 2 * d)] =
                        dU[a * 2 + c] * conj(U[b * 2 + d]) + U[a * 2 + c] * conj(dU[b * 2 + d]);
    pq[0] = op->q[0];
    pq[1] = op->q[0] + n;
    return 2;
}

/* Sec. III.E: L = <<I|H C(theta)|0>> and its gradient by Algorithm 2 on |rho>>:
 * Phi = C|0^{2n}>>, Psi = vec(H) (Psi_ab = H_ab); for j = M..1:
 * Phi <- S_j^{-1} Phi; grads = Re <<Psi|dS_j|Phi>>; Psi <- S_j^dag Psi. */
int orc_noisy_adjoint_grad(int n, const orc_op *ops, int n_ops, const double *theta,
                           int n_params, const double *coeff, const char *paulis, int n_terms,
                           double *energy, double *grad)
{
    int N = 2 * n, j, t, rc = 0;
    int64_t dim = (int64_t)1 << n, len = (int64_t)1 << N, b;
    cplx *phi = (cplx *)calloc((size_t)len, sizeof(cplx));
    cplx *psi = (cplx *)calloc((size_t)len, sizeof(cplx));
    cplx *tmp = (cplx *)malloc(sizeof(cplx) * (size_t)len);
    cplx *eb = (cplx *)calloc((size_t)dim, sizeof(cplx)), *hb = (cplx *)malloc(sizeof(cplx) * (size_t)dim);
    cplx S[256], Sinv[256], Sdag[256];
    int pq[4];
    phi[0] = 1;
    for (j = 0; j < n_ops; j++) {
        int k2 = superop(&ops[j], theta, n, S, pq);
        if (k2 < 0) { rc = -1; goto done; }
        apply_k(phi, N, k2, pq, S);
    }
    /* Psi = vec(H): column b of H is H e_b */
    for (b = 0; b < dim; b++) {
        int64_t a;
        eb[b] = 1;
        for (a = 0; a < dim; a++) psi[a + b * dim] = 0;
        for (t = 0; t < n_terms; t++) {
            pauli_string_apply(hb, eb, n, paulis + (size_t)t * n);
            for (a = 0; a < dim; a++) psi[a + b * dim] += coeff[t] * hb[a];
        }
        eb[b] = 0;
    }
    *energy = creal(inner(psi, phi, len));
    for (j = 0; j < n_params; j++) grad[j] = 0;
    for (j = n_ops - 1; j >= 0; j--) {
        int k2 = superop(&ops[j], theta, n, S, pq), D = 1 << k2, r, c;
        if (k2 < 0 || invert(D, S, Sinv) != 0) { rc = -3; goto done; }
        for (r = 0; r < D; r++)
            for (c = 0; c < D; c++) Sdag[r * D + c] = conj(S[c * D + r]);
        apply_k(phi, N, k2, pq, Sinv);
        if (ops[j].param >= 0 && ops[j].kind == O_FSIM) {  /* one term per variational parameter */
            int b2, r = 0, dq[4];
            for (b2 = 0; b2 < 5; b2++) {
                if (!((ops[j].pmask >> b2) & 1)) continue;
                superop_derivative_fsim(&ops[j], theta, n, b2, S, dq);  /* S reused as scratch */
                memcpy(tmp, phi, sizeof(cplx) * (size_t)len);
                apply_k(tmp, N, 4, dq, S);
                grad[ops[j].param + r++] += creal(inner(psi, tmp, len));
            }
        } else if (ops[j].param >= 0) {
            cplx dS[16];
            int dq[2];
            if (superop_derivative(&ops[j], theta, n, dS, dq) < 0) { rc = -4; goto done; }
            memcpy(tmp, phi, sizeof(cplx) * (size_t)len);
            apply_k(tmp, N, 2, dq, dS);
            grad[ops[j].param] += creal(inner(psi, tmp, len));
        }
        apply_k(psi, N, k2, pq, Sdag);
    }
done:
    free(phi); free(psi); free(tmp); free(eb); free(hb);
    return rc;
}

/* Vectorised noisy evolution with superoperators (used by tests to compare with the
 * Kraus-sum evolution above). */
int orc_vec_apply_circuit(double *vec_, int n, const orc_op *ops, int n_ops, const double *theta)
{
    cplx S[256];
    int pq[4], j;
    for (j = 0; j < n_ops; j++) {
        int k2 = superop(&ops[j], theta, n, S, pq);
        if (k2 < 0) return -1;
        apply_k((cplx *)vec_, 2 * n, k2, pq, S);
    }
    return 0;
}

/* measure!(state, q) (Sec. II.D) on a pure state (density = 0, 2^n amplitudes) or a
 * density matrix (density = 1, rho_ab at a + 2^n b).  P(k) = (sum of |psi_a|^2, or of
 * rho_aa, over a with bit q of a equal to k) / (the same sum over all a).  The outcome
 * is 0 if u < P(0), else 1 (u is the caller's uniform draw in [0, 1)); the state is
 * projected on it and renormalised (pure: psi / sqrt(sum kept); density: P rho P / its
 * trace).  Writes the outcome and its probability. */
int orc_measure(double *state_, int n, int density, int q, double u, int *outcome, double *prob)
{
    cplx *st = (cplx *)state_;
    const int64_t dim = (int64_t)1 << n;
    double s[2] = {0.0, 0.0};
    int64_t a, b;
    if (q < 0 || q >= n) return -1;
    for (a = 0; a < dim; a++) {
        const int bit = (int)((a >> q) & 1);
        if (density) s[bit] += creal(st[a + dim * a]);
        else s[bit] += creal(st[a]) * creal(st[a]) + cimag(st[a]) * cimag(st[a]);
    }
    {
        const double total = s[0] + s[1];
        const int k = u < s[0] / total ? 0 : 1;
        *outcome = k;
        *prob = s[k] / total;
        if (!density) {
            const double scale = 1.0 / sqrt(s[k]);
            for (a = 0; a < dim; a++) st[a] = ((int)((a >> q) & 1) == k) ? st[a] * scale : 0.0;
        } else {
            const double scale = 1.0 / s[k];
            for (b = 0; b < dim; b++)
                for (a = 0; a < dim; a++) {
                    const int keep = (int)((a >> q) & 1) == k && (int)((b >> q) & 1) == k;
                    st[a + dim * b] = keep ? st[a + dim * b] * scale : 0.0;
                }
        }
    }
    return 0;
}

/* Sampling (repeated measurement of every qubit on fresh copies of the state): with
 * w_a = |psi_a|^2 (pure) or rho_aa (density) and the total W, shot s returns the least
 * index a with u_s W < w_0 + ... + w_a (sums in FP64 in index order); u_s in [0, 1) are
 * the caller's uniform draws. */
int orc_sample(const double *state_, int n, int density, const double *u, int n_shots, int64_t *out)
{
    const cplx *st = (const cplx *)state_;
    const int64_t dim = (int64_t)1 << n;
    double *cdf = (double *)malloc(sizeof(double) * (size_t)dim);
    double acc = 0.0;
    int64_t a;
    int s;
    if (!cdf) return -1;
    for (a = 0; a < dim; a++) {
        const cplx v = density ? st[a + dim * a] : st[a];
        acc += density ? creal(v) : creal(v) * creal(v) + cimag(v) * cimag(v);
        cdf[a] = acc;
    }
    for (s = 0; s < n_shots; s++) {
        const double target = u[s] * acc;
        int64_t lo = 0, hi = dim - 1;  /* least a with target < cdf[a] */
        while (lo < hi) {
            const int64_t mid = lo + (hi - lo) / 2;
            if (target < cdf[mid]) hi = mid;
            else lo = mid + 1;
        }
        out[s] = lo;
    }
    free(cdf);
    return 0;
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    extern int omp_get_max_threads(void);
    return omp_get_max_threads();
#else
    return 1;
#endif
}
