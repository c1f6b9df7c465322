// Host-side gate matrices (Sec. II.B), Kraus sets and superoperators (Sec. III.D),
// and the structural classification that picks a gate's sweep.
#include "api_internal.h"

// ------------------------------------------------------------------ host matrices

Mat mat_from(const double *m, int d)
{
    Mat M(d * d);
    for (int i = 0; i < d * d; i++) M[i] = cd(m[2 * i], m[2 * i + 1]);
    return M;
}

void mat_to(const Mat &M, double *m)
{
    for (int i = 0; i < 32; i++) m[i] = 0.0;
    for (size_t i = 0; i < M.size(); i++) {
        m[2 * i] = M[i].real();
        m[2 * i + 1] = M[i].imag();
    }
}

Mat mat_dagger(const Mat &M, int d)
{
    Mat D(d * d);
    for (int r = 0; r < d; r++)
        for (int c = 0; c < d; c++) D[r * d + c] = std::conj(M[c * d + r]);
    return D;
}

Mat mat_conj(const Mat &M)
{
    Mat D(M.size());
    for (size_t i = 0; i < M.size(); i++) D[i] = std::conj(M[i]);
    return D;
}

// Inverse by Gauss-Jordan elimination with partial pivoting (channels are not unitary).
bool mat_inverse(const Mat &A, int d, Mat &out)
{
    std::vector<cd> m(d * 2 * d);
    for (int r = 0; r < d; r++)
        for (int c = 0; c < 2 * d; c++) m[r * 2 * d + c] = c < d ? A[r * d + c] : cd(c - d == r ? 1 : 0);
    for (int k = 0; k < d; k++) {
        int piv = k;
        for (int r = k + 1; r < d; r++)
            if (std::abs(m[r * 2 * d + k]) > std::abs(m[piv * 2 * d + k])) piv = r;
        if (std::abs(m[piv * 2 * d + k]) < 1e-14) return false;
        for (int c = 0; c < 2 * d; c++) std::swap(m[k * 2 * d + c], m[piv * 2 * d + c]);
        cd p = m[k * 2 * d + k];
        for (int c = 0; c < 2 * d; c++) m[k * 2 * d + c] /= p;
        for (int r = 0; r < d; r++)
            if (r != k) {
                cd f = m[r * 2 * d + k];
                for (int c = 0; c < 2 * d; c++) m[r * 2 * d + c] -= f * m[k * 2 * d + c];
            }
    }
    out.assign(d * d, 0);
    for (int r = 0; r < d; r++)
        for (int c = 0; c < d; c++) out[r * d + c] = m[r * 2 * d + d + c];
    return true;
}

bool is_channel(int kind) { return kind >= GBVQC_DEPOL && kind <= GBVQC_KRAUS2; }
bool is_channel2(int kind) { return kind == GBVQC_DEPOL2 || kind == GBVQC_KRAUS2; }
bool is_rotation(int kind) { return kind == GBVQC_RX || kind == GBVQC_RY || kind == GBVQC_RZ; }
int kind_qubits(int kind)
{
    return (kind >= GBVQC_CNOT && kind <= GBVQC_CONTROL) || kind == GBVQC_DENSE2 || is_channel2(kind) ? 2 : 1;
}

// Matrix of a unitary op with its fixed parameters (Sec. II.B); rotations use params[0].
Mat gate_matrix(const gbvqc_op &op)
{
    const double r2 = 1.0 / std::sqrt(2.0);
    const cd I(0, 1);
    if (is_rotation(op.kind)) {
        double m[8];
        rot2(op.kind - GBVQC_RX, VAR_FWD, op.params[0], m);
        return mat_from(m, 2);
    }
    switch (op.kind) {
    case GBVQC_X: return {0, 1, 1, 0};
    case GBVQC_Y: return {0, -I, I, 0};
    case GBVQC_Z: return {1, 0, 0, -1};
    case GBVQC_H: return {r2, r2, r2, -r2};
    case GBVQC_S: return {1, 0, 0, I};
    case GBVQC_T: return {1, 0, 0, std::exp(I * (M_PI / 4))};
    case GBVQC_SX: return {cd(0.5, 0.5), cd(0.5, -0.5), cd(0.5, -0.5), cd(0.5, 0.5)};
    case GBVQC_SY: return {cd(0.5, 0.5), cd(-0.5, -0.5), cd(0.5, 0.5), cd(0.5, 0.5)};
    case GBVQC_SW: return {cd(0.5, 0.5), cd(0, -r2), cd(r2, 0), cd(0.5, 0.5)};
    case GBVQC_DENSE1: return mat_from(op.data, 2);
    default: break;
    }
    Mat M(16, 0);
    auto at = [&](int r, int c) -> cd & { return M[r * 4 + c]; };
    switch (op.kind) {
    case GBVQC_CNOT:  // control = qubits[0] (matrix bit 0), target = qubits[1]
        at(0, 0) = 1; at(2, 2) = 1; at(1, 3) = 1; at(3, 1) = 1;
        break;
    case GBVQC_CZ: at(0, 0) = 1; at(1, 1) = 1; at(2, 2) = 1; at(3, 3) = -1; break;
    case GBVQC_SWAP: at(0, 0) = 1; at(1, 2) = 1; at(2, 1) = 1; at(3, 3) = 1; break;
    case GBVQC_ISWAP: at(0, 0) = 1; at(1, 2) = I; at(2, 1) = I; at(3, 3) = 1; break;
    case GBVQC_FSIM: {  // Eq. (FSIM)
        double th = op.params[0], ph = op.params[1], dp = op.params[2], dm = op.params[3],
               dmo = op.params[4];
        at(0, 0) = 1;
        at(1, 1) = std::exp(I * (dp + dm)) * std::cos(th);
        at(1, 2) = -I * std::exp(I * (dp - dmo)) * std::sin(th);
        at(2, 1) = -I * std::exp(I * (dp + dmo)) * std::sin(th);
        at(2, 2) = std::exp(I * (dp - dm)) * std::cos(th);
        at(3, 3) = std::exp(I * (2 * dp - ph));
        break;
    }
    case GBVQC_CONTROL:
        at(0, 0) = 1; at(2, 2) = 1;
        at(1, 1) = cd(op.data[0], op.data[1]);
        at(1, 3) = cd(op.data[2], op.data[3]);
        at(3, 1) = cd(op.data[4], op.data[5]);
        at(3, 3) = cd(op.data[6], op.data[7]);
        break;
    case GBVQC_DENSE2: return mat_from(op.data, 4);
    default: break;
    }
    return M;
}

// Kraus operators of a single-qubit channel (Sec. II.B; depolarising with p/4 weights).
std::vector<Mat> channel_kraus(int kind, double g, const double *kraus, int n_kraus)
{
    const cd I(0, 1);
    switch (kind) {
    case GBVQC_AMPDAMP: return {{1, 0, 0, std::sqrt(1 - g)}, {0, std::sqrt(g), 0, 0}};
    case GBVQC_PHASEDAMP: return {{1, 0, 0, std::sqrt(1 - g)}, {0, 0, 0, std::sqrt(g)}};
    case GBVQC_DEPOL: {
        double a = std::sqrt(1 - 0.75 * g), b = std::sqrt(0.25 * g);
        return {{a, 0, 0, a}, {0, b, b, 0}, {0, -I * b, I * b, 0}, {b, 0, 0, -b}};
    }
    default: {
        std::vector<Mat> ks;
        for (int s = 0; s < n_kraus; s++) ks.push_back(mat_from(kraus + 8 * s, 2));
        return ks;
    }
    }
}

// Kraus operators (4x4, matrix bit 0 = the first qubit) of a two-qubit channel.
std::vector<Mat> channel_kraus2(int kind, double g, const double *kraus, int n_kraus)
{
    std::vector<Mat> ks;
    if (kind == GBVQC_KRAUS2) {
        for (int s = 0; s < n_kraus; s++) ks.push_back(mat_from(kraus + 32 * s, 4));
        return ks;
    }
    const cd I(0, 1);
    const cd P[4][4] = {{1, 0, 0, 1}, {0, 1, 1, 0}, {0, -I, I, 0}, {1, 0, 0, -1}};  // I, X, Y, Z
    for (int b = 0; b < 4; b++)      // Pauli on the second qubit
        for (int a = 0; a < 4; a++) {  // Pauli on the first qubit
            const double w = (a == 0 && b == 0) ? std::sqrt(1 - 15 * g / 16) : std::sqrt(g / 16);
            Mat K(16, 0);
            for (int r = 0; r < 4; r++)
                for (int c = 0; c < 4; c++)
                    K[r * 4 + c] = w * P[a][2 * (r & 1) + (c & 1)] * P[b][2 * (r >> 1) + (c >> 1)];
            ks.push_back(K);
        }
    return ks;
}

// Superoperator of a two-qubit channel on (ket q0, ket q1, bra q0, bra q1) (matrix bits
// 0..3): S[(r + 4 r'), (c + 4 c')] = sum_s K[r][c] conj(K[r'][c']), 16 x 16.
Mat superop2(const std::vector<Mat> &ks)
{
    Mat S(256, 0);
    for (const Mat &K : ks)
        for (int r = 0; r < 4; r++)
            for (int r2 = 0; r2 < 4; r2++)
                for (int c = 0; c < 4; c++)
                    for (int c2 = 0; c2 < 4; c2++)
                        S[(r + 4 * r2) * 16 + (c + 4 * c2)] += K[r * 4 + c] * std::conj(K[r2 * 4 + c2]);
    return S;
}

// Superoperator on (ket q, bra q): S[(r1 + 2 r2), (c1 + 2 c2)] = sum_s K[r1][c1] conj(K[r2][c2])
// (Eq. channel2 with the conjugate on the bra index: vec(K rho K^dag)).
Mat superop(const std::vector<Mat> &ks)
{
    Mat S(16, 0);
    for (const Mat &K : ks)
        for (int r1 = 0; r1 < 2; r1++)
            for (int r2 = 0; r2 < 2; r2++)
                for (int c1 = 0; c1 < 2; c1++)
                    for (int c2 = 0; c2 < 2; c2++)
                        S[(r1 + 2 * r2) * 4 + (c1 + 2 * c2)] += K[r1 * 2 + c1] * std::conj(K[r2 * 2 + c2]);
    return S;
}

static bool nz(cd v) { return v.real() != 0.0 || v.imag() != 0.0; }

int classify(const Mat &M)
{
    if (M.size() == 4) {
        if (!nz(M[1]) && !nz(M[2])) return SH_DIAG1;
        if (!nz(M[0]) && !nz(M[3])) return SH_ANTI1;
        bool real = true;
        for (cd v : M) real = real && v.imag() == 0.0;
        if (real) return SH_REAL1;
        const bool imag = M[0].imag() == 0.0 && M[3].imag() == 0.0 && M[1].real() == 0.0 && M[2].real() == 0.0;
        return imag ? SH_IMAG1 : SH_DENSE1;
    }
    bool diag = true;
    for (int r = 0; r < 4; r++)
        for (int c = 0; c < 4; c++)
            if (r != c && nz(M[r * 4 + c])) diag = false;
    if (diag) return M[0] == cd(1) && M[5] == cd(1) && M[10] == cd(1) && M[15] == cd(-1) ? SH_CZ : SH_DIAG2;
    // exactly CNOT with the first qubit as control (rows 1 and 3 swapped, unit entries)
    if (M[0] == cd(1) && M[10] == cd(1) && M[7] == cd(1) && M[13] == cd(1)) {
        int others = 0;
        for (int i = 0; i < 16; i++) others += nz(M[i]);
        if (others == 4) return SH_CX;
    }
    // controlled: identity on the q0 = 0 block (indices 0, 2), no coupling to 1, 3
    bool ctrl = M[0] == cd(1) && M[10] == cd(1) && !nz(M[2]) && !nz(M[8]);
    for (int r : {0, 2})
        for (int c : {1, 3}) ctrl = ctrl && !nz(M[r * 4 + c]) && !nz(M[c * 4 + r]);
    if (ctrl) return SH_CTRL2;
    bool perm = true;
    for (int r = 0; r < 4 && perm; r++) {
        int cnt = 0, cntc = 0;
        for (int c = 0; c < 4; c++) {
            cnt += nz(M[r * 4 + c]);
            cntc += nz(M[c * 4 + r]);
        }
        perm = cnt == 1 && cntc == 1;
    }
    if (perm) return SH_PERM2;
    // block: only (0,0), (3,3) and the 2x2 on rows/columns {1, 2} are non-zero
    bool block = true;
    for (int r = 0; r < 4; r++)
        for (int c = 0; c < 4; c++) {
            const bool inside = (r == c && (r == 0 || r == 3)) || ((r == 1 || r == 2) && (c == 1 || c == 2));
            if (!inside && nz(M[r * 4 + c])) block = false;
        }
    if (block) return SH_BLOCK2;
    // parity-preserving: entry (r, c) is zero unless r ^ c is 0 or 3, i.e. |00> couples
    // only to |11> and |01> only to |10>
    bool par = true, real = true;
    for (int r = 0; r < 4; r++)
        for (int c = 0; c < 4; c++) {
            if (((r ^ c) == 1 || (r ^ c) == 2) && nz(M[r * 4 + c])) par = false;
            real = real && M[r * 4 + c].imag() == 0.0;
        }
    if (par) return real ? SH_RPAR2 : SH_PAR2;
    return SH_DENSE2;
}

int perm_bits(const Mat &M)
{
    int bits = 0;
    for (int r = 0; r < 4; r++)
        for (int c = 0; c < 4; c++)
            if (nz(M[r * 4 + c])) bits |= c << (2 * r);
    return bits;
}

// Shape that covers two matrices (reverse sweeps apply different matrices to Phi, Psi).
int join_shape(int a, int b)
{
    if (a == b) return a;
    if (shape_qubits(a) == 1) return SH_DENSE1;
    auto par = [](int s) { return s == SH_DIAG2 || s == SH_BLOCK2 || s == SH_PAR2 || s == SH_RPAR2; };
    return par(a) && par(b) ? SH_PAR2 : SH_DENSE2;
}

int ftype_of(int sh)
{
    switch (sh) {
    case SH_DENSE1: return FT_DENSE1;
    case SH_REAL1: return FT_REAL1;
    case SH_ANTI1: return FT_ANTI1;
    case SH_DIAG1: return FT_DIAG1;
    case SH_DENSE2: return FT_DENSE2;
    case SH_DIAG2: return FT_DIAG2;
    case SH_PERM2: return FT_PERM2;
    case SH_BLOCK2: return FT_BLOCK2;
    case SH_IMAG1: return FT_IMAG1;
    case SH_CZ: return FT_DIAG2;
    case SH_PAR2: return FT_PAR2;
    case SH_RPAR2: return FT_RPAR2;
    default: return FT_CTRL2;
    }
}
