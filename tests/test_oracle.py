"""Pins of the FP64 CPU oracle against what the paper and mathematics fix.

Every check compares the oracle with something other than itself: closed forms,
scipy's matrix exponential, dense numpy Kronecker products, hand-derived values of
the paper's Listing 4, invariants, parameter shift and finite differences.
"""
import math
import os

import numpy as np
import pytest
import scipy.linalg

from oracle import oracle as O
from paper_2406_19212_gb300 import inputs as I
from tests.dense_ref import PAULI, embed, pauli_operator

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def op(name, qubits, param=-1, fixed=(), data=None, pmask=0):
    return I.Op(name, tuple(qubits), param, tuple(fixed), data, pmask)


# ----------------------------------------------------------------- gate matrices

@pytest.mark.parametrize("t", [0.0, 0.3, 1.7, -2.9, 5.5])
def test_rotations_are_pauli_exponentials(t):
    # Sec. II.B: Rx, Ry, Rz == exp(-i t P / 2) (Ry and Rz per the readings of the garbles)
    for name, P in (("RX", "X"), ("RY", "Y"), ("RZ", "Z")):
        M = O.gate_matrix(op(name, (0,), fixed=(t,)))
        np.testing.assert_allclose(M, scipy.linalg.expm(-0.5j * t * PAULI[P]), atol=1e-15)


@pytest.mark.parametrize("t", [0.0, 0.4, 2.2, 4.0])
def test_rotation_expectation_closed_forms(t):
    z0 = O.zero_state(1)
    Z = [(1.0, ((0, "Z"),))]
    X = [(1.0, ((0, "X"),))]
    c = I.Circuit(1, [op("RX", (0,), fixed=(t,))], 0)
    assert O.expect(Z, O.apply_circuit(c, []), 1) == pytest.approx(math.cos(t), abs=1e-15)
    c = I.Circuit(1, [op("RY", (0,), fixed=(t,))], 0)
    psi = O.apply_circuit(c, [])
    assert O.expect(Z, psi, 1) == pytest.approx(math.cos(t), abs=1e-15)
    assert O.expect(X, psi, 1) == pytest.approx(math.sin(t), abs=1e-15)
    c = I.Circuit(1, [op("H", (0,)), op("RZ", (0,), fixed=(t,))], 0)
    assert O.expect(X, O.apply_circuit(c, []), 1) == pytest.approx(math.cos(t), abs=1e-15)
    assert z0[0] == 1


def test_fixed_gates_textbook():
    r = 1 / math.sqrt(2)
    np.testing.assert_allclose(O.gate_matrix(op("H", (0,))), [[r, r], [r, -r]], atol=1e-16)
    np.testing.assert_allclose(O.gate_matrix(op("S", (0,))), [[1, 0], [0, 1j]], atol=1e-16)
    np.testing.assert_allclose(O.gate_matrix(op("T", (0,))),
                               [[1, 0], [0, np.exp(1j * np.pi / 4)]], atol=1e-16)
    for name in "XYZ":
        np.testing.assert_allclose(O.gate_matrix(op(name, (0,))), PAULI[name], atol=0)
    W = (PAULI["X"] + PAULI["Y"]) / math.sqrt(2)
    for name, G in (("SX", PAULI["X"]), ("SY", PAULI["Y"]), ("SW", W)):
        M = O.gate_matrix(op(name, (0,)))
        np.testing.assert_allclose(M @ M, G, atol=1e-15)          # square root
        np.testing.assert_allclose(M, scipy.linalg.sqrtm(G), atol=1e-12)  # principal root
        np.testing.assert_allclose(M.conj().T @ M, np.eye(2), atol=1e-15)


def _basis_map(name, n=2):
    """Gate action on computational basis states |b0 b1> (index b0 + 2 b1)."""
    M = O.gate_matrix(op(name, (0, 1)))
    return {c: {r: M[r, c] for r in range(4) if M[r, c] != 0} for c in range(4)}


def test_two_qubit_gate_semantics():
    # CNOT(control q0, target q1): flips q1 when q0 = 1
    m = _basis_map("CNOT")
    assert m == {0: {0: 1}, 1: {3: 1}, 2: {2: 1}, 3: {1: 1}}
    assert _basis_map("CZ") == {0: {0: 1}, 1: {1: 1}, 2: {2: 1}, 3: {3: -1}}
    assert _basis_map("SWAP") == {0: {0: 1}, 1: {2: 1}, 2: {1: 1}, 3: {3: 1}}
    assert _basis_map("ISWAP") == {0: {0: 1}, 1: {2: 1j}, 2: {1: 1j}, 3: {3: 1}}
    # CONTROL with X as the target block is CNOT
    ctl = O.gate_matrix(op("CONTROL", (0, 1), data=PAULI["X"]))
    np.testing.assert_allclose(ctl, O.gate_matrix(op("CNOT", (0, 1))), atol=0)


def test_fsim_special_cases():
    # Eq. (FSIM): fsim(pi/2, 0) = iSWAP^dag; fsim(0, phi) = diag(1, 1, 1, e^{-i phi})
    F = O.gate_matrix(op("FSIM", (0, 1), fixed=(math.pi / 2, 0.0)))
    iswap = O.gate_matrix(op("ISWAP", (0, 1)))
    np.testing.assert_allclose(F, iswap.conj().T, atol=1e-15)
    F = O.gate_matrix(op("FSIM", (0, 1), fixed=(0.0, 0.7)))
    np.testing.assert_allclose(F, np.diag([1, 1, 1, np.exp(-0.7j)]), atol=1e-15)
    rng = np.random.default_rng(5)
    for _ in range(5):
        F = O.gate_matrix(op("FSIM", (0, 1), fixed=tuple(rng.uniform(-3, 3, 5))))
        np.testing.assert_allclose(F.conj().T @ F, np.eye(4), atol=1e-14)
    # theta, phi part is exp(-i theta (XX+YY)/2) followed by the |11> phase
    th = 0.83
    XXYY = np.kron(PAULI["X"], PAULI["X"]) + np.kron(PAULI["Y"], PAULI["Y"])
    F = O.gate_matrix(op("FSIM", (0, 1), fixed=(th, 0.0)))
    np.testing.assert_allclose(F, scipy.linalg.expm(-0.5j * th * XXYY), atol=1e-14)


def _zphase_layer(a0, a1):
    """exp(i (a0 n0 + a1 n1)) on two qubits, n_k the excitation number of qubit k
    (basis index = bit(q0) + 2 bit(q1)): a single-qubit Z rotation on each qubit, up to
    a global phase."""
    return np.diag([1.0, np.exp(1j * a0), np.exp(1j * a1), np.exp(1j * (a0 + a1))])


def test_fsim_delta_entries_from_single_qubit_phases():
    """Pin of the Delta entries of Eq. (FSIM), built from physics rather than from the
    printed entries.  The five-parameter FSIM is the (theta, phi) core
    C = exp(-i theta (XX+YY)/2) diag(1, 1, 1, e^{-i phi}) between two layers of single-qubit
    Z phases, D(a) C D(b) with D(a) = exp(i (a0 n0 + a1 n1)).  In the single-excitation
    block D(a) C D(b) carries the phases a_i + b_j on entry (i, j) (i, j = 0 for |10>, 1
    for |01>):
      - Delta_+ is their mean over the diagonal, (a0 + b0 + a1 + b1) / 2;
      - Delta_- is half the difference of the two diagonal phases, ((a0 + b0) - (a1 + b1)) / 2;
      - Delta_-,off is half the difference of the two off-diagonal phases,
        ((a1 + b0) - (a0 + b1)) / 2;
    and |11> collects a0 + a1 + b0 + b1 = 2 Delta_+ on top of the core's e^{-i phi}.
    So, for random a, b, theta, phi, the oracle's FSIM at those Deltas must equal
    D(a) C D(b) exactly: a sign slip between the off-diagonal entries, between the
    diagonal ones, or Delta_+ in place of 2 Delta_+ on |11> fails here."""
    rng = np.random.default_rng(11)
    XXYY = np.kron(PAULI["X"], PAULI["X"]) + np.kron(PAULI["Y"], PAULI["Y"])
    for _ in range(8):
        th, ph = rng.uniform(-3, 3, 2)
        a0, a1, b0, b1 = rng.uniform(-3, 3, 4)
        core = scipy.linalg.expm(-0.5j * th * XXYY) @ np.diag([1, 1, 1, np.exp(-1j * ph)])
        want = _zphase_layer(a0, a1) @ core @ _zphase_layer(b0, b1)
        dp = (a0 + b0 + a1 + b1) / 2
        dm = ((a0 + b0) - (a1 + b1)) / 2
        dmo = ((a1 + b0) - (a0 + b1)) / 2
        assert len({round(v, 6) for v in (th, ph, dp, dm, dmo)}) == 5
        F = O.gate_matrix(op("FSIM", (0, 1), fixed=(th, ph, dp, dm, dmo)))
        np.testing.assert_allclose(F, want, atol=1e-14, rtol=0)


@pytest.mark.parametrize("name,strength", [("DEPOL", 0.13), ("AMPDAMP", 0.21),
                                           ("PHASEDAMP", 0.4)])
def test_kraus_completeness(name, strength):
    ks = O.kraus(op(name, (0,), fixed=(strength,)))
    np.testing.assert_allclose(sum(k.conj().T @ k for k in ks), np.eye(2), atol=1e-15)


# ------------------------------------------------------------- state evolution

@pytest.mark.parametrize("n,seed", [(1, 0), (2, 1), (3, 2), (4, 3), (5, 4), (6, 5)])
def test_circuit_matches_dense_kronecker(n, seed):
    w = I.random_circuit(n, 40, seed)
    U = np.eye(1 << n, dtype=complex)
    for o in w.circuit.ops:
        U = embed(O.gate_matrix(o, w.theta), o.qubits, n) @ U
    psi = O.apply_circuit(w.circuit, w.theta)
    np.testing.assert_allclose(psi, U[:, 0], atol=1e-13)
    start = I.random_state(n, seed + 100)
    np.testing.assert_allclose(O.apply_circuit(w.circuit, w.theta, start), U @ start, atol=1e-13)


@pytest.mark.parametrize("n", [1, 2, 5, 12])
def test_ghz_closed_form(n):
    ops = [op("H", (0,))] + [op("CNOT", (i, i + 1)) for i in range(n - 1)]
    psi = O.apply_circuit(I.Circuit(n, ops, 0), [])
    ref = np.zeros(1 << n, dtype=complex)
    ref[0] = ref[-1] = 1 / math.sqrt(2)
    np.testing.assert_allclose(psi, ref, atol=1e-15)


def qft_ops(n):
    ops = []
    for i in range(1, n + 1):
        t = n - i
        ops.append(op("H", (t,)))
        for j in range(i + 1, n + 1):
            ang = 2 * math.pi / 2 ** (j - i + 1)
            ops.append(op("CONTROL", (n - j, t), data=np.diag([1, np.exp(1j * ang)])))
    for i in range(1, n // 2 + 1):
        ops.append(op("SWAP", (n - i, i - 1)))
    return ops


@pytest.mark.parametrize("n,x", [(3, 5), (5, 19), (8, 201)])
def test_qft_closed_form(n, x):
    psi0 = np.zeros(1 << n, dtype=complex)
    psi0[x] = 1
    psi = O.apply_circuit(I.Circuit(n, qft_ops(n), 0), [], psi0)
    y = np.arange(1 << n)
    np.testing.assert_allclose(psi, np.exp(2j * np.pi * x * y / 2 ** n) / 2 ** (n / 2), atol=1e-13)


def _golden(name):
    vals = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                k, expr = line.split(None, 1)
                vals[k] = eval(expr, {"math": math})
    return vals


def test_listing4_golden():
    g = _golden("listing4.txt")
    c = I.Circuit(2, [op("H", (0,)), op("RY", (0,), fixed=(math.pi / 4,)),
                      op("CNOT", (0, 1))], 0)
    psi = O.apply_circuit(c, [])
    for i in range(4):
        assert psi[i].real == pytest.approx(g[f"amp_re_{i}"], abs=1e-15)
        assert psi[i].imag == pytest.approx(g[f"amp_im_{i}"], abs=1e-15)
    p0 = abs(psi[0]) ** 2 + abs(psi[1]) ** 2
    assert p0 == pytest.approx(g["prob_q1_0"], abs=1e-15)
    assert 1 - p0 == pytest.approx(g["prob_q1_1"], abs=1e-15)


def test_norm_preserved_and_inverse():
    w = I.random_circuit(10, 200, 7)
    psi = O.apply_circuit(w.circuit, w.theta)
    assert np.linalg.norm(psi) == pytest.approx(1.0, abs=1e-13)


# ----------------------------------------------------------------- expectation

@pytest.mark.parametrize("n,seed", [(1, 0), (3, 1), (5, 2), (6, 3)])
def test_expectation_matches_dense(n, seed):
    w = I.random_circuit(n, 10, seed)
    terms = w.observable + I.heisenberg_1d(n) if n > 1 else w.observable
    psi = I.random_state(n, seed)
    H = pauli_operator(terms, n)
    e, im = O.expect(terms, psi, n, return_imag=True)
    assert e == pytest.approx((psi.conj() @ H @ psi).real, abs=1e-13)
    assert abs(im) < 1e-13
    np.testing.assert_allclose(O.apply_hamiltonian(terms, psi, n), H @ psi, atol=1e-13)


# -------------------------------------------------------------------- gradients

@pytest.mark.parametrize("n,seed,share", [(3, 11, False), (5, 12, True), (6, 13, False)])
def test_adjoint_matches_parameter_shift(n, seed, share):
    w = I.random_circuit(n, 60, seed, param_share=share)
    e, g = O.adjoint_grad(w.circuit, w.theta, w.observable)
    assert e == pytest.approx(O.energy(w.circuit, w.theta, w.observable), abs=1e-13)
    ps = O.parameter_shift_grad(w.circuit, w.theta, w.observable)
    np.testing.assert_allclose(g, ps, atol=1e-12)


def test_adjoint_matches_finite_difference_plain10():
    w = I.plain_10q()
    e, g = O.adjoint_grad(w.circuit, w.theta, w.observable)
    idx = [0, 13, 57, 119]
    fd = O.finite_difference_grad(w.circuit, w.theta, w.observable, idx, h=1e-5)
    np.testing.assert_allclose(g[idx], fd, atol=1e-8)


# --------------------------------------------------------------------- density

def test_single_qubit_channel_closed_forms():
    rng = np.random.default_rng(3)
    rho = I.random_density(1, 9).reshape(2, 2, order="F")
    vec = rho.reshape(-1, order="F")
    p, g = 0.23, 0.31
    out = O.rho_apply_circuit(I.Circuit(1, [op("DEPOL", (0,), fixed=(p,))], 0, True), [], vec)
    np.testing.assert_allclose(out.reshape(2, 2, order="F"),
                               (1 - p) * rho + p * np.trace(rho) * np.eye(2) / 2, atol=1e-15)
    one = np.array([0, 0, 0, 1], dtype=complex)          # |1><1|
    out = O.rho_apply_circuit(I.Circuit(1, [op("AMPDAMP", (0,), fixed=(g,))], 0, True), [], one)
    np.testing.assert_allclose(out, [g, 0, 0, 1 - g], atol=1e-15)
    out = O.rho_apply_circuit(I.Circuit(1, [op("PHASEDAMP", (0,), fixed=(g,))], 0, True), [], vec)
    r = out.reshape(2, 2, order="F")
    np.testing.assert_allclose(np.diag(r), np.diag(rho), atol=1e-15)
    np.testing.assert_allclose(r[0, 1], rho[0, 1] * math.sqrt(1 - g), atol=1e-15)
    assert rng is not None


@pytest.mark.parametrize("n,seed", [(1, 1), (2, 2), (3, 3)])
def test_density_matches_dense_matrices(n, seed):
    w = I.random_circuit(n, 25, seed, density=True, with_channels=True)
    rho = I.random_density(n, seed).reshape(1 << n, 1 << n, order="F")
    ref = rho.copy()
    for o in w.circuit.ops:
        if o.name in I.CHANNELS:
            ks = [embed(k, o.qubits, n) for k in O.kraus(o)]
            ref = sum(k @ ref @ k.conj().T for k in ks)
        else:
            U = embed(O.gate_matrix(o, w.theta), o.qubits, n)
            ref = U @ ref @ U.conj().T
    out = O.rho_apply_circuit(w.circuit, w.theta, rho.reshape(-1, order="F"))
    np.testing.assert_allclose(out, ref.reshape(-1, order="F"), atol=1e-13)
    vec = O.vec_apply_circuit(w.circuit, w.theta, rho.reshape(-1, order="F"))
    np.testing.assert_allclose(vec, ref.reshape(-1, order="F"), atol=1e-13)
    H = pauli_operator(w.observable, n)
    e, im = O.rho_expect(w.observable, out, n, return_imag=True)
    assert e == pytest.approx(np.trace(H @ ref).real, abs=1e-13)
    assert abs(im) < 1e-13


def test_unitary_density_equals_pure_projector():
    w = I.random_circuit(4, 50, 21)
    psi = O.apply_circuit(w.circuit, w.theta)
    rho = O.rho_apply_circuit(I.Circuit(4, w.circuit.ops, w.circuit.n_params, True), w.theta)
    np.testing.assert_allclose(rho, np.outer(psi, psi.conj()).reshape(-1, order="F"), atol=1e-14)


def test_noisy_trace_hermitian_positive():
    w = I.noisy_hea(4, 3, 5)
    rho = O.rho_apply_circuit(w.circuit, w.theta).reshape(16, 16, order="F")
    assert np.trace(rho).real == pytest.approx(1.0, abs=1e-14)
    np.testing.assert_allclose(rho, rho.conj().T, atol=1e-15)
    assert np.linalg.eigvalsh(rho).min() > -1e-14


@pytest.mark.parametrize("n,seed", [(2, 31), (3, 32)])
def test_noisy_adjoint_matches_parameter_shift(n, seed):
    w = I.random_circuit(n, 30, seed, density=True, with_channels=True)
    e, g = O.noisy_adjoint_grad(w.circuit, w.theta, w.observable)
    assert e == pytest.approx(O.energy(w.circuit, w.theta, w.observable), abs=1e-13)
    ps = O.parameter_shift_grad(w.circuit, w.theta, w.observable)
    np.testing.assert_allclose(g, ps, atol=1e-12)


def test_noisy_hea_adjoint_matches_shift():
    w = I.noisy_hea(3, 2, 8, p1=0.05, p2=0.1, gamma=0.07)
    e, g = O.noisy_adjoint_grad(w.circuit, w.theta, w.observable)
    ps = O.parameter_shift_grad(w.circuit, w.theta, w.observable)
    np.testing.assert_allclose(g, ps, atol=1e-12)


# ----------------------------------------------------------------- measurement

def test_measure_listing4_golden():
    """measure!(state, 2) of the paper's Listing 4: outcome probabilities derived by hand
    (tests/golden/listing4.txt) and the collapsed states |00> or |11>."""
    g = _golden("listing4.txt")
    c = I.Circuit(2, [op("H", (0,)), op("RY", (0,), fixed=(math.pi / 4,)),
                      op("CNOT", (0, 1))], 0)
    psi = O.apply_circuit(c, [])
    k, p, post = O.measure(psi, 2, 1, 0.1)
    assert k == 0 and p == pytest.approx(g["prob_q1_0"], abs=1e-15)
    np.testing.assert_allclose(post, [1, 0, 0, 0], atol=1e-15)
    k, p, post = O.measure(psi, 2, 1, 0.9)
    assert k == 1 and p == pytest.approx(g["prob_q1_1"], abs=1e-15)
    np.testing.assert_allclose(post, [0, 0, 0, 1], atol=1e-15)


def test_measure_ghz_closed_form():
    n = 6
    ops = [op("H", (0,))] + [op("CNOT", (i, i + 1)) for i in range(n - 1)]
    psi = O.apply_circuit(I.Circuit(n, ops, 0), [])
    for u, k_ref, idx in ((0.3, 0, 0), (0.7, 1, (1 << n) - 1)):
        k, p, post = O.measure(psi, n, 3, u)
        assert k == k_ref and p == pytest.approx(0.5, abs=1e-15)
        ref = np.zeros(1 << n, complex)
        ref[idx] = 1.0
        np.testing.assert_allclose(post, ref, atol=1e-15)


def test_measure_density_matches_pure():
    """On rho = |psi><psi| the density branch gives the same outcome and probability and
    the projector of the pure branch's collapsed state (two independent code paths)."""
    n = 5
    w = I.random_circuit(n, 60, 13)
    psi = O.apply_circuit(w.circuit, w.theta)
    rho = np.outer(psi, psi.conj())
    vec = rho.T.reshape(-1)  # rho_ab at a + 2^n b
    for q, u in ((0, 0.2), (3, 0.42), (4, 0.97)):
        k1, p1, post = O.measure(psi, n, q, u)
        k2, p2, post_rho = O.measure(vec, n, q, u, density=True)
        assert k1 == k2 and p1 == pytest.approx(p2, abs=1e-13)
        np.testing.assert_allclose(post_rho, np.outer(post, post.conj()).T.reshape(-1), atol=1e-13)
        assert np.linalg.norm(post) == pytest.approx(1.0, abs=1e-13)
        # the collapsed state lives on the outcome's half and keeps the kept amplitudes' ratios
        idx = np.arange(1 << n)
        assert np.all(post[((idx >> q) & 1) != k1] == 0)
        kept = ((idx >> q) & 1) == k1
        np.testing.assert_allclose(post[kept] * math.sqrt(p1), psi[kept], atol=1e-13)


# ----------------------------------------------------- variational FSIM (five parameters)

def test_fsim_derivative_matches_matrix_differences():
    """The oracle's analytic dFSIM/dp_k against central differences of the matrix."""
    vals = [1.1, 0.7, 0.3, -0.2, 0.45]
    for k in range(5):
        c = I.Circuit(2, [op("FSIM", (0, 1), param=0, fixed=tuple(vals), pmask=1 << k)], 1)
        h = 1e-6
        Mp = O.gate_matrix(I.Op("FSIM", (0, 1), fixed=tuple(v + (h if i == k else 0) for i, v in enumerate(vals))))
        Mm = O.gate_matrix(I.Op("FSIM", (0, 1), fixed=tuple(v - (h if i == k else 0) for i, v in enumerate(vals))))
        # gradient of <psi|H|psi> for a single FSIM on a fixed input, two ways
        psi0 = I.random_state(2, 3 + k)
        terms = [(0.8, ((0, "X"), (1, "Y"))), (-0.3, ((1, "Z"),)), (0.5, ((0, "Y"),))]
        Hm = pauli_operator(terms, 2)
        fd = ((Mp @ psi0).conj() @ Hm @ (Mp @ psi0) - (Mm @ psi0).conj() @ Hm @ (Mm @ psi0)).real / (2 * h)
        prep = [op("DENSE2", (0, 1), data=_prep_unitary(psi0))]
        c2 = I.Circuit(2, prep + c.ops, 1)
        _, g = O.adjoint_grad(c2, [vals[k]], terms)
        assert g[0] == pytest.approx(fd, abs=1e-7)


def _prep_unitary(psi0):
    """A unitary whose first column is psi0 (Householder-style via QR)."""
    A = np.random.default_rng(0).normal(size=(4, 4)) + 1j * np.random.default_rng(1).normal(size=(4, 4))
    A[:, 0] = psi0
    Q, R = np.linalg.qr(A)
    Q[:, 0] *= R[0, 0] / abs(R[0, 0])
    assert np.allclose(Q[:, 0], psi0)
    return Q


def test_fsim_grad_shift_rules_and_fd():
    """Variational FSIM on a 3x3 grid circuit.  theta: its generator (XX+YY)/2 has
    eigenvalues -1, 0, 0, 1, so the loss holds frequencies 1 and 2 in theta and the exact
    four-term rule f' = (1 - sqrt2)/2 [f(+pi/2) - f(-pi/2)] + [f(+pi/4) - f(-pi/4)] applies
    (solving 2 c1 sin(w s1) + 2 c2 sin(w s2) = w for w = 1, 2); phi: generator |11><11|
    (eigenvalues 0, 1), the two-term +-pi/2 rule; the Delta's by central differences."""
    w = I.fsim_grid_vqe(3, 3, 4, 7, pmask=0b11111)
    e, g = O.adjoint_grad(w.circuit, w.theta, w.observable)
    assert e == pytest.approx(O.energy(w.circuit, w.theta, w.observable), abs=1e-12)
    L = lambda th: O.energy(w.circuit, th, w.observable)
    for j in range(0, w.circuit.n_params, 3):
        comp = j % 5  # parameters of a gate are consecutive: k = j mod 5 with all bits set
        t = np.array(w.theta, dtype=float)
        if comp == 0:
            def shift(s):
                tp, tm = t.copy(), t.copy(); tp[j] += s; tm[j] -= s
                return L(tp) - L(tm)
            ref = (1 - math.sqrt(2)) / 2 * shift(np.pi / 2) + shift(np.pi / 4)
        elif comp == 1:
            tp, tm = t.copy(), t.copy(); tp[j] += np.pi / 2; tm[j] -= np.pi / 2
            ref = 0.5 * (L(tp) - L(tm))
        else:
            ref = O.finite_difference_grad(w.circuit, t, w.observable, [j], h=1e-5)[0]
        assert g[j] == pytest.approx(ref, abs=1e-8 if comp < 2 else 1e-7)


# ------------------------------------------------------------- two-qubit channels

def _partial_trace_pair(rho, n, qa, qb):
    """Tr over qubits qa, qb of a 2^n x 2^n matrix, embedded back as X (x) I_{qa,qb}/... :
    returns sum_{s} (<s| on qa,qb) rho (|s>) expanded with the identity on qa, qb."""
    d = 1 << n
    out = np.zeros_like(rho)
    idx = np.arange(d)
    mask = (1 << qa) | (1 << qb)
    for a in range(d):
        for b in range(d):
            if (a & mask) != (b & mask):
                continue
            # (Tr_{qa,qb} rho)[a without qa,qb; b without qa,qb] = sum over s of rho[a|s, b|s]
            s = 0.0
            for t in range(4):
                bits = ((t & 1) << qa) | (((t >> 1) & 1) << qb)
                s += rho[(a & ~mask) | bits, (b & ~mask) | bits]
            out[a, b] = s
    return out


def test_depol2_closed_form():
    """Two-qubit depolarising (reading: K0 = sqrt(1-15p/16) I, the 15 others sqrt(p/16)
    s_a (x) s_b) gives (1-p) rho + p/4 Tr_{q0 q1}(rho) (x) I on the pair."""
    n, p = 3, 0.23
    rho = I.random_density(n, 4).reshape(1 << n, 1 << n, order="F")
    c = I.Circuit(n, [op("DEPOL2", (0, 2), fixed=(p,))], 0, True)
    out = O.rho_apply_circuit(c, [], rho.reshape(-1, order="F")).reshape(1 << n, 1 << n, order="F")
    ref = (1 - p) * rho + p / 4 * _partial_trace_pair(rho, n, 0, 2)
    np.testing.assert_allclose(out, ref, atol=1e-14)
    ks = O.kraus(op("DEPOL2", (0, 2), fixed=(p,)))
    assert len(ks) == 16 and ks[0].shape == (4, 4)
    np.testing.assert_allclose(sum(k.conj().T @ k for k in ks), np.eye(4), atol=1e-14)


@pytest.mark.parametrize("seed", [1, 2])
def test_kraus2_density_against_dense_and_superoperator(seed):
    """General two-qubit Kraus channels inside a noisy circuit: the Kraus-sum evolution
    equals dense K rho K^dag products, and the superoperator evolution equals both."""
    n = 3
    rng = np.random.default_rng(seed)
    ops = [op("RY", (0,), param=0), op("CNOT", (0, 1)), op("KRAUS2", (1, 2), data=I.random_kraus2(rng, 3)),
           op("RX", (2,), param=1), op("DEPOL2", (2, 0), fixed=(0.1,)), op("KRAUS2", (0, 1), data=I.random_kraus2(rng, 2))]
    circ = I.Circuit(n, ops, 2, True)
    theta = [0.7, -1.3]
    for o in ops:
        if o.name == "KRAUS2":
            np.testing.assert_allclose(sum(k.conj().T @ k for k in O.kraus(o)), np.eye(4), atol=1e-13)
    rho = I.random_density(n, seed).reshape(1 << n, 1 << n, order="F")
    ref = rho.copy()
    for o in ops:
        if o.name in I.CHANNELS + I.CHANNELS2:
            ks = [embed(k, o.qubits, n) for k in O.kraus(o)]
            ref = sum(k @ ref @ k.conj().T for k in ks)
        else:
            U = embed(O.gate_matrix(o, theta), o.qubits, n)
            ref = U @ ref @ U.conj().T
    out = O.rho_apply_circuit(circ, theta, rho.reshape(-1, order="F"))
    np.testing.assert_allclose(out, ref.reshape(-1, order="F"), atol=1e-13)
    vec = O.vec_apply_circuit(circ, theta, rho.reshape(-1, order="F"))
    np.testing.assert_allclose(vec, ref.reshape(-1, order="F"), atol=1e-13)
    # noisy Algorithm 2 through two-qubit channels vs parameter shift (exact for Rx, Ry)
    terms = [(0.6, ((0, "Z"), (2, "X"))), (-0.4, ((1, "Y"),)), (0.3, ((2, "Z"),))]
    e, g = O.noisy_adjoint_grad(circ, theta, terms)
    np.testing.assert_allclose(g, O.parameter_shift_grad(circ, theta, terms), atol=1e-12)


# ----------------------------------------------------------------- sampling

def test_sample_quantiles_of_a_product_state():
    """Ry(t_q) on every qubit of |0...0> gives P(a) = prod_q (cos^2 or sin^2)(t_q/2); with
    the quantile grid u_i = (i + 1/2)/N the number of shots returning a equals the number
    of grid points inside [CDF(a-1), CDF(a)) of that closed form."""
    n, N = 4, 2000
    ts = [0.3, 1.1, 2.0, 2.9]
    ops = [op("RY", (q,), fixed=(ts[q],)) for q in range(n)]
    psi = O.apply_circuit(I.Circuit(n, ops, 0), [])
    P = np.array([np.prod([(math.sin(ts[q] / 2) ** 2) if (a >> q) & 1 else (math.cos(ts[q] / 2) ** 2)
                           for q in range(n)]) for a in range(1 << n)])
    u = (np.arange(N) + 0.5) / N
    got = O.sample(psi, n, u)
    cdf = np.cumsum(P)
    lo = np.concatenate([[0.0], cdf[:-1]])
    expect = [int(np.sum((u >= lo[a]) & (u < cdf[a]))) for a in range(1 << n)]
    assert np.bincount(got, minlength=1 << n).tolist() == expect


def test_sample_basis_state_ghz_and_density():
    n = 5
    psi = np.zeros(1 << n, complex)
    psi[19] = 1
    assert set(O.sample(psi, n, [0.0, 0.3, 0.999999]).tolist()) == {19}
    ghz = O.apply_circuit(I.Circuit(n, [op("H", (0,))] + [op("CNOT", (i, i + 1)) for i in range(n - 1)], 0), [])
    assert O.sample(ghz, n, [0.2, 0.49, 0.51, 0.97]).tolist() == [0, 0, 31, 31]
    rho = np.outer(ghz, ghz.conj()).T.reshape(-1)
    assert O.sample(rho, n, [0.2, 0.49, 0.51, 0.97], density=True).tolist() == [0, 0, 31, 31]


def test_noisy_fsim_gradient_matches_shift_rules():
    """Variational FSIM inside a noisy density circuit: the noisy Algorithm 2 with the
    16x16 superoperator derivative vs the exact shift rules (theta: four-term, phi:
    two-term) and FP64 differences (Delta's)."""
    n = 3
    ops = [op("RX", (0,), param=0), op("FSIM", (0, 1), param=1, fixed=(1.0, 0.6, 0.2, -0.3, 0.4), pmask=0b11111),
           op("DEPOL", (1,), fixed=(0.05,)), op("AMPDAMP", (0,), fixed=(0.1,)), op("RY", (2,), param=6),
           op("FSIM", (1, 2), param=7, fixed=(0.5, 1.1), pmask=0b00011)]
    circ = I.Circuit(n, ops, 9, True)
    theta = np.array([0.4, 1.0, 0.6, 0.2, -0.3, 0.4, 0.9, 0.5, 1.1])
    terms = [(0.7, ((0, "Z"), (1, "Z"))), (-0.5, ((2, "X"),)), (0.3, ((1, "Y"), (2, "Y")))]
    e, g = O.noisy_adjoint_grad(circ, theta, terms)
    L = lambda th: O.energy(circ, th, terms)

    def shift(j, s):
        tp, tm = theta.copy(), theta.copy()
        tp[j] += s
        tm[j] -= s
        return L(tp) - L(tm)
    for j in (1, 7):   # theta of each FSIM
        assert g[j] == pytest.approx((1 - math.sqrt(2)) / 2 * shift(j, np.pi / 2) + shift(j, np.pi / 4), abs=1e-11)
    for j in (2, 8):   # phi
        assert g[j] == pytest.approx(0.5 * shift(j, np.pi / 2), abs=1e-11)
    for j in (3, 4, 5):
        assert g[j] == pytest.approx(O.finite_difference_grad(circ, theta, terms, [j], h=1e-5)[0], abs=1e-8)
    for j in (0, 6):   # the rotations, by the two-term rule
        assert g[j] == pytest.approx(0.5 * shift(j, np.pi / 2), abs=1e-11)


def test_sample_largest_draw_never_returns_zero_weight():
    """The largest draw u = nextafter(1, 0) with zero-weight amplitudes at the end of the
    index range returns the last index of non-zero weight: u W stays below W in
    round-to-nearest, so the least index with u W < CDF(a) exists and has weight."""
    n = 6
    rng = np.random.default_rng(4)
    for last in (0, 5, 37, 62):
        psi = np.zeros(1 << n, complex)
        psi[: last + 1] = rng.normal(size=last + 1) + 1j * rng.normal(size=last + 1)
        got = O.sample(psi, n, [np.nextafter(1.0, 0.0), 0.0])
        assert got.tolist() == [last, 0]
