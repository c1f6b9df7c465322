"""Dense Kronecker-product reference for tiny systems (n <= 6), used to pin the oracle.

Builds the full 2^n x 2^n operator of a k-qubit matrix with numpy.kron from
elementary |r><c| factors: the textbook construction, independent of the oracle's
gather/scatter loops.  Kronecker order is big-endian: the leftmost factor acts on the
most significant index bit, i.e. qubit n-1.
"""
from __future__ import annotations

import itertools
from typing import Sequence

import numpy as np

PAULI = {
    "I": np.eye(2, dtype=complex),
    "X": np.array([[0, 1], [1, 0]], dtype=complex),
    "Y": np.array([[0, -1j], [1j, 0]], dtype=complex),
    "Z": np.array([[1, 0], [0, -1]], dtype=complex),
}


def _unit(r: int, c: int) -> np.ndarray:
    e = np.zeros((2, 2), dtype=complex)
    e[r, c] = 1.0
    return e


def embed(mat: np.ndarray, qubits: Sequence[int], n: int) -> np.ndarray:
    """Full operator of `mat` (index = sum_t bit(q_t) 2^t) acting on `qubits`."""
    k = len(qubits)
    d = 1 << k
    full = np.zeros((1 << n, 1 << n), dtype=complex)
    for r, c in itertools.product(range(d), range(d)):
        if mat[r, c] == 0:
            continue
        factors = [np.eye(2, dtype=complex) for _ in range(n)]
        for t, q in enumerate(qubits):
            factors[q] = _unit((r >> t) & 1, (c >> t) & 1)
        term = np.array([[1.0 + 0j]])
        for q in reversed(range(n)):          # qubit n-1 leftmost
            term = np.kron(term, factors[q])
        full += mat[r, c] * term
    return full


def pauli_operator(terms, n: int) -> np.ndarray:
    H = np.zeros((1 << n, 1 << n), dtype=complex)
    for coeff, factors in terms:
        mats = ["I"] * n
        for q, p in factors:
            mats[q] = p
        term = np.array([[1.0 + 0j]])
        for q in reversed(range(n)):
            term = np.kron(term, PAULI[mats[q]])
        H += coeff * term
    return H
