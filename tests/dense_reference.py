"""Brute-force dense 2^n x 2^n operators from textbook definitions.

Used only by the tests to pin the oracle.  Nothing here shares code with the
oracle: gates are built as matrix exponentials of their generators
(scipy.linalg.expm), projector sums and Kronecker products with wire 0 as the
leftmost factor (the most significant index bit).
"""
from functools import reduce

import numpy as np
from scipy.linalg import expm

I2 = np.eye(2, dtype=complex)
X = np.array([[0, 1], [1, 0]], dtype=complex)
Y = np.array([[0, -1j], [1j, 0]], dtype=complex)
Z = np.array([[1, 0], [0, -1]], dtype=complex)
P0 = np.array([[1, 0], [0, 0]], dtype=complex)   # |0><0|
P1 = np.array([[0, 0], [0, 1]], dtype=complex)   # |1><1|
PAULI = {"X": X, "Y": Y, "Z": Z}


def kron_all(mats):
    return reduce(np.kron, mats)


def embed(n, ops):
    """Tensor product with ops[q] on wire q (identity elsewhere)."""
    return kron_all([ops.get(q, I2) for q in range(n)])


def rotation(P, theta):
    """R_P(theta) = exp(-i theta P / 2)."""
    return expm(-0.5j * theta * P)


def u3_euler(theta, phi, lam):
    """U3 by the Z-Y-Z Euler decomposition of a one-qubit unitary (Nielsen &
    Chuang, Theorem 4.1): e^{i(phi+lam)/2} R_Z(phi) R_Y(theta) R_Z(lam), the
    global phase chosen so that the (0, 0) entry cos(theta/2) is real."""
    return np.exp(0.5j * (phi + lam)) * rotation(Z, phi) @ rotation(Y, theta) @ rotation(Z, lam)


def one_qubit(kind, theta):
    if kind == "u3":
        return u3_euler(*theta)
    if kind == "p":
        # phase shift = exp(i t |1><1|)
        return expm(1j * theta * P1)
    if kind == "h":
        return (X + Z) / np.sqrt(2.0)
    if kind == "x":
        return X
    if kind == "y":
        return Y
    if kind == "z":
        return Z
    if kind == "s":
        return P0 + 1j * P1
    return rotation({"rx": X, "ry": Y, "rz": Z}[kind], theta)


def gate_operator(n, kind, wires, theta):
    """Dense operator of one gate on n qubits."""
    if len(wires) == 1:
        return embed(n, {wires[0]: one_qubit(kind, theta)})
    if kind == "ccx":
        c0, c1, t = wires
        # identity off the |11> control subspace, X on it
        return embed(n, {}) - embed(n, {c0: P1, c1: P1}) + embed(n, {c0: P1, c1: P1, t: X})
    a, b = wires
    if kind in ("rxx", "ryy", "rzz"):
        P = {"rxx": X, "ryy": Y, "rzz": Z}[kind]
        return expm(-0.5j * theta * embed(n, {a: P, b: P}))
    if kind == "swap":
        # SWAP = (II + XX + YY + ZZ) / 2
        return 0.5 * (embed(n, {}) + embed(n, {a: X, b: X}) + embed(n, {a: Y, b: Y})
                      + embed(n, {a: Z, b: Z}))
    c, t = a, b
    if kind == "cp":
        # controlled phase = exp(i phi |11><11|)
        return expm(1j * theta * embed(n, {c: P1, t: P1}))
    if kind in ("crx", "cry", "crz"):
        P = {"crx": X, "cry": Y, "crz": Z}[kind]
        return expm(-0.5j * theta * embed(n, {c: P1, t: P}))
    V = {"cnot": X, "cz": Z}[kind]
    return embed(n, {c: P0}) + embed(n, {c: P1, t: V})


def angle_of(g, params, data_row):
    """The gate's angle (U3: the tuple theta, phi, lam from consecutive slots)."""
    if g.kind == "u3":
        if g.param >= 0:
            return tuple(float(params[g.param + k]) for k in range(3))
        return tuple(float(data_row[g.data + k]) for k in range(3))
    if g.param >= 0:
        return float(params[g.param])
    if g.data >= 0:
        return float(data_row[g.data])
    return float(g.angle)


def circuit_operator(n, gates, params=None, data_row=None):
    U = np.eye(1 << n, dtype=complex)
    for g in gates:
        U = gate_operator(n, g.kind, g.wires, angle_of(g, params, data_row)) @ U
    return U


def pauli_operator(n, xmask, zmask):
    ops = {}
    for q in range(n):
        x, z = (xmask >> q) & 1, (zmask >> q) & 1
        if x and z:
            ops[q] = Y
        elif x:
            ops[q] = X
        elif z:
            ops[q] = Z
    return embed(n, ops)


def observable_operator(n, terms):
    O = np.zeros((1 << n, 1 << n), dtype=complex)
    for c, x, z in terms:
        O += c * pauli_operator(n, x, z)
    return O
