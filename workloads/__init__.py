"""Seeded synthetic inputs shared by the FP64 oracle and the CUDA library.

This module only *describes* inputs: gate lists, parameter and feature arrays,
Pauli-sum observables and the five workload configurations.  It contains none
of the method's arithmetic (no gate matrices, no state updates, no
expectations), so the oracle and the GPU path can both consume it without
sharing any simulation code.

Conventions (the paper leaves them open; the readings are listed in the design
notes):

* A gate is ``Gate(kind, wires, param, data, angle)``.  ``kind`` is one of
  :data:`GATE_KINDS`; ``wires`` is ``(target,)`` for one-qubit gates,
  ``(control, target)`` for controlled gates, ``(a, b)`` for SWAP and the
  two-qubit rotations RXX/RYY/RZZ, and ``(control0, control1, target)`` for
  CCX.  The rotation angle is ``params[param]`` when ``param >= 0``, else
  ``data[row, data]`` when ``data >= 0`` (an encoded input feature, the
  ``encode=True`` gates of the paper's qubit API), else the fixed ``angle``.
  U3 reads its three angles (theta, phi, lam) from ``params[param + 0..2]``
  or ``data[row, data + 0..2]``.
* A Pauli term is ``(coeff, xmask, zmask)`` with bit ``q`` of a mask
  referring to wire ``q``; a wire with both bits set carries ``Y``.  An
  observable is a list of terms whose weighted sum is measured.
* Random numbers come from splitmix64 (Steele, Lea & Flood, "Fast splittable
  pseudorandom number generators", OOPSLA 2014), mapped to doubles in [0, 1)
  with the top 53 bits.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, NamedTuple, Optional, Sequence, Tuple

import numpy as np

GATE_KINDS = (
    "h", "x", "y", "z", "s",
    "rx", "ry", "rz",
    "cnot", "cz", "cp", "swap",
    "crx", "cry", "crz",
    "p", "u3", "rxx", "ryy", "rzz", "ccx",
)
ONE_QUBIT = {"h", "x", "y", "z", "s", "rx", "ry", "rz", "p", "u3"}
TWO_QUBIT = {"cnot", "cz", "cp", "swap", "crx", "cry", "crz", "rxx", "ryy", "rzz"}
THREE_QUBIT = {"ccx"}
PARAMETRIC = {"rx", "ry", "rz", "cp", "crx", "cry", "crz", "p", "u3", "rxx", "ryy", "rzz"}
# consecutive parameter / feature slots a gate reads (U3: theta, phi, lam)
ANGLE_SPAN = {"u3": 3}
# single-qubit noise channels (density-matrix circuits only); the probability
# is the gate's fixed `angle`
NOISE_KINDS = ("bitflip", "phaseflip", "depolarizing", "ampdamp")

MASK64 = (1 << 64) - 1
BASE_SEED = 0x2512_18995


class Gate(NamedTuple):
    kind: str
    wires: Tuple[int, ...]
    param: int = -1
    data: int = -1
    angle: float = 0.0


Term = Tuple[float, int, int]  # (coeff, xmask by wire, zmask by wire)


# --------------------------------------------------------------------------
# splitmix64
# --------------------------------------------------------------------------
class SplitMix64:
    """splitmix64 stream (Steele, Lea & Flood 2014)."""

    def __init__(self, seed: int):
        self.state = seed & MASK64

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
        return z ^ (z >> 31)

    def uniform(self) -> float:
        """Double in [0, 1) from the top 53 bits."""
        return (self.next_u64() >> 11) * (1.0 / 9007199254740992.0)

    def uniform_range(self, lo: float, hi: float) -> float:
        return lo + (hi - lo) * self.uniform()

    def integer(self, lo: int, hi: int) -> int:
        """Integer uniform in [lo, hi] inclusive (multiply-shift on 64 bits)."""
        span = hi - lo + 1
        return lo + ((self.next_u64() * span) >> 64)


def uniform_array(seed: int, count: int, lo: float, hi: float) -> np.ndarray:
    """``count`` doubles uniform in [lo, hi) from one splitmix64 stream."""
    rng = SplitMix64(seed)
    out = np.empty(count, dtype=np.float64)
    for i in range(count):
        out[i] = rng.uniform_range(lo, hi)
    return out


# --------------------------------------------------------------------------
# circuit builders (gate lists only)
# --------------------------------------------------------------------------
def random_unitary(nw: int, seed: int) -> np.ndarray:
    """A 2^nw x 2^nw unitary: Q of the QR factorisation of a matrix whose
    entries have real and imaginary parts uniform in [-1, 1)."""
    d = 1 << nw
    v = uniform_array(seed, 2 * d * d, -1.0, 1.0)
    q, _ = np.linalg.qr((v[0::2] + 1j * v[1::2]).reshape(d, d))
    return np.ascontiguousarray(q)


def hea_layers(n: int, layers: int, first_param: int = 0,
               ring: Optional[Sequence[Sequence[int]]] = None) -> List[Gate]:
    """Hardware-efficient ansatz: per layer RY on every wire, RZ on every wire,
    then a CNOT ring q -> q+1 (mod n) applied in wire order.

    Parameter index is layer-major: RY of wire q in layer l uses
    ``first_param + 2*n*l + q`` and RZ uses ``first_param + 2*n*l + n + q``.
    ``ring`` optionally replaces the single ring by several rings, each a list
    of wires (used to build factorised circuits whose result is a product of
    small independent states).
    """
    gates: List[Gate] = []
    rings = [list(range(n))] if ring is None else [list(r) for r in ring]
    for l in range(layers):
        base = first_param + 2 * n * l
        for q in range(n):
            gates.append(Gate("ry", (q,), param=base + q))
        for q in range(n):
            gates.append(Gate("rz", (q,), param=base + n + q))
        for r in rings:
            m = len(r)
            if m < 2:
                continue
            for i in range(m):
                gates.append(Gate("cnot", (r[i], r[(i + 1) % m])))
    return gates


def encode_layer(n: int, wires: Optional[Sequence[int]] = None, first_feature: int = 0) -> List[Gate]:
    """``rylayer(encode=True)``: RY on each wire with angle = data feature."""
    ws = range(n) if wires is None else wires
    return [Gate("ry", (q,), data=first_feature + i) for i, q in enumerate(ws)]


def qft_gates(n: int, swaps: bool = True) -> List[Gate]:
    """QFT gate list in the order of the paper's distributed-QFT example
    (Sec. "Distributed Quantum Fourier Transform"): for each wire q a Hadamard,
    then controlled phases CP(pi / 2**(i - q)) with control i > q and target q,
    then (unless reversed) swaps of wire q with wire n-1-q."""
    gates: List[Gate] = []
    for q in range(n):
        gates.append(Gate("h", (q,)))
        for i in range(q + 1, n):
            gates.append(Gate("cp", (i, q), angle=math.pi / float(2 ** (i - q))))
    if swaps:
        for q in range(n // 2):
            gates.append(Gate("swap", (q, n - 1 - q)))
    return gates


def qcnn_gates(n: int = 12) -> Tuple[List[Gate], int, int]:
    """The QCNN of the paper's Quantum Machine Learning section, as a gate
    list: features are angle-encoded by RY on the active wires, each
    convolution puts RXX then RYY on neighbouring pairs (0,1), (2,3), ...,
    each pooling applies CRY with control 2i+1 and target 2i, halving the
    active wires 12 -> 6 -> 3; the last stage convolves (0,1), (1,2) and pools
    with CRY(1 -> 0), CRY(2 -> 0).  Every RXX/RYY/CRY owns a parameter.
    Returns (gates, nparams, nfeatures)."""
    gates: List[Gate] = []
    npar = nfeat = 0

    def encode(m):
        nonlocal nfeat
        for q in range(m):
            gates.append(Gate("ry", (q,), data=nfeat))
            nfeat += 1

    def pair(kind, a, b):
        nonlocal npar
        gates.append(Gate(kind, (a, b), param=npar))
        npar += 1

    m = n
    encode(m)
    while m > 3:
        for i in range(0, m - 1, 2):
            pair("rxx", i, i + 1)
            pair("ryy", i, i + 1)
        for i in range(m // 2):
            pair("cry", 2 * i + 1, 2 * i)
        m //= 2
        encode(m)
    for i in range(m - 1):
        pair("rxx", i, i + 1)
        pair("ryy", i, i + 1)
    for c in range(1, m):
        pair("cry", c, 0)
    return gates, npar, nfeat


def qnn_u3_gates(residual: bool) -> Tuple[int, List[Gate], int, int, List[List[Term]]]:
    """The small data re-uploading QNNs of the paper's Quantum Machine Learning
    section.  Plain: one qubit, U3, RY(x), U3, measured in Z.  Residual: two
    qubits, RY on wire 0 and U3 on wire 1, an encoded RY(x) on wire 1
    controlled by wire 0, then RY and U3 again; observables Z_1 and Z_0 Z_1.
    Returns (n, gates, nparams, nfeatures, observables)."""
    if not residual:
        g = [Gate("u3", (0,), param=0), Gate("ry", (0,), data=0), Gate("u3", (0,), param=3)]
        return 1, g, 6, 1, [obs_z(0)]
    g = [Gate("ry", (0,), param=0), Gate("u3", (1,), param=1), Gate("cry", (0, 1), data=0),
         Gate("ry", (0,), param=4), Gate("u3", (1,), param=5)]
    return 2, g, 8, 1, [obs_z(1), [pauli_term(1.0, {0: "Z", 1: "Z"})]]


def tfim_trotter_gates(n: int, steps: int, J: float = 1.0, h: float = 1.2, dt: float = 0.1,
                       periodic: bool = True) -> List[Gate]:
    """Second-order (Strang) Trotterisation of H = -J sum Z_i Z_{i+1} - h sum X_i
    on a chain: per step exp(-i H_x dt/2) exp(-i H_zz dt) exp(-i H_x dt/2),
    i.e. RX(-h dt) on every wire, RZZ(-2 J dt) on the even bonds, the odd
    bonds and (periodic) the bond (n-1, 0), then RX(-h dt) again
    (RX(t) = exp(-i t X / 2), RZZ(t) = exp(-i t Z Z / 2)).  Fixed angles."""
    gates: List[Gate] = []
    for _ in range(steps):
        gates += [Gate("rx", (q,), angle=-h * dt) for q in range(n)]
        for start in (0, 1):
            for i in range(start, n - 1, 2):
                gates.append(Gate("rzz", (i, i + 1), angle=-2.0 * J * dt))
        if periodic and n > 2:
            gates.append(Gate("rzz", (n - 1, 0), angle=-2.0 * J * dt))
        gates += [Gate("rx", (q,), angle=-h * dt) for q in range(n)]
    return gates


def random_circuit(seed: int, nmin: int = 8, nmax: int = 16, dmin: int = 10, dmax: int = 40,
                   kinds: Sequence[str] = ("h", "rx", "ry", "rz", "cnot", "cz")):
    """One circuit of the uneven batch: returns (n, gates, angles).

    Draw order from one splitmix64 stream: n ~ U{nmin..nmax}, depth ~
    U{dmin..dmax}; then per gate: kind ~ U(kinds); a one-qubit target ~ U{0..n-1}
    or an ordered pair of distinct wires (control first, then target drawn from
    the remaining n-1 wires), or three distinct wires drawn the same way; for
    rotations an angle ~ U[0, 2pi) per angle slot.  Each rotation owns its
    parameters (its own indices), so gradients are per circuit.
    """
    rng = SplitMix64(seed)
    n = rng.integer(nmin, nmax)
    depth = rng.integer(dmin, dmax)
    gates: List[Gate] = []
    angles: List[float] = []
    for _ in range(depth):
        kind = kinds[rng.integer(0, len(kinds) - 1)]
        if kind in TWO_QUBIT:
            c = rng.integer(0, n - 1)
            t = rng.integer(0, n - 2)
            if t >= c:
                t += 1
            wires = (c, t)
        elif kind in THREE_QUBIT:
            picked: List[int] = []
            for k in range(3):
                w = rng.integer(0, n - 1 - k)
                for p in sorted(picked):
                    if w >= p:
                        w += 1
                picked.append(w)
            wires = tuple(picked)
        else:
            wires = (rng.integer(0, n - 1),)
        if kind in PARAMETRIC:
            gates.append(Gate(kind, wires, param=len(angles)))
            for _ in range(ANGLE_SPAN.get(kind, 1)):
                angles.append(rng.uniform_range(0.0, 2.0 * math.pi))
        else:
            gates.append(Gate(kind, wires))
    return n, gates, np.asarray(angles, dtype=np.float64)


# --------------------------------------------------------------------------
# observables
# --------------------------------------------------------------------------
def pauli_term(coeff: float, ops: dict) -> Term:
    """Term from {wire: 'X'|'Y'|'Z'}."""
    x = z = 0
    for q, p in ops.items():
        p = p.upper()
        if p in ("X", "Y"):
            x |= 1 << q
        if p in ("Z", "Y"):
            z |= 1 << q
    return (float(coeff), x, z)


def obs_z(q: int) -> List[Term]:
    return [pauli_term(1.0, {q: "Z"})]


def obs_sum_z(n: int) -> List[Term]:
    return [pauli_term(1.0, {q: "Z"}) for q in range(n)]


def obs_tfim_open(n: int, hx: float = 0.5) -> List[Term]:
    """sum_i Z_i Z_{i+1} (open chain) + hx * sum_i X_i."""
    terms = [pauli_term(1.0, {i: "Z", i + 1: "Z"}) for i in range(n - 1)]
    terms += [pauli_term(hx, {i: "X"}) for i in range(n)]
    return terms


def obs_zz01_x0() -> List[Term]:
    return [pauli_term(1.0, {0: "Z", 1: "Z"}), pauli_term(0.5, {0: "X"})]


# --------------------------------------------------------------------------
# workload configurations
# --------------------------------------------------------------------------
@dataclass
class Workload:
    name: str
    n: int
    dtype: str                      # "c64" | "c128"
    batch: int
    gates: List[Gate]
    nparams: int
    params: np.ndarray              # (nparams,) shared, or (batch, nparams) per row
    params_per_row: bool
    nfeatures: int
    data: Optional[np.ndarray]      # (batch, nfeatures) or None
    observables: List[List[Term]]
    want_grad: bool
    want_state: bool
    extra: dict = field(default_factory=dict)


def _seed(tag: int) -> int:
    return (BASE_SEED * 1_000_003 + tag) & MASK64


def config_c1(n: int = 10, layers: int = 4) -> Workload:
    """10-qubit hardware-efficient ansatz, complex128, batch 1, 4 layers,
    80 parameters U[0, 2pi), <Z_0> and the full state."""
    g = hea_layers(n, layers)
    p = uniform_array(_seed(1), 2 * n * layers, 0.0, 2 * math.pi)
    return Workload("c1_hea10_c128", n, "c128", 1, g, p.size, p, False, 0, None,
                    [obs_z(0)], False, True)


def config_c2(n: int = 20, layers: int = 8) -> Workload:
    """20-qubit ansatz, 8 layers (320 params), complex64, batch 1, sum_i Z_i,
    forward only."""
    g = hea_layers(n, layers)
    p = uniform_array(_seed(2), 2 * n * layers, 0.0, 2 * math.pi)
    return Workload("c2_hea20_c64", n, "c64", 1, g, p.size, p, False, 0, None,
                    [obs_sum_z(n)], False, True)


def config_c3(n: int = 12, batch: int = 4096, layers: int = 6) -> Workload:
    """Batched QML: 12 features U[-pi, pi] angle-encoded by RY, then 6 layers
    of RY/RZ + CNOT ring (144 shared params); <Z_0> per sample and the adjoint
    gradient of the batch sum."""
    g = encode_layer(n) + hea_layers(n, layers)
    p = uniform_array(_seed(3), 2 * n * layers, 0.0, 2 * math.pi)
    x = uniform_array(_seed(30), batch * n, -math.pi, math.pi).reshape(batch, n)
    return Workload("c3_qml12x4096_c64", n, "c64", batch, g, p.size, p, False, n, x,
                    [obs_z(0)], True, False)


def config_c4(ncirc: int = 1024):
    """Uneven batch: ``ncirc`` random circuits (per-circuit seed), observable
    Z_0 Z_1 + 0.5 X_0.  Returns a list of (n, gates, angles)."""
    return [random_circuit(_seed(4000 + c)) for c in range(ncirc)]


def config_c5(n: int = 30, layers: int = 10, ring=None) -> Workload:
    """30-qubit single state: QFT then 10 layers RY/RZ + CNOT ring (600
    params), transverse-field Ising observable on an open chain, forward plus
    adjoint gradient."""
    g = qft_gates(n) + hea_layers(n, layers, ring=ring)
    p = uniform_array(_seed(5), 2 * n * layers, 0.0, 2 * math.pi)
    return Workload(f"c5_qft_hea{n}_c64", n, "c64", 1, g, p.size, p, False, 0, None,
                    [obs_tfim_open(n, 0.5)], True, False)


def interleaved_rings(n: int, groups: int) -> List[List[int]]:
    """Wires split into ``groups`` interleaved sets {g, g+groups, ...}."""
    return [list(range(gi, n, groups)) for gi in range(groups)]
