"""Pins of the FP64 oracle against facts that do not come from the oracle.

Each check compares the oracle with something fixed by the paper or by the
mathematics: gate matrices as exponentials of their generators (rotations are
exp(-i t P / 2), the convention the paper's Trotterised TFIM example relies
on), closed forms (Bell/GHZ amplitudes, the QFT of a basis state equals the
DFT, <Z> of RY(t)|0> = cos t from the Bloch form), brute-force dense
Kronecker products for n <= 6, unitarity and norm invariants, and gradients by
the exact parameter-shift rule and by central finite differences.  The last
test compiles deliberately mutated copies of the oracle and checks that the
pins reject every one of them.
"""
import math
import os
import re
import shutil
import tempfile

import numpy as np
import pytest

import workloads as W
from workloads import Gate
from tests import dense_reference as D

RNG = np.random.default_rng(1234)


def random_gates(n, depth, rng, nparams_box, data_features=0, kinds=None):
    """Random gate list over every kind; parameters each used once (U3 takes
    three consecutive slots and never a fixed angle)."""
    kinds = kinds or W.GATE_KINDS
    gates = []
    np_ = 0
    for _ in range(depth):
        k = kinds[rng.integers(len(kinds))]
        if k in W.TWO_QUBIT or k in W.THREE_QUBIT:
            nw = 3 if k in W.THREE_QUBIT else 2
            if n < nw:
                continue
            wires = tuple(int(w) for w in rng.choice(n, size=nw, replace=False))
        else:
            wires = (int(rng.integers(n)),)
        span = W.ANGLE_SPAN.get(k, 1)
        if k in W.PARAMETRIC:
            if data_features >= span and rng.random() < 0.3:
                gates.append(Gate(k, wires, data=int(rng.integers(data_features - span + 1))))
            elif span == 1 and rng.random() < 0.15:
                gates.append(Gate(k, wires, angle=float(rng.uniform(-4, 4))))
            else:
                gates.append(Gate(k, wires, param=np_))
                np_ += span
        else:
            gates.append(Gate(k, wires))
    nparams_box.append(np_)
    return gates


# ---------------------------------------------------------------------------
# pin suite shared with the mutation check
# ---------------------------------------------------------------------------
def pin_failures(oracle, lib=None):
    """Run quick pins; return the names of those that fail."""
    bad = []

    def check(name, ok):
        if not ok:
            bad.append(name)

    # gate blocks = exponentials of generators / textbook matrices
    for kind in ("h", "x", "y", "z", "s", "rx", "ry", "rz"):
        for t in (0.0, 0.3, -1.7, 2.9):
            got = oracle.gate_block(kind, t, lib=lib)
            check(f"block-{kind}", np.allclose(got, D.one_qubit(kind, t), atol=1e-14))
    # closed forms: Bell, GHZ
    st = oracle.run(2, [Gate("h", (0,)), Gate("cnot", (0, 1))], lib=lib)[0]
    bell = np.zeros(4, complex)
    bell[0] = bell[3] = 1 / math.sqrt(2)
    check("bell", np.allclose(st, bell, atol=1e-15))
    # Bloch: RZ(phi) RY(theta)|0> = e^{-i phi/2}(cos t/2|0> + e^{i phi} sin t/2 |1>)
    th, ph = 1.1, 0.7
    st = oracle.run(1, [Gate("ry", (0,), angle=th), Gate("rz", (0,), angle=ph)], lib=lib)[0]
    ref = np.exp(-0.5j * ph) * np.array([math.cos(th / 2), np.exp(1j * ph) * math.sin(th / 2)])
    check("bloch", np.allclose(st, ref, atol=1e-15))
    # wire order + every kind against dense products (n = 3, 4)
    rng = np.random.default_rng(7)
    for n in (3, 4):
        box = []
        gates = random_gates(n, 40, rng, box)
        params = rng.uniform(-3, 3, size=max(box[0], 1))
        got = oracle.run(n, gates, params, lib=lib)[0]
        ref = D.circuit_operator(n, gates, params)[:, 0]
        check(f"dense-{n}", np.allclose(got, ref, atol=1e-12))
    # QFT of basis states = DFT
    n = 4
    N = 1 << n
    basis = np.eye(N, dtype=complex)
    got = oracle.apply(n, W.qft_gates(n), basis, lib=lib)
    F = np.exp(2j * np.pi * np.outer(np.arange(N), np.arange(N)) / N) / math.sqrt(N)
    check("qft", np.allclose(got, F.T, atol=1e-12))
    # expectation with Y terms against dense
    n = 3
    psi = rng.normal(size=N // 2) + 1j * rng.normal(size=N // 2)
    psi /= np.linalg.norm(psi)
    terms = [(0.7, 0b101, 0b001), (-1.3, 0b010, 0b110), (0.4, 0, 0b011)]
    got = oracle.expect(n, psi[None], [terms], lib=lib)[0, 0]
    ref = np.real(np.vdot(psi, D.observable_operator(n, terms) @ psi))
    check("expect", abs(got - ref) < 1e-13)
    # adjoint gradient vs central differences (all parametric kinds)
    n = 3
    box = []
    gates = random_gates(n, 30, rng, box, kinds=("h", "rx", "ry", "rz", "cnot", "cp",
                                                  "crx", "cry", "crz", "swap", "cz"))
    params = rng.uniform(-3, 3, size=max(box[0], 1))
    obs = [[(1.0, 0, 0b001), (0.5, 0b010, 0)]]
    _, gp, _ = oracle.adjoint(n, gates, obs, params, lib=lib)
    fd = np.zeros_like(params)
    h = 1e-5
    for p in range(params.size):
        e = np.zeros_like(params)
        e[p] = h
        fp = oracle.expect(n, oracle.run(n, gates, params + e, lib=lib), obs, lib=lib)[0, 0]
        fm = oracle.expect(n, oracle.run(n, gates, params - e, lib=lib), obs, lib=lib)[0, 0]
        fd[p] = (fp - fm) / (2 * h)
    check("adjoint-fd", np.allclose(gp, fd, atol=1e-8))
    # U3 against the Z-Y-Z Euler form; RXX/RYY/RZZ against expm; CCX truth table
    for th, ph, la in ((0.3, -1.2, 2.1), (2.5, 0.4, -0.9)):
        got = oracle.apply(1, [Gate("u3", (0,), param=0)], np.eye(2), np.array([th, ph, la]), lib=lib)
        check("u3-euler", np.allclose(got.T, D.u3_euler(th, ph, la), atol=1e-14))
    for kind in ("rxx", "ryy", "rzz"):
        got = oracle.apply(3, [Gate(kind, (2, 0), angle=0.9)], np.eye(8), lib=lib)
        check(f"pair-{kind}", np.allclose(got.T, D.gate_operator(3, kind, (2, 0), 0.9), atol=1e-14))
    got = oracle.apply(3, [Gate("ccx", (2, 0, 1))], np.eye(8), lib=lib)
    check("ccx", np.allclose(got.T, D.gate_operator(3, "ccx", (2, 0, 1), 0.0), atol=1e-15))
    # adjoint gradient vs central differences for the wider gate set, with
    # encoded U3 angles (grad_data)
    n = 3
    box = []
    gates = random_gates(n, 24, rng, box, data_features=3, kinds=("h", "p", "u3", "rxx", "ryy", "rzz", "ccx",
                                                                     "cnot", "ry"))
    params = rng.uniform(-3, 3, size=max(box[0], 1))
    data = rng.uniform(-3, 3, size=(1, 3))
    obs = [[(1.0, 0b011, 0b001), (0.5, 0b100, 0), (0.8, 0, 0b110)]]
    _, gp, gd = oracle.adjoint(n, gates, obs, params, data, lib=lib)

    def f(pv, dv):
        return oracle.expect(n, oracle.run(n, gates, pv, dv, lib=lib), obs, lib=lib)[0, 0]

    h = 1e-5
    fd = np.array([(f(params + h * e, data) - f(params - h * e, data)) / (2 * h) for e in np.eye(params.size)])
    fdd = np.array([(f(params, data + h * e) - f(params, data - h * e)) / (2 * h) for e in np.eye(3)])
    check("adjoint-fd-wide", np.allclose(gp, fd, atol=1e-8) and np.allclose(gd[0], fdd, atol=1e-8))
    # Hessian against gradient differences (closed form pair, U3 same-gate terms)
    gates = [Gate("rx", (0,), param=0), Gate("ry", (0,), param=1), Gate("u3", (1,), param=2),
             Gate("cnot", (0, 1)), Gate("u3", (0,), param=5)]
    params = np.array([0.3, 1.2, -0.7, 0.4, 2.2, 0.9, -1.1, 0.5])
    obs = [[(1.0, 0b01, 0b11), (0.6, 0b10, 0b00)]]
    H = oracle.hessian(2, gates, obs, params, lib=lib)
    fdH = np.zeros_like(H)
    for j in range(params.size):
        e = np.zeros(params.size)
        e[j] = 1e-5
        fdH[j] = (oracle.adjoint(2, gates, obs, params + e, lib=lib)[1]
                  - oracle.adjoint(2, gates, obs, params - e, lib=lib)[1]) / 2e-5
    check("hessian-fd", np.allclose(H, fdH, atol=1e-7))
    # density matrices: pure circuits give |psi><psi|; channel closed forms
    gates = [Gate("h", (0,)), Gate("ry", (1,), angle=0.7), Gate("cnot", (0, 1)), Gate("u3", (1,), param=0)]
    params = np.array([0.4, -1.2, 0.8])
    _, rho = oracle.density(2, gates, None, params, lib=lib)
    psi = oracle.run(2, gates, params, lib=lib)[0]
    check("density-pure", np.allclose(rho[0], np.outer(psi, psi.conj()), atol=1e-13))
    _, r = oracle.density(1, [Gate("bitflip", (0,), angle=0.3)], lib=lib)
    check("bitflip", np.allclose(r[0], np.diag([0.7, 0.3]), atol=1e-15))
    _, r = oracle.density(1, [Gate("x", (0,)), Gate("ampdamp", (0,), angle=0.3)], lib=lib)
    _, r2 = oracle.density(1, [Gate("h", (0,)), Gate("ampdamp", (0,), angle=0.3)], lib=lib)
    check("ampdamp", np.allclose(r[0], np.diag([0.3, 0.7]), atol=1e-15)
          and abs(r2[0][0, 1] - math.sqrt(0.7) / 2) < 1e-15)
    _, r = oracle.density(1, [Gate("h", (0,)), Gate("depolarizing", (0,), angle=0.3)], lib=lib)
    check("depolarizing", abs(np.real(r[0][0, 1]) - 0.5 * (1 - 0.4)) < 1e-15)
    # sampling: inversion of the cumulative distribution, marginal packing
    n = 4
    st = rng.normal(size=(1, 16)) + 1j * rng.normal(size=(1, 16))
    st[0, 5] = 0
    c = np.cumsum(st[0].real ** 2 + st[0].imag ** 2)
    u = np.concatenate([rng.random(200), c[:8] / c[-1]])[None]   # includes exact boundaries
    got = oracle.sample(n, st, u, lib=lib)
    check("sample", (got[0] == np.searchsorted(c, u[0] * c[-1], side="right")).all())
    got2 = oracle.sample(n, st, u, wires=[2, 0], lib=lib)
    check("sample-marginal", (got2 == ((((got >> 3) & 1) << 1) | ((got >> 1) & 1))).all())
    # dense block on the low wires = I (x) U as a Kronecker product
    n, nw = 5, 3
    U = W.random_unitary(nw, 11)
    st = rng.standard_normal((2, 1 << n)) + 1j * rng.standard_normal((2, 1 << n))
    got = oracle.apply_dense(n, nw, U, st, lib=lib)
    ref = st @ np.kron(np.eye(1 << (n - nw)), U).T
    check("dense-kron", np.allclose(got, ref, atol=1e-12))
    return bad


def test_pin_suite_passes(oracle_mod):
    assert pin_failures(oracle_mod) == []


# ---------------------------------------------------------------------------
# individual pins, larger
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("kind", ["h", "x", "y", "z", "s", "rx", "ry", "rz"])
def test_one_qubit_blocks_unitary_and_match_definition(oracle_mod, kind):
    for t in np.linspace(-7, 7, 15):
        U = oracle_mod.gate_block(kind, t)
        np.testing.assert_allclose(U.conj().T @ U, np.eye(2), atol=1e-15)
        np.testing.assert_allclose(U, D.one_qubit(kind, t), atol=1e-14)


@pytest.mark.parametrize("n", range(2, 11))
def test_ghz(oracle_mod, n):
    gates = [Gate("h", (0,))] + [Gate("cnot", (q, q + 1)) for q in range(n - 1)]
    st = oracle_mod.run(n, gates)[0]
    ref = np.zeros(1 << n, complex)
    ref[0] = ref[-1] = 1 / math.sqrt(2)
    np.testing.assert_allclose(st, ref, atol=1e-15)


@pytest.mark.parametrize("n", [1, 2, 3, 5, 6, 8])
def test_qft_of_basis_states_is_dft(oracle_mod, n):
    """QFT|x> = N^{-1/2} sum_y exp(2 pi i x y / N) |y> (paper's QFT gate order,
    with the final swaps)."""
    N = 1 << n
    xs = range(N) if n <= 6 else [0, 1, 77, 128, 255]
    basis = np.zeros((len(xs), N), complex)
    for r, x in enumerate(xs):
        basis[r, x] = 1
    got = oracle_mod.apply(n, W.qft_gates(n), basis)
    y = np.arange(N)
    for r, x in enumerate(xs):
        ref = np.exp(2j * np.pi * x * y / N) / math.sqrt(N)
        np.testing.assert_allclose(got[r], ref, atol=1e-13)


def test_ry_expectation_closed_form(oracle_mod):
    """<Z> of RY(t)|0> = cos t and d<Z>/dt = -sin t (Bloch form)."""
    for t in np.linspace(-6, 6, 25):
        exp, gp, _ = oracle_mod.adjoint(1, [Gate("ry", (0,), param=0)], [W.obs_z(0)],
                                        np.array([t]))
        assert abs(exp[0, 0] - math.cos(t)) < 1e-14
        assert abs(gp[0] + math.sin(t)) < 1e-14


def test_cnot_equals_h_cz_h(oracle_mod):
    """CNOT = (I x H) CZ (I x H) (identity used in the dual-rail CNOT section)."""
    n = 2
    basis = np.eye(4, dtype=complex)
    a = oracle_mod.apply(n, [Gate("cnot", (0, 1))], basis)
    b = oracle_mod.apply(n, [Gate("h", (1,)), Gate("cz", (0, 1)), Gate("h", (1,))], basis)
    np.testing.assert_allclose(a, b, atol=1e-15)


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 6])
def test_random_circuits_match_dense_products(oracle_mod, n):
    rng = np.random.default_rng(100 + n)
    for trial in range(3):
        box = []
        gates = random_gates(n, 12 * n + 5, rng, box, data_features=3)
        params = rng.uniform(-4, 4, size=max(box[0], 1))
        data = rng.uniform(-3, 3, size=(2, 3))
        U0 = D.circuit_operator(n, gates, params, data[0])
        U1 = D.circuit_operator(n, gates, params, data[1])
        st = oracle_mod.run(n, gates, params, data, batch=2)
        np.testing.assert_allclose(st[0], U0[:, 0], atol=1e-12)
        np.testing.assert_allclose(st[1], U1[:, 0], atol=1e-12)
        # arbitrary input states, and the inverse sweep
        psi = rng.normal(size=(2, 1 << n)) + 1j * rng.normal(size=(2, 1 << n))
        out = oracle_mod.apply(n, gates, psi, params, data)
        np.testing.assert_allclose(out[0], U0 @ psi[0], atol=1e-11)
        np.testing.assert_allclose(out[1], U1 @ psi[1], atol=1e-11)
        back = oracle_mod.apply(n, gates, out, params, data, dagger=True)
        np.testing.assert_allclose(back, psi, atol=1e-11)


def test_norm_preserved_after_every_gate(oracle_mod):
    n = 12
    rng = np.random.default_rng(5)
    box = []
    gates = random_gates(n, 60, rng, box)
    params = rng.uniform(-4, 4, size=max(box[0], 1))
    psi = oracle_mod.run(n, [], None)[0]
    for g in gates:
        psi = oracle_mod.apply(n, [g], psi, params)[0]
        assert abs(np.linalg.norm(psi) - 1.0) < 1e-13


@pytest.mark.parametrize("n", [2, 3, 5])
def test_expectation_matches_dense(oracle_mod, n):
    rng = np.random.default_rng(n)
    N = 1 << n
    psi = rng.normal(size=(3, N)) + 1j * rng.normal(size=(3, N))
    psi /= np.linalg.norm(psi, axis=1, keepdims=True)
    obs = []
    for _ in range(3):
        terms = [(float(rng.normal()), int(rng.integers(N)), int(rng.integers(N))) for _ in range(4)]
        obs.append(terms)
    got = oracle_mod.expect(n, psi, obs)
    for r in range(3):
        for o, terms in enumerate(obs):
            ref = np.real(np.vdot(psi[r], D.observable_operator(n, terms) @ psi[r]))
            assert abs(got[r, o] - ref) < 1e-13


def test_adjoint_matches_parameter_shift(oracle_mod):
    """Two-term shift rule, exact for RX/RY/RZ: d f = [f(t+pi/2) - f(t-pi/2)]/2."""
    n = 5
    rng = np.random.default_rng(11)
    box = []
    gates = random_gates(n, 50, rng, box, kinds=("h", "rx", "ry", "rz", "cnot", "cz", "swap"))
    gates = [g if g.param >= 0 or g.kind not in W.PARAMETRIC else g._replace(angle=0.4) for g in gates]
    params = rng.uniform(0, 2 * math.pi, size=box[0])
    obs = [W.obs_tfim_open(n, 0.5)]
    _, gp, _ = oracle_mod.adjoint(n, gates, obs, params)
    for p in range(params.size):
        e = np.zeros_like(params)
        e[p] = math.pi / 2
        fp = oracle_mod.expect(n, oracle_mod.run(n, gates, params + e), obs)[0, 0]
        fm = oracle_mod.expect(n, oracle_mod.run(n, gates, params - e), obs)[0, 0]
        assert abs(gp[p] - 0.5 * (fp - fm)) < 1e-12


def test_adjoint_matches_finite_differences_everything(oracle_mod):
    """Controlled rotations, CP, encoded data, several observables, row
    weights, shared and per-row parameters against central differences."""
    n = 4
    batch = 3
    rng = np.random.default_rng(21)
    box = []
    gates = random_gates(n, 45, rng, box, data_features=2)
    nparams = max(box[0], 1)
    obs = [W.obs_tfim_open(n, 0.5), [(0.3, 0b0110, 0b0010), (1.0, 0, 0b1001)]]
    data = rng.uniform(-3, 3, size=(batch, 2))
    w = rng.normal(size=(batch, 2))
    h = 1e-5

    def loss(params, data, ppr):
        st = oracle_mod.run(n, gates, params, data, batch=batch, params_per_row=ppr)
        return float(np.sum(w * oracle_mod.expect(n, st, obs)))

    for ppr in (False, True):
        params = rng.uniform(-3, 3, size=(batch, nparams) if ppr else nparams)
        exp, gp, gd = oracle_mod.adjoint(n, gates, obs, params, data, batch=batch,
                                         params_per_row=ppr, row_weights=w)
        st = oracle_mod.run(n, gates, params, data, batch=batch, params_per_row=ppr)
        np.testing.assert_allclose(exp, oracle_mod.expect(n, st, obs), atol=1e-14)
        flat = params.reshape(-1)
        for i in range(flat.size):
            e = np.zeros_like(flat)
            e[i] = h
            fd = (loss((flat + e).reshape(params.shape), data, ppr)
                  - loss((flat - e).reshape(params.shape), data, ppr)) / (2 * h)
            assert abs(gp.reshape(-1)[i] - fd) < 1e-7, (ppr, i)
        for i in range(data.size):
            e = np.zeros(data.size)
            e[i] = h
            fd = (loss(params, (data.reshape(-1) + e).reshape(data.shape), ppr)
                  - loss(params, (data.reshape(-1) - e).reshape(data.shape), ppr)) / (2 * h)
            assert abs(gd.reshape(-1)[i] - fd) < 1e-7


def test_distributed_example_four_qubits(oracle_mod):
    """The paper's minimal distributed example: data = arange(4) encoded by an
    RY layer, a CNOT ring, observables Z_0 and X_1, loss = their sum, gradient
    with respect to the data -- checked against dense products and central
    differences."""
    n = 4
    gates = W.encode_layer(n) + [Gate("cnot", (q, (q + 1) % n)) for q in range(n)]
    data = np.arange(4, dtype=np.float64)[None]
    obs = [W.obs_z(0), [W.pauli_term(1.0, {1: "X"})]]
    exp, _, gd = oracle_mod.adjoint(n, gates, obs, None, data)
    U = D.circuit_operator(n, gates, None, data[0])
    psi = U[:, 0]
    for o, terms in enumerate(obs):
        ref = np.real(np.vdot(psi, D.observable_operator(n, terms) @ psi))
        assert abs(exp[0, o] - ref) < 1e-13
    h = 1e-6
    for f in range(4):
        e = np.zeros((1, 4))
        e[0, f] = h
        fp = oracle_mod.expect(n, oracle_mod.run(n, gates, None, data + e), obs).sum()
        fm = oracle_mod.expect(n, oracle_mod.run(n, gates, None, data - e), obs).sum()
        assert abs(gd[0, f] - (fp - fm) / (2 * h)) < 1e-8


# ---------------------------------------------------------------------------
# the wider gate set: P, U3, RXX / RYY / RZZ, CCX
# ---------------------------------------------------------------------------
def _u3(oracle_mod, th, ph, la):
    return oracle_mod.apply(1, [Gate("u3", (0,), param=0)], np.eye(2), np.array([th, ph, la])).T


def test_u3_special_cases_and_bloch_column(oracle_mod):
    """U3(t, 0, 0) = RY(t); U3(t, -pi/2, pi/2) = RX(t); U3(0, 0, l) = P(l) =
    diag(1, e^{il}); U3|0> = cos(t/2)|0> + e^{i phi} sin(t/2)|1> (the Bloch
    form of the Background section); U3 is unitary."""
    for t in np.linspace(-5, 5, 11):
        np.testing.assert_allclose(_u3(oracle_mod, t, 0, 0), D.rotation(D.Y, t), atol=1e-14)
        np.testing.assert_allclose(_u3(oracle_mod, t, -math.pi / 2, math.pi / 2), D.rotation(D.X, t), atol=1e-14)
        np.testing.assert_allclose(_u3(oracle_mod, 0, 0, t), np.diag([1, np.exp(1j * t)]), atol=1e-14)
        ph, la = 0.37 * t + 0.2, -0.6 * t
        U = _u3(oracle_mod, t, ph, la)
        np.testing.assert_allclose(U[:, 0], [math.cos(t / 2), np.exp(1j * ph) * math.sin(t / 2)], atol=1e-14)
        np.testing.assert_allclose(U.conj().T @ U, np.eye(2), atol=1e-14)
        np.testing.assert_allclose(U, D.u3_euler(t, ph, la), atol=1e-14)


def test_phase_shift_special_cases(oracle_mod):
    """P(pi/2) = S, P(pi) = Z, P(t) = e^{it/2} RZ(t)."""
    basis = np.eye(2)
    S = oracle_mod.apply(1, [Gate("p", (0,), angle=math.pi / 2)], basis).T
    Zm = oracle_mod.apply(1, [Gate("p", (0,), angle=math.pi)], basis).T
    np.testing.assert_allclose(S, D.one_qubit("s", 0), atol=1e-15)
    np.testing.assert_allclose(Zm, D.Z, atol=1e-15)
    for t in (-2.2, 0.4, 3.0):
        Pm = oracle_mod.apply(1, [Gate("p", (0,), angle=t)], basis).T
        np.testing.assert_allclose(Pm, np.exp(0.5j * t) * D.rotation(D.Z, t), atol=1e-14)


@pytest.mark.parametrize("kind", ["rxx", "ryy", "rzz"])
def test_two_qubit_rotations_match_expm(oracle_mod, kind):
    """R_PP(t) = exp(-i t P(x)P / 2) on every ordered wire pair of 4 qubits."""
    n = 4
    for a in range(n):
        for b in range(n):
            if a == b:
                continue
            t = 0.3 + a - 0.7 * b
            got = oracle_mod.apply(n, [Gate(kind, (a, b), angle=t)], np.eye(1 << n)).T
            np.testing.assert_allclose(got, D.gate_operator(n, kind, (a, b), t), atol=1e-13)


def test_rzz_phases_by_parity(oracle_mod):
    """RZZ(t)|b> = e^{-it/2}|b> when the two bits agree, e^{+it/2}|b> otherwise
    (Z(x)Z has eigenvalue +1 on equal bits)."""
    n, t = 3, 1.3
    got = oracle_mod.apply(n, [Gate("rzz", (0, 2), angle=t)], np.eye(1 << n)).T
    for i in range(1 << n):
        same = ((i >> 2) & 1) == (i & 1)
        assert abs(got[i, i] - np.exp(-0.5j * t if same else 0.5j * t)) < 1e-15
    assert np.allclose(got - np.diag(np.diag(got)), 0)


def test_ccx_truth_table(oracle_mod):
    """CCX flips the target exactly when both controls are 1, for every
    assignment of the three roles to wires of a 4-qubit register."""
    n = 4
    import itertools
    for c0, c1, t in itertools.permutations(range(n), 3):
        got = oracle_mod.apply(n, [Gate("ccx", (c0, c1, t))], np.eye(1 << n)).T
        for i in range(1 << n):
            bits = [(i >> (n - 1 - q)) & 1 for q in range(n)]
            j = i ^ (1 << (n - 1 - t)) if bits[c0] and bits[c1] else i
            assert got[j, i] == 1 and abs(got[:, i]).sum() == 1


def test_two_qubit_rotations_parameter_shift(oracle_mod):
    """The two-term shift rule is exact for R_PP(t) = exp(-i t P(x)P/2) (the
    generator P(x)P/2 has eigenvalues +-1/2)."""
    n = 4
    rng = np.random.default_rng(17)
    box = []
    gates = random_gates(n, 30, rng, box, kinds=("h", "rxx", "ryy", "rzz", "cnot", "ccx"))
    gates = [g if g.param >= 0 or g.kind not in W.PARAMETRIC else g._replace(angle=0.4) for g in gates]
    params = rng.uniform(0, 2 * math.pi, size=box[0])
    obs = [W.obs_tfim_open(n, 0.5)]
    _, gp, _ = oracle_mod.adjoint(n, gates, obs, params)
    for p in range(params.size):
        e = np.zeros_like(params)
        e[p] = math.pi / 2
        fp = oracle_mod.expect(n, oracle_mod.run(n, gates, params + e), obs)[0, 0]
        fm = oracle_mod.expect(n, oracle_mod.run(n, gates, params - e), obs)[0, 0]
        assert abs(gp[p] - 0.5 * (fp - fm)) < 1e-12


def test_u3_gradients_finite_differences(oracle_mod):
    """Adjoint gradients of U3 angles (trainable and encoded, per row) against
    central differences."""
    n, batch = 3, 2
    gates = [Gate("u3", (0,), param=0), Gate("u3", (1,), data=0), Gate("cnot", (0, 2)),
             Gate("u3", (2,), param=3), Gate("ccx", (0, 1, 2)), Gate("u3", (1,), param=6),
             Gate("rxx", (1, 2), data=3)]
    rng = np.random.default_rng(4)
    params = rng.uniform(-3, 3, size=9)
    data = rng.uniform(-3, 3, size=(batch, 4))
    obs = [[(1.0, 0b001, 0b011), (0.6, 0b110, 0)]]
    _, gp, gd = oracle_mod.adjoint(n, gates, obs, params, data, batch=batch)

    def loss(pv, dv):
        return oracle_mod.expect(n, oracle_mod.run(n, gates, pv, dv, batch=batch), obs).sum()

    h = 1e-6
    for i in range(params.size):
        e = np.zeros(params.size)
        e[i] = h
        assert abs(gp[i] - (loss(params + e, data) - loss(params - e, data)) / (2 * h)) < 1e-7
    for i in range(data.size):
        e = np.zeros(data.size)
        e[i] = h
        dp, dm = (data.reshape(-1) + e).reshape(data.shape), (data.reshape(-1) - e).reshape(data.shape)
        assert abs(gd.reshape(-1)[i] - (loss(params, dp) - loss(params, dm)) / (2 * h)) < 1e-7


# ---------------------------------------------------------------------------
# planted mistakes: each mutant of the oracle must fail at least one pin
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("n,nw", [(3, 1), (5, 3), (7, 6), (6, 6)])
def test_dense_block_is_kronecker_product(oracle_mod, n, nw):
    """(I (x) U) psi with the block on the low wires, against numpy.kron."""
    rng = np.random.default_rng(n * 10 + nw)
    U = W.random_unitary(nw, 100 + nw)
    assert np.allclose(U.conj().T @ U, np.eye(1 << nw), atol=1e-12)
    st = rng.standard_normal((3, 1 << n)) + 1j * rng.standard_normal((3, 1 << n))
    got = oracle_mod.apply_dense(n, nw, U, st)
    ref = st @ np.kron(np.eye(1 << (n - nw)), U).T
    np.testing.assert_allclose(got, ref, atol=1e-12)


@pytest.mark.parametrize("nw", [1, 2, 4])
def test_dense_dft_block_on_basis_states(oracle_mod, nw):
    """The DFT matrix on the low wires maps |h, x> to (1/sqrt N) sum_y w^{xy} |h, y>
    with w = e^{2 pi i / N} (closed form), leaving the high wires h alone."""
    n = nw + 2
    N = 1 << nw
    F = np.exp(2j * np.pi * np.outer(np.arange(N), np.arange(N)) / N) / math.sqrt(N)
    for h in range(4):
        for x in range(N):
            st = np.zeros(1 << n, complex)
            st[h * N + x] = 1.0
            got = oracle_mod.apply_dense(n, nw, F, st)[0]
            ref = np.zeros(1 << n, complex)
            ref[h * N:(h + 1) * N] = np.exp(2j * np.pi * x * np.arange(N) / N) / math.sqrt(N)
            np.testing.assert_allclose(got, ref, atol=1e-13)


def test_dense_block_of_gates_equals_gate_sequence(oracle_mod):
    """A group of gates on the low wires, multiplied into one matrix by dense
    Kronecker products, acts like the gates applied one by one."""
    n, nw = 6, 3
    rng = np.random.default_rng(3)
    low = list(range(n - nw, n))
    gates = [Gate("h", (low[0],)), Gate("ry", (low[1],), angle=0.4), Gate("cnot", (low[1], low[2])),
             Gate("cp", (low[2], low[0]), angle=1.1), Gate("rx", (low[2],), angle=-0.8),
             Gate("crz", (low[0], low[1]), angle=0.3), Gate("swap", (low[0], low[2]))]
    U = D.circuit_operator(nw, [Gate(g.kind, tuple(w - (n - nw) for w in g.wires), angle=g.angle)
                                for g in gates], np.zeros(1))
    st = rng.standard_normal((2, 1 << n)) + 1j * rng.standard_normal((2, 1 << n))
    np.testing.assert_allclose(oracle_mod.apply_dense(n, nw, U, st), oracle_mod.apply(n, gates, st), atol=1e-12)


MUTANTS = {
    "dense-transposed": ("for (int64_t j = 0; j < bw; ++j) acc += U[i * bw + j] * x[j];",
                         "for (int64_t j = 0; j < bw; ++j) acc += U[j * bw + i] * x[j];"),
    "rx-sign": ("case O_CRX:  m[0] = c;  m[1] = -I * s; m[2] = -I * s;",
                "case O_CRX:  m[0] = c;  m[1] = I * s; m[2] = I * s;"),
    "ry-transposed": ("case O_CRY:  m[0] = c;  m[1] = -s;  m[2] = s;",
                      "case O_CRY:  m[0] = c;  m[1] = s;  m[2] = -s;"),
    "full-angle": ("const double c = cos(0.5 * t), s = sin(0.5 * t);",
                   "const double c = cos(t), s = sin(t);"),
    "lsb-wire-order": ("static inline int bitpos(int n, int q) { return n - 1 - q; }",
                       "static inline int bitpos(int n, int q) { (void)n; return q; }"),
    "cp-phase-sign": ("case O_CP:   m[0] = 1;  m[1] = 0;   m[2] = 0;  m[3] = cexp(I * t);",
                      "case O_CP:   m[0] = 1;  m[1] = 0;   m[2] = 0;  m[3] = cexp(-I * t);"),
    "grad-factor": ("const double d = 2.0 * cimag(inner(dim, lam, tmp));",
                    "const double d = cimag(inner(dim, lam, tmp));"),
    "generator-sign": ("case O_RZ: case O_CRZ: g[0] = 0.5;       g[3] = -0.5;",
                       "case O_RZ: case O_CRZ: g[0] = -0.5;       g[3] = 0.5;"),
    "y-pauli-sign": ("case O_Y:    m[0] = 0;  m[1] = -I;  m[2] = I;",
                     "case O_Y:    m[0] = 0;  m[1] = I;  m[2] = -I;"),
    "swap-dropped": ("            psi[j] = t;\n",
                     "            psi[j] = psi[i];\n"),
    "hadamard-sign": ("case O_H:    m[0] = r;  m[1] = r;   m[2] = r;  m[3] = -r;",
                      "case O_H:    m[0] = r;  m[1] = r;   m[2] = r;  m[3] = r;"),
    "u3-phi-lam-swapped": ("case 0: m[0] = ch;        m[1] = -el * sh;      m[2] = ep * sh;",
                           "case 0: m[0] = ch;        m[1] = -ep * sh;      m[2] = el * sh;"),
    "u3-dphi-dropped-phase": ("case 2: m[0] = 0;         m[1] = 0;             m[2] = I * ep * sh;",
                              "case 2: m[0] = 0;         m[1] = 0;             m[2] = ep * sh;"),
    "phase-shift-sign": ("case O_P:    m[0] = 1;  m[1] = 0;   m[2] = 0;  m[3] = cexp(I * t);",
                         "case O_P:    m[0] = 1;  m[1] = 0;   m[2] = 0;  m[3] = cexp(-I * t);"),
    "ryy-as-rxx": ("*zm = (kind == O_RZZ || kind == O_RYY) ? w : 0;",
                   "*zm = (kind == O_RZZ) ? w : 0;"),
    "pair-generator-unhalved": ("for (int64_t i = 0; i < dim; ++i) tmp[i] *= 0.5;",
                                "for (int64_t i = 0; i < dim; ++i) tmp[i] *= 1.0;"),
    "ccx-one-control": ("if ((i & tb) || !(i & b0) || !(i & b1)) continue;",
                        "if ((i & tb) || !(i & b0)) continue;"),
    "hessian-cross-term-dropped": ("const double h = 2.0 * creal(inner(dim, pab, Opsi) + inner(dim, pa + (int64_t)a * dim,",
                                   "const double h = 2.0 * creal(inner(dim, pab, Opsi) + 0.0 * inner(dim, pa + (int64_t)a * dim,"),
    "u3-second-theta-sign": ("const double f2 = -0.25 * f0;", "const double f2 = 0.25 * f0;"),
    "bitflip-as-phaseflip": ("for (int e = 0; e < 4; ++e) { K[0][e] = a * I2[e]; K[1][e] = sqrt(p) * X[e]; }",
                             "for (int e = 0; e < 4; ++e) { K[0][e] = a * I2[e]; K[1][e] = sqrt(p) * Z[e]; }"),
    "depolarizing-p-over-4": ("const double b = sqrt(p / 3.0);", "const double b = sqrt(p / 4.0);"),
    "damping-no-sqrt": ("K[0][0] = 1; K[0][1] = 0; K[0][2] = 0; K[0][3] = a;",
                        "K[0][0] = 1; K[0][1] = 0; K[0][2] = 0; K[0][3] = 1.0 - p;"),
    "density-rows-unconjugated": ("for (int64_t j = 0; j < dim; ++j) row[j] = conj(col[j]);",
                                  "for (int64_t j = 0; j < dim; ++j) row[j] = col[j];"),
    "sample-inclusive-bound": ("if (target < cum[mid]) hi = mid;", "if (target <= cum[mid]) hi = mid;"),
    "sample-marginal-lsb-first": ("if ((wire_mask >> q) & 1) o = (o << 1) | ((idx >> bitpos(n, q)) & 1);",
                                  "if ((wire_mask >> q) & 1) o |= ((idx >> bitpos(n, q)) & 1) << q;"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_reject_planted_mistake(oracle_mod, name):
    src_path = os.path.join(os.path.dirname(oracle_mod.__file__), "oracle.c")
    src = open(src_path).read()
    old, new = MUTANTS[name]
    assert src.count(old) == 1, f"mutation anchor for {name} not unique"
    tmpdir = tempfile.mkdtemp(prefix="oracle_mutant_")
    try:
        mpath = os.path.join(tmpdir, "oracle_mutant.c")
        with open(mpath, "w") as f:
            f.write(src.replace(old, new))
        so = oracle_mod.compile_source(mpath, os.path.join(tmpdir, f"lib_{re.sub('[^a-z]', '_', name)}.so"))
        lib = oracle_mod.load_library(so)
        assert pin_failures(oracle_mod, lib=lib), f"mutant {name} passed every pin"
    finally:
        shutil.rmtree(tmpdir, ignore_errors=True)


# ---------------------------------------------------------------------------
# shot sampling
# ---------------------------------------------------------------------------
def test_sampling_basis_state_is_deterministic(oracle_mod):
    """A basis state |x> yields x on every shot, whatever the uniforms."""
    n = 5
    for x in (0, 7, 31):
        st = np.zeros((1, 1 << n), complex)
        st[0, x] = 1j
        u = np.linspace(0, 1, 50, endpoint=False)[None]
        assert (oracle_mod.sample(n, st, u) == x).all()


def test_sampling_inverts_the_cumulative_distribution(oracle_mod):
    """Against numpy's cumulative sum and search: smallest i with u Z < C(i);
    zero-probability outcomes never appear."""
    rng = np.random.default_rng(9)
    n = 7
    st = rng.normal(size=(3, 1 << n)) + 1j * rng.normal(size=(3, 1 << n))
    st[:, ::3] = 0                         # a third of the outcomes impossible
    u = rng.random((3, 400))
    got = oracle_mod.sample(n, st, u)
    for r in range(3):
        c = np.cumsum(st[r].real ** 2 + st[r].imag ** 2)
        ref = np.searchsorted(c, u[r] * c[-1], side="right")
        assert (got[r] == ref).all()
        assert (got[r] % 3 != 0).all()


def test_sampling_frequencies_match_born_rule(oracle_mod):
    """Empirical frequencies of 200k shots of a 4-qubit state pass a
    chi-square test against |psi|^2 (fixed seed, 0.1% level)."""
    from scipy.stats import chi2
    rng = np.random.default_rng(3)
    n = 4
    st = rng.normal(size=(1, 16)) + 1j * rng.normal(size=(1, 16))
    st /= np.linalg.norm(st)
    p = np.abs(st[0]) ** 2
    shots = 200_000
    u = W.uniform_array(77, shots, 0.0, 1.0)[None]
    counts = np.bincount(oracle_mod.sample(n, st, u)[0], minlength=16)
    stat = float(np.sum((counts - shots * p) ** 2 / (shots * p)))
    assert stat < chi2.ppf(0.999, 15)


def test_sampling_marginal_wires(oracle_mod):
    """The packed outcome of a wire subset is the projection of the full
    outcome (first selected wire most significant), and for a product state
    the marginal of one wire follows that wire's own probabilities."""
    rng = np.random.default_rng(5)
    n = 6
    st = rng.normal(size=(2, 1 << n)) + 1j * rng.normal(size=(2, 1 << n))
    u = rng.random((2, 300))
    full = oracle_mod.sample(n, st, u)
    part = oracle_mod.sample(n, st, u, wires=[4, 1, 2])
    proj = (((full >> (n - 1 - 1)) & 1) << 2) | (((full >> (n - 1 - 2)) & 1) << 1) | ((full >> (n - 1 - 4)) & 1)
    assert (part == proj).all()
    # product state RY(t)|0> on wire 3 (others |0>): P(1) = sin^2(t/2)
    t = 1.1
    prod = oracle_mod.run(n, [Gate("ry", (3,), angle=t)])
    uu = W.uniform_array(5, 100_000, 0.0, 1.0)[None]
    ones = oracle_mod.sample(n, prod, uu, wires=[3]).mean()
    assert abs(ones - math.sin(t / 2) ** 2) < 5 * math.sqrt(0.25 / 100_000)


# ---------------------------------------------------------------------------
# Hessian (product rule)
# ---------------------------------------------------------------------------
def test_hessian_closed_form_two_rotations(oracle_mod):
    """<Z> of RY(b) RX(a)|0> is cos(a) cos(b): its Hessian in (a, b) is
    [[-cos a cos b, sin a sin b], [sin a sin b, -cos a cos b]]."""
    gates = [Gate("rx", (0,), param=0), Gate("ry", (0,), param=1)]
    for a, b in ((0.3, 1.2), (-2.0, 0.7), (2.9, -1.4)):
        H = oracle_mod.hessian(1, gates, [W.obs_z(0)], np.array([a, b]))
        ref = np.array([[-math.cos(a) * math.cos(b), math.sin(a) * math.sin(b)],
                        [math.sin(a) * math.sin(b), -math.cos(a) * math.cos(b)]])
        np.testing.assert_allclose(H, ref, atol=1e-14)


@pytest.mark.parametrize("kinds", [("h", "rx", "ry", "rz", "cnot", "cp", "p", "rzz"),
                                   ("h", "crx", "cry", "crz", "cnot", "u3", "rxx", "ryy", "ccx")])
def test_hessian_matches_gradient_differences(oracle_mod, kinds):
    """Against central differences of the (pinned) adjoint gradient, with a
    parameter shared by two gates, encoded data, two rows and row weights;
    the Hessian is symmetric."""
    n, batch = 3, 2
    rng = np.random.default_rng(len(kinds))
    box = []
    gates = random_gates(n, 16, rng, box, data_features=3, kinds=kinds)
    npar = max(box[0], 1)
    gates.append(Gate("rx", (1,), param=0))       # parameter 0 used twice
    params = rng.uniform(-3, 3, size=npar)
    data = rng.uniform(-3, 3, size=(batch, 3))
    obs = [[(1.0, 0b011, 0b001), (0.5, 0b100, 0)], [(0.7, 0, 0b110)]]
    w = rng.normal(size=(batch, 2))
    H = oracle_mod.hessian(n, gates, obs, params, data, batch=batch, row_weights=w)
    h = 1e-5
    for j in range(npar):
        e = np.zeros(npar)
        e[j] = h
        gp = oracle_mod.adjoint(n, gates, obs, params + e, data, batch=batch, row_weights=w)[1]
        gm = oracle_mod.adjoint(n, gates, obs, params - e, data, batch=batch, row_weights=w)[1]
        np.testing.assert_allclose(H[j], (gp - gm) / (2 * h), atol=2e-7)
    np.testing.assert_allclose(H, H.T, atol=1e-12)


# ---------------------------------------------------------------------------
# density matrices and noise channels
# ---------------------------------------------------------------------------
def bloch(rho):
    """(<X>, <Y>, <Z>) of a one-qubit density matrix."""
    return np.array([np.real(np.trace(D.X @ rho)), np.real(np.trace(D.Y @ rho)), np.real(np.trace(D.Z @ rho))])


def test_density_of_pure_circuits_is_the_outer_product(oracle_mod):
    """Without channels rho = |psi><psi| of the (pinned) state-vector oracle,
    and Tr(P rho) = <psi|P|psi>, for random circuits over every gate kind."""
    rng = np.random.default_rng(31)
    for n in (1, 2, 3, 4):
        box = []
        gates = random_gates(n, 10 * n + 6, rng, box, data_features=3)
        params = rng.uniform(-3, 3, size=max(box[0], 1))
        data = rng.uniform(-3, 3, size=(2, 3))
        obs = [W.obs_tfim_open(n, 0.5) if n > 1 else W.obs_z(0), [(0.7, (1 << n) - 1, 1)]]
        exp, rho = oracle_mod.density(n, gates, obs, params, data, batch=2)
        psi = oracle_mod.run(n, gates, params, data, batch=2)
        for r in range(2):
            np.testing.assert_allclose(rho[r], np.outer(psi[r], psi[r].conj()), atol=1e-13)
        np.testing.assert_allclose(exp, oracle_mod.expect(n, psi, obs), atol=1e-13)


@pytest.mark.parametrize("p", [0.0, 0.13, 0.5, 0.9])
def test_channels_closed_forms(oracle_mod, p):
    """Textbook actions (Nielsen & Chuang, Sec. 8.3): bit flip on |0> gives
    diag(1-p, p); phase flip on |+> scales the coherence by 1-2p; amplitude
    damping on |1> gives diag(p, 1-p) and on |+> coherence sqrt(1-p)/2;
    depolarizing (p <= 3/4) shrinks the Bloch vector by 1 - 4p/3."""
    G = Gate
    _, r = oracle_mod.density(1, [G("bitflip", (0,), angle=p)])
    np.testing.assert_allclose(r[0], np.diag([1 - p, p]), atol=1e-15)
    _, r = oracle_mod.density(1, [G("h", (0,)), G("phaseflip", (0,), angle=p)])
    np.testing.assert_allclose(r[0], 0.5 * np.array([[1, 1 - 2 * p], [1 - 2 * p, 1]]), atol=1e-15)
    _, r = oracle_mod.density(1, [G("x", (0,)), G("ampdamp", (0,), angle=p)])
    np.testing.assert_allclose(r[0], np.diag([p, 1 - p]), atol=1e-15)
    _, r = oracle_mod.density(1, [G("h", (0,)), G("ampdamp", (0,), angle=p)])
    ref = np.array([[(1 + p) / 2, math.sqrt(1 - p) / 2], [math.sqrt(1 - p) / 2, (1 - p) / 2]])
    np.testing.assert_allclose(r[0], ref, atol=1e-15)
    if p <= 0.75:
        prep = [G("ry", (0,), angle=1.1), G("rz", (0,), angle=-0.6)]
        _, r0 = oracle_mod.density(1, prep)
        _, r1 = oracle_mod.density(1, prep + [G("depolarizing", (0,), angle=p)])
        np.testing.assert_allclose(bloch(r1[0]), (1 - 4 * p / 3) * bloch(r0[0]), atol=1e-14)


def test_noisy_circuits_stay_density_matrices(oracle_mod):
    """Random circuits with channels on every qubit: trace 1, Hermitian,
    positive semidefinite; the depolarizing channel at p = 3/4 leaves the
    maximally mixed state on its qubit (partial trace = I/2)."""
    rng = np.random.default_rng(8)
    n = 3
    gates = []
    for _ in range(30):
        k = ("h", "ry", "cnot", "rxx", "bitflip", "phaseflip", "depolarizing", "ampdamp")[rng.integers(8)]
        if k in W.NOISE_KINDS:
            gates.append(Gate(k, (int(rng.integers(n)),), angle=float(rng.uniform(0, 0.75))))
        elif k in ("cnot", "rxx"):
            a, b = rng.choice(n, size=2, replace=False)
            gates.append(Gate(k, (int(a), int(b)), angle=float(rng.uniform(-3, 3))))
        else:
            gates.append(Gate(k, (int(rng.integers(n)),), angle=float(rng.uniform(-3, 3))))
    _, r = oracle_mod.density(n, gates)
    rho = r[0]
    assert abs(np.trace(rho) - 1) < 1e-13
    np.testing.assert_allclose(rho, rho.conj().T, atol=1e-14)
    assert np.linalg.eigvalsh(rho).min() > -1e-13
    _, r = oracle_mod.density(n, gates + [Gate("depolarizing", (1,), angle=0.75)])
    red = np.einsum("ajbj->ab", r[0].reshape(2, 2, 2, 2, 2, 2).transpose(1, 0, 2, 4, 3, 5).reshape(2, 4, 2, 4))
    np.testing.assert_allclose(red, np.eye(2) / 2, atol=1e-14)


def test_trotter_steps_converge_to_exp_of_tfim(oracle_mod):
    """Second-order Trotter steps of H = -J sum Z_i Z_{i+1} - h sum X_i
    (periodic chain, rx(-h dt) half steps and rzz(-2 J dt) bonds) approach
    exp(-i H t) |0> with error O(dt^2) at fixed t: halving dt divides the
    error by about four.  This holds only with R_P(t) = exp(-i t P / 2) for
    RX and RZZ (the convention the paper's Trotterised TFIM relies on)."""
    from scipy.linalg import expm
    n, J, h, t = 4, 1.0, 1.2, 0.8
    Hm = np.zeros((1 << n, 1 << n), complex)
    for i in range(n):
        Hm -= J * D.embed(n, {i: D.Z, (i + 1) % n: D.Z})
        Hm -= h * D.embed(n, {i: D.X})
    exact = expm(-1j * Hm * t)[:, 0]
    errs = []
    for steps in (4, 8, 16):
        dt = t / steps
        st = oracle_mod.run(n, W.tfim_trotter_gates(n, steps, J, h, dt))[0]
        errs.append(np.linalg.norm(st - exact))
    assert errs[-1] < 5e-3
    for a, b in zip(errs, errs[1:]):
        assert 3.5 < a / b < 4.5, errs
