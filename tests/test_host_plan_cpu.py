"""CPU checks of the library's host-side planning: argument validation, the
lowering of composite gates and noise channels to kernel-level ops, the tile
schedules of the fused path and the shift-rule tables of the Hessian and the
density gradients.  They call the C ABI's inspection entry points
(dq_lower_circuit, dq_tile_schedule, dq_shift_rules), which run the same host
code as the compute calls and touch no GPU.

Expected values come from textbook operators (tests/dense_reference.py, built
from matrix exponentials of generators and Kraus sums) and from the oracle;
nothing is taken from the library itself.
"""
import math

import numpy as np
import pytest

import workloads as W
from workloads import Gate
from tests import dense_reference as D


@pytest.fixture(scope="module")
def L():
    from paper_2512_18995_gb300 import build
    build.build()
    from paper_2512_18995_gb300 import _lib
    _lib.load_library()
    return _lib


ONE_WIRE = ("h", "x", "y", "z", "s", "rx", "ry", "rz", "p")
KINDS_SEED = {k: i + 40 for i, k in enumerate(W.GATE_KINDS)}
DIAGONAL = ("z", "s", "rz", "p", "cz", "cp", "crz")


def op_angle(op, params, data_row):
    if op["param"] >= 0:
        return float(params[op["param"]])
    if op["data"] >= 0:
        return float(data_row[op["data"]])
    return float(op["angle"])


def op_matrix(op, params=None, data_row=None):
    """Dense matrix of one kernel-level op on its own wires (wires[0] is the
    most significant factor), from the textbook definitions."""
    kind = op["kind"]
    if kind == "block":
        m = np.array(op["block"], dtype=complex)
    elif kind == "cblock":
        m = np.kron(D.P0, D.I2) + np.kron(D.P1, np.array(op["block"], dtype=complex))
    elif kind in ONE_WIRE:
        m = D.one_qubit(kind, op_angle(op, params, data_row))
    else:
        m = D.gate_operator(2, kind, (0, 1), op_angle(op, params, data_row))
    return m.conj() if op["conj"] else m


def apply_op(states, n, op, params=None, data_row=None):
    """states: (batch, 2^n); the op acts on its wires (wire 0 = MSB)."""
    m = op_matrix(op, params, data_row)
    w = list(op["wires"])
    b = states.shape[0]
    t = states.reshape([b] + [2] * n)
    axes = [1 + q for q in w]
    t = np.moveaxis(t, axes, list(range(1, 1 + len(w))))
    sh = t.shape
    t = t.reshape(b, 1 << len(w), -1)
    t = np.einsum("ij,bjk->bik", m, t)
    t = np.moveaxis(t.reshape(sh), list(range(1, 1 + len(w))), axes)
    return t.reshape(b, -1)


def lowered_operator(ops, n, params=None, data_row=None):
    U = np.eye(1 << n, dtype=complex)
    # columns of U are states: apply to the transpose's rows
    S = U.T.copy()
    for op in ops:
        S = apply_op(S, n, op, params, data_row)
    return S.T


def random_circuit(n, depth, rng, kinds, data_features=0):
    gates, np_ = [], 0
    for _ in range(depth):
        k = kinds[rng.integers(len(kinds))]
        nw = 3 if k in W.THREE_QUBIT else 2 if k in W.TWO_QUBIT else 1
        wires = tuple(int(x) for x in rng.choice(n, size=nw, replace=False))
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
    return gates, np_


# ---------------------------------------------------------------------------
# lowering
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("kind", ["u3", "rxx", "ryy", "rzz", "ccx", "crx", "cry", "crz", "cp", "p", "swap"])
def test_lowered_gate_equals_its_operator(L, kind):
    """Each gate's kernel-level product equals the textbook operator exactly
    (no global phase), with its angle from a parameter and from a data row."""
    n = 3
    rng = np.random.default_rng(KINDS_SEED[kind])
    nw = 3 if kind in W.THREE_QUBIT else 2 if kind in W.TWO_QUBIT else 1
    for trial in range(4):
        wires = tuple(int(x) for x in rng.choice(n, size=nw, replace=False))
        params = rng.uniform(-4, 4, size=3)
        data_row = rng.uniform(-4, 4, size=3)
        if kind in W.PARAMETRIC:
            g = Gate(kind, wires, param=0) if trial % 2 == 0 else Gate(kind, wires, data=0)
        else:
            g = Gate(kind, wires)
        c = L.Circuit(n, [g], nparams=3, nfeatures=3)
        ops = L.lower_circuit(c)
        assert all(o["kind"] in ONE_WIRE + ("cnot", "cz", "cp", "swap", "crx", "cry", "crz") for o in ops)
        got = lowered_operator(ops, n, params, data_row)
        ref = D.circuit_operator(n, [g], params, data_row)
        np.testing.assert_allclose(got, ref, atol=1e-13)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_lowered_random_circuits_equal_dense_products(L, seed):
    n = 4
    rng = np.random.default_rng(seed)
    gates, P = random_circuit(n, 35, rng, W.GATE_KINDS, data_features=3)
    params = rng.uniform(-4, 4, size=max(P, 1))
    data_row = rng.uniform(-4, 4, size=3)
    c = L.Circuit(n, gates, nparams=max(P, 1), nfeatures=3)
    got = lowered_operator(L.lower_circuit(c), n, params, data_row)
    np.testing.assert_allclose(got, D.circuit_operator(n, gates, params, data_row), atol=1e-12)


def kraus(kind, p):
    s = math.sqrt
    if kind == "bitflip":
        return [s(1 - p) * D.I2, s(p) * D.X]
    if kind == "phaseflip":
        return [s(1 - p) * D.I2, s(p) * D.Z]
    if kind == "depolarizing":
        return [s(1 - p) * D.I2] + [s(p / 3) * P for P in (D.X, D.Y, D.Z)]
    return [np.array([[1, 0], [0, s(1 - p)]], dtype=complex), np.array([[0, s(p)], [0, 0]], dtype=complex)]


@pytest.mark.parametrize("kind", W.NOISE_KINDS)
@pytest.mark.parametrize("p", [0.0, 0.13, 0.5, 0.75])
def test_lowered_channel_equals_kraus_superoperator(L, kind, p):
    """On row-major vec(rho), rho -> sum_k K rho K^dagger is sum_k K (x) conj(K)
    (wire 0 carries the row bit, wire 1 the column bit)."""
    ops = L.lower_circuit(L.Circuit(1, [Gate(kind, (0,), angle=p)]), density=True)
    got = lowered_operator(ops, 2)
    ref = sum(np.kron(K, K.conj()) for K in kraus(kind, p))
    np.testing.assert_allclose(got, ref, atol=1e-14)


@pytest.mark.parametrize("seed", [5, 6, 7])
def test_lowered_density_circuit_matches_the_oracle(L, oracle_mod, seed):
    """Gates (trainable, encoded and fixed angles) and channels on 3 qubits:
    the lowered 6-wire ops applied to vec(|0><0|) give the oracle's density
    matrix."""
    n = 3
    rng = np.random.default_rng(seed)
    gates, P = random_circuit(n, 16, rng, W.GATE_KINDS, data_features=3)
    data = rng.uniform(-3, 3, size=(1, 3))
    noisy = []
    for i, g in enumerate(gates):
        noisy.append(g)
        if i % 2 == 0:
            noisy.append(Gate(W.NOISE_KINDS[(i // 2) % 4], (int(rng.integers(n)),),
                              angle=float(rng.uniform(0.02, 0.4))))
    params = rng.uniform(-4, 4, size=max(P, 1))
    ops = L.lower_circuit(L.Circuit(n, noisy, nparams=max(P, 1), nfeatures=3), density=True)
    v = np.zeros((1, 1 << (2 * n)), dtype=complex)
    v[0, 0] = 1.0
    for op in ops:
        v = apply_op(v, 2 * n, op, params, data[0])
    _, rho = oracle_mod.density(n, noisy, None, params, data)
    np.testing.assert_allclose(v[0], rho[0].reshape(-1), atol=1e-12)


def test_lowered_counts(L):
    sizes = {"u3": 3, "rzz": 3, "rxx": 7, "ryy": 7, "ccx": 7, "h": 1, "crx": 1, "swap": 1}
    for kind, size in sizes.items():
        nw = 3 if kind in W.THREE_QUBIT else 2 if kind in W.TWO_QUBIT else 1
        g = Gate(kind, tuple(range(nw)), param=0) if kind in W.PARAMETRIC else Gate(kind, tuple(range(nw)))
        assert len(L.lower_circuit(L.Circuit(3, [g], nparams=3))) == size
        assert len(L.lower_circuit(L.Circuit(3, [g], nparams=3), density=True)) == 2 * size
    assert L.lower_circuit(L.Circuit(2, [])) == []


# ---------------------------------------------------------------------------
# validation (the same checks every compute call makes before a launch)
# ---------------------------------------------------------------------------
INVALID = [
    ("wire out of range", 3, [Gate("h", (3,))], {}, False),
    ("negative wire", 3, [Gate("rx", (-1,), angle=0.1)], {}, False),
    ("coinciding wires", 3, [Gate("cnot", (1, 1))], {}, False),
    ("coinciding ccx wires", 3, [Gate("ccx", (0, 1, 0))], {}, False),
    ("param out of range", 2, [Gate("rx", (0,), param=2)], {"nparams": 2}, False),
    ("u3 span past nparams", 2, [Gate("u3", (0,), param=1)], {"nparams": 3}, False),
    ("data out of range", 2, [Gate("ry", (0,), data=1)], {"nfeatures": 1}, False),
    ("param and data", 2, [Gate("ry", (0,), param=0, data=0)], {"nparams": 1, "nfeatures": 1}, False),
    ("angle on a fixed gate", 2, [Gate("h", (0,), param=0)], {"nparams": 1}, False),
    ("u3 with a fixed angle", 2, [Gate("u3", (0,), angle=0.3)], {}, False),
    ("channel on the pure path", 2, [Gate("bitflip", (0,), angle=0.1)], {}, False),
    ("probability above 1", 2, [Gate("bitflip", (0,), angle=1.2)], {}, True),
    ("negative probability", 2, [Gate("ampdamp", (0,), angle=-0.1)], {}, True),
    ("depolarizing above 3/4", 2, [Gate("depolarizing", (1,), angle=0.8)], {}, True),
    ("channel with a parameter", 2, [Gate("phaseflip", (0,), param=0)], {"nparams": 1}, True),
    ("density above 17 qubits", 18, [Gate("h", (0,))], {}, True),
    ("no qubits", 0, [], {}, False),
    ("35 qubits", 35, [Gate("h", (0,))], {}, False),
    ("unknown kind", 2, [(99, (0,), -1, -1, 0.0)], {}, False),
]


@pytest.mark.parametrize("case", INVALID, ids=[c[0] for c in INVALID])
def test_invalid_circuits_are_rejected(L, case):
    _, n, gates, kw, density = case
    with pytest.raises(L.DQError) as e:
        L.lower_circuit(L.Circuit(n, gates, **kw), density=density)
    assert e.value.status == 1


def test_boundary_values_are_accepted(L):
    ok = [Gate("depolarizing", (0,), angle=0.75), Gate("ampdamp", (1,), angle=1.0),
          Gate("bitflip", (0,), angle=0.0)]
    assert len(L.lower_circuit(L.Circuit(2, ok), density=True)) == 13 + 7 + 3
    assert len(L.lower_circuit(L.Circuit(17, [Gate("h", (16,))]), density=True)) == 2
    assert len(L.lower_circuit(L.Circuit(34, [Gate("cnot", (0, 33))]))) == 1


# ---------------------------------------------------------------------------
# tile schedules of the fused path
# ---------------------------------------------------------------------------
def nondiagonal_bits(op, n):
    bit = lambda w: n - 1 - w
    kind = op["kind"]
    if kind in DIAGONAL:
        return set()
    if kind == "swap":
        return {bit(op["wires"][0]), bit(op["wires"][1])}
    return {bit(op["wires"][-1])}


def tma_dims(T, wb):
    """TMA box dimensions a tile bit set needs: the amplitude bits shifted up
    by wb (a complex128 amplitude is two 8-byte elements, wb = 1), cut into
    runs of consecutive bits, each box side covering at most 8 bits (256
    elements)."""
    w = (T << wb) | ((1 << wb) - 1)
    dims, b = 0, 0
    while w >> b:
        if not (w >> b) & 1:
            b += 1
            continue
        run = 0
        while (w >> (b + run)) & 1:
            run += 1
        dims += (run + 7) // 8
        b += run
    return dims


SCHEDULES = [(9, 8, 5, 3), (10, 8, 6, 3), (10, 10, 7, 2), (11, 9, 5, 4), (12, 10, 7, 5), (12, 12, 5, 4)]


def swap_part(op, k):
    """The k-th of the three CNOTs a SWAP of wires a < b runs as."""
    a, b = sorted(op["wires"])
    wires = (b, a) if k in (0, 2) else (a, b)
    return {"kind": "cnot", "wires": wires, "param": -1, "data": -1, "angle": 0.0, "conj": False}


def check_entries(ops, idx, flags):
    """Every op once (a SWAP as its three CNOTs); parity triples listed as
    CNOT, diagonal, CNOT on one pair; returns the ops to apply in order."""
    seq, seen = [], {}
    j = 0
    while j < len(idx):
        i, f = idx[j], flags[j]
        if f & 1:
            a, d, e = (ops[x] for x in idx[j:j + 3])
            assert flags[j:j + 3] == [1, 1, 1] and idx[j + 1] == i + 1 and idx[j + 2] == i + 2
            assert a["kind"] == e["kind"] == "cnot" and a["wires"] == e["wires"]
            assert d["kind"] in DIAGONAL and d["wires"] == (a["wires"][1],)
            seq += [a, d, e]
            for x in idx[j:j + 3]:
                seen[x] = seen.get(x, 0) + 1
            j += 3
            continue
        if f & 2:
            assert ops[i]["kind"] == "swap"
            seq.append(swap_part(ops[i], seen.get(i, 0)))
        else:
            assert ops[i]["kind"] != "swap"
            seq.append(ops[i])
        seen[i] = seen.get(i, 0) + 1
        j += 1
    assert sorted(seen) == list(range(len(ops)))
    for i, cnt in seen.items():
        assert cnt == (3 if ops[i]["kind"] == "swap" else 1), (i, ops[i], cnt)
    return seq


def assert_same_evolution(n, ops, seq, params, data_row):
    s0 = np.zeros((1, 1 << n), dtype=complex)
    s0[0, 0] = 1.0
    for q in range(n):
        s0 = apply_op(s0, n, {"kind": "h", "wires": (q,), "param": -1, "data": -1, "angle": 0.0, "conj": False})
    a, b = s0.copy(), s0.copy()
    for op in ops:
        a = apply_op(a, n, op, params, data_row)
    for op in seq:
        b = apply_op(b, n, op, params, data_row)
    np.testing.assert_allclose(b, a, atol=1e-12)


@pytest.mark.parametrize("n,k,low,M", SCHEDULES)
@pytest.mark.parametrize("adjoint", [False, True])
def test_tile_schedule_is_an_exact_reordering(L, n, k, low, M, adjoint):
    """Every lowered op runs exactly once; each pass's tile has k bits,
    contains the resident low bits and every bit its ops act on
    non-diagonally (parity triples act diagonally), fits five TMA box
    dimensions; and the execution order -- passes regrouped, ops within a
    pass reordered for register layouts -- gives the same state as circuit
    order."""
    rng = np.random.default_rng(n * 100 + k * 10 + M)
    gates, P = random_circuit(n, 60, rng, W.GATE_KINDS, data_features=2)
    params = rng.uniform(-4, 4, size=max(P, 1))
    data_row = rng.uniform(-4, 4, size=2)
    c = L.Circuit(n, gates, nparams=max(P, 1), nfeatures=2)
    ops = L.lower_circuit(c)
    for dtype, wb in ((L.DQ_C64, 0), (L.DQ_C128, 1)):
        if dtype == L.DQ_C128 and M > 4:
            with pytest.raises(L.DQError):
                L.tile_schedule(c, k, low, M, dtype=dtype, adjoint=adjoint)
            continue
        passes = L.tile_schedule(c, k, low, M, dtype=dtype, adjoint=adjoint)
        idx = [i for _, ix, _ in passes for i in ix]
        flags = [f for _, _, fl in passes for f in fl]
        seq = check_entries(ops, idx, flags)
        for T, ix, fl in passes:
            assert bin(T).count("1") == k
            assert T & ((1 << low) - 1) == (1 << low) - 1
            assert tma_dims(T, wb) <= 5
            if adjoint:
                assert not any(f & 1 for f in fl)
            for i, f in zip(ix, fl):
                if f & 1:
                    continue
                for b in nondiagonal_bits(ops[i], n):
                    assert (T >> b) & 1, (i, ops[i], b, bin(T))
        assert_same_evolution(n, ops, seq, params, data_row)


def test_tile_schedule_fuses_parity_triples_on_forward_passes(L):
    n = 10
    gates = [Gate("rzz", (q, (q + 3) % n), param=q) for q in range(n)]
    c = L.Circuit(n, gates)
    fwd = L.tile_schedule(c, 9, 5, 4)
    assert all(f == L.FLAG_PARITY_TRIPLE for _, _, fl in fwd for f in fl)
    rev = L.tile_schedule(c, 9, 5, 4, adjoint=True)
    assert not any(f for _, _, fl in rev for f in fl)


@pytest.mark.parametrize("n", [7, 9, 12, 14, 16])
@pytest.mark.parametrize("dtype", [0, 1])
def test_row_program_is_an_exact_reordering(L, n, dtype):
    """The whole-row kernel's single pass: every op once, parity triples
    fused, and its execution order gives the circuit's state.  (The kernel
    itself takes rows of up to 12 qubits for complex64 and 11 for
    complex128; larger n only exercise the planner with an explicit register
    width.)"""
    rng = np.random.default_rng(700 + n + 50 * dtype)
    gates, P = random_circuit(n, 70, rng, W.GATE_KINDS, data_features=2)
    params = rng.uniform(-4, 4, size=max(P, 1))
    data_row = rng.uniform(-4, 4, size=2)
    c = L.Circuit(n, gates, nparams=max(P, 1), nfeatures=2)
    ops = L.lower_circuit(c)
    for M in ([0, 2, 3, 4] if dtype == 0 else [0, 2, 3]):
        if M and n < 5 + M:
            continue
        if M == 0 and n > (12 if dtype == 0 else 11):    # rows of 2^12 c64 / 2^11 c128 at most
            with pytest.raises(L.DQError) as e:
                L.row_program(c, M, dtype=dtype)
            assert e.value.status == 2
            continue
        m, idx, flags = L.row_program(c, M, dtype=dtype)
        assert m == M or (M == 0 and 2 <= m <= 4 - dtype)
        seq = check_entries(ops, idx, flags)
        if n <= 12:
            assert_same_evolution(n, ops, seq, params, data_row)


def test_row_program_rejects_rows_that_do_not_fit(L):
    # 17 qubits; 6 < 5 lane bits + 3 register bits; 5 register bits (c64); 4 (c128)
    for n, M, dtype in ((17, 0, 0), (6, 3, 0), (9, 5, 0), (9, 4, 1)):
        with pytest.raises(L.DQError) as e:
            L.row_program(L.Circuit(n, [Gate("h", (0,))]), M, dtype=dtype)
        assert e.value.status == 2


@pytest.mark.parametrize("n,k,low,M,dtype", [(10, 11, 5, 3, 0), (10, 9, 5, 6, 0), (10, 9, 5, 5, 1),
                                             (8, 8, 5, 3, 0), (10, 9, 4, 3, 0), (10, 9, 8, 3, 0),
                                             (10, 7, 5, 3, 0)])
def test_tile_schedule_rejects_impossible_shapes(L, n, k, low, M, dtype):
    c = L.Circuit(n, [Gate("h", (0,)), Gate("cnot", (0, n - 1))])
    with pytest.raises(L.DQError) as e:
        L.tile_schedule(c, k, low, M, dtype=dtype)
    assert e.value.status == 2


# ---------------------------------------------------------------------------
# shift-rule tables (Hessian and density gradients)
# ---------------------------------------------------------------------------
def test_shift_rule_table_reproduces_adjoint_gradients(L, oracle_mod):
    """The library's table, applied with the oracle to one virtual parameter
    per occurrence, gives the adjoint gradient of every occurrence, and its
    parameter map folds them into the gradient of the shared parameters."""
    n = 4
    rng = np.random.default_rng(31)
    kinds = tuple(sorted(W.PARAMETRIC)) + ("h", "cnot", "ccx")
    gates, P = random_circuit(n, 36, rng, kinds)
    gates = [g._replace(param=g.param % 6) if g.param >= 0 and g.kind != "u3" else g for g in gates]
    P = max([g.param + W.ANGLE_SPAN.get(g.kind, 1) for g in gates if g.param >= 0] + [6])
    occ, row0, shift, weight = L.shift_rules(L.Circuit(n, gates, nparams=P))
    # expected occurrence map: gate order, U3 angles theta, phi, lam
    exp_occ, vg = [], []
    for g in gates:
        if g.param >= 0:
            vg.append(g._replace(param=len(exp_occ)))
            exp_occ += [g.param + s for s in range(W.ANGLE_SPAN.get(g.kind, 1))]
        else:
            vg.append(g)
    assert occ == exp_occ
    kinds_of = [g.kind for g in gates if g.param >= 0 for _ in range(W.ANGLE_SPAN.get(g.kind, 1))]
    for v, kd in enumerate(kinds_of):
        assert row0[v + 1] - row0[v] == (4 if kd in ("crx", "cry", "crz") else 2)
    params = rng.uniform(-3, 3, size=P)
    t = params[np.array(occ)]
    obs = [W.obs_tfim_open(n, 0.6)]

    def f(tv):
        return oracle_mod.expect(n, oracle_mod.run(n, vg, tv), obs)[0, 0]

    _, gv, _ = oracle_mod.adjoint(n, vg, obs, t)
    for v in range(len(occ)):
        e = np.zeros(len(occ))
        e[v] = 1.0
        got = sum(weight[j] * f(t + shift[j] * e) for j in range(row0[v], row0[v + 1]))
        assert abs(got - gv[v]) < 1e-12
    _, gp, _ = oracle_mod.adjoint(n, gates, obs, params)
    folded = np.zeros(P)
    np.add.at(folded, np.array(occ), gv)
    np.testing.assert_allclose(folded, gp, atol=1e-12)


def test_shift_rule_table_accepts_noisy_circuits(L):
    gates = [Gate("crx", (0, 1), param=0), Gate("depolarizing", (1,), angle=0.2), Gate("u3", (0,), param=1)]
    occ, row0, shift, weight = L.shift_rules(L.Circuit(2, gates))
    assert occ == [0, 1, 2, 3] and row0 == [0, 4, 6, 8, 10]
    with pytest.raises(L.DQError):
        L.shift_rules(L.Circuit(2, [Gate("depolarizing", (1,), angle=0.9)]))
    assert L.shift_rules(L.Circuit(2, [Gate("h", (0,))])) == ([], [0], [], [])


def test_inspection_calls_reject_null_arguments(L):
    import ctypes
    lib = L.load_library()
    c = L.Circuit(9, [Gate("h", (0,))])
    n = ctypes.c_int(0)
    i32 = (ctypes.c_int32 * 8)()
    u64 = (ctypes.c_uint64 * 8)()
    assert lib.dq_lower_circuit(None, 0, None, 0, ctypes.byref(n)) == 1
    assert lib.dq_lower_circuit(c.ref(), 0, None, 0, None) == 1
    assert lib.dq_lower_circuit(c.ref(), 2, None, 0, ctypes.byref(n)) == 1           # density flag 0 or 1
    assert lib.dq_tile_schedule(None, 0, 8, 5, 3, 0, 8, i32, i32, u64, None, ctypes.byref(n)) == 1
    assert lib.dq_tile_schedule(c.ref(), 0, 8, 5, 3, 0, 8, None, i32, u64, None, ctypes.byref(n)) == 1
    assert lib.dq_tile_schedule(c.ref(), 5, 8, 5, 3, 0, 8, i32, i32, u64, None, ctypes.byref(n)) == 1  # dtype
    m = ctypes.c_int(0)
    assert lib.dq_row_program(None, 0, 0, 8, i32, None, ctypes.byref(n), ctypes.byref(m)) == 1
    assert lib.dq_row_program(c.ref(), 0, 0, 8, i32, None, None, ctypes.byref(m)) == 1
    assert lib.dq_shift_rules(None, 0, 0, None, None, None, None, ctypes.byref(n), ctypes.byref(m)) == 1
    assert lib.dq_shift_rules(c.ref(), 0, 0, None, None, None, None, None, ctypes.byref(m)) == 1
    # too small an output array: rejected with nothing written
    ops = (L.dq_lowered_op * 1)()
    c3 = L.Circuit(3, [Gate("ccx", (0, 1, 2))])
    assert lib.dq_lower_circuit(c3.ref(), 0, ops, 1, ctypes.byref(n)) == 1 and n.value == 7
    assert ops[0].param_idx == 0 and ops[0].data_idx == 0     # untouched (a written op holds -1 there)


def test_specialised_pass_source_compiles():
    """The run-time specialised forward passes of a schedule: one op runner
    and one kernel per pass in the source, and the source compiles for
    sm_103a with NVRTC (no device needed)."""
    from paper_2512_18995_gb300 import _lib
    n = 11
    gates = W.hea_layers(n, 2) + [W.Gate("cry", (0, n - 1), param=4 * n), W.Gate("rzz", (2, 7), angle=0.5),
                                  W.Gate("swap", (1, 9))] + W.qft_gates(n)
    c = _lib.Circuit(n, gates, nparams=4 * n + 1)
    sched = _lib.tile_schedule(c, 9, 5, 3)
    src = _lib.jit_source(c, 9, 5, 3)
    assert src.count("struct JitPass") == len(sched) and src.count("__global__") == len(sched)
    st, log = _lib.jit_compile_check(c, 9, 5, 3, cc=103)
    if st == 2:
        pytest.skip("NVRTC is not available here")
    assert st == 0, log
    # the reverse sweep's passes (gradients on the parametric gates)
    rsched = _lib.tile_schedule(c, 9, 5, 3, adjoint=True)
    rsrc = _lib.jit_source(c, 9, 5, 3, adjoint=True)
    assert rsrc.count("struct JitRev") == len(rsched) and "adj_pair" in rsrc and "eng_adjoint" not in rsrc
    st, log = _lib.jit_compile_check(c, 9, 5, 3, cc=103, adjoint=True)
    assert st == 0, log


def test_specialised_row_kernel_source_compiles():
    """The whole-row kernel with a row program's ops compiled in: one kernel,
    forward and reverse segments as direct handler calls (parity-diagonal
    ops included), compiled for sm_103a with NVRTC (no device needed)."""
    from paper_2512_18995_gb300 import _lib
    n = 9
    gates = W.encode_layer(n) + W.hea_layers(n, 1) + [W.Gate("rzz", (2, 7), param=2 * n),
                                                       W.Gate("swap", (1, 8)), W.Gate("crx", (0, 5), angle=0.4)]
    c = _lib.Circuit(n, gates, nparams=2 * n + 1, nfeatures=n)
    _, order, flags = _lib.row_program(c)
    src = _lib.jit_source(c, 0, 0, 0, kind=_lib.JIT_ROWS)
    assert src.count("__global__") == 1 and "dq_jit_rows" in src and "struct JitRows" in src
    assert "adj_pdiag" in src and "eng_pdiag" in src and any(f & 1 for f in flags)
    assert "eng_adjoint" not in src and "eng_apply" not in src
    with pytest.raises(_lib.DQError):
        _lib.jit_source(c, 0, 0, 0, kind=3)
    st, log = _lib.jit_compile_check(c, 0, 0, 0, kind=_lib.JIT_ROWS, cc=103)
    if st == 2:
        pytest.skip("NVRTC is not available here")
    assert st == 0, log
