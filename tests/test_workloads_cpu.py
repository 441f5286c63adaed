"""CPU checks of the input builders and of the binding's host-side gate
packing (no GPU): the QCNN and QNN structures of the paper's examples, the
Trotter step, random circuits over every kind, and parameter-count
inference with U3's three angle slots."""
import math

import numpy as np

import workloads as W


def test_qcnn_structure():
    """12 -> 6 -> 3 active wires: RY encodings of 12 + 6 + 3 features, RXX/RYY
    on neighbouring pairs, CRY pooling from wire 2i+1 to 2i, then the last
    stage's two convolutions and CRY(1 -> 0), CRY(2 -> 0)."""
    gates, npar, nfeat = W.qcnn_gates(12)
    assert (len(gates), npar, nfeat) == (54, 33, 21)
    enc = [g for g in gates if g.data >= 0]
    assert [g.data for g in enc] == list(range(21))
    assert all(g.kind == "ry" for g in enc)
    pools = [g.wires for g in gates if g.kind == "cry"]
    assert pools == [(1, 0), (3, 2), (5, 4), (7, 6), (9, 8), (11, 10), (1, 0), (3, 2), (5, 4), (1, 0), (2, 0)]
    params = sorted(g.param for g in gates if g.param >= 0)
    assert params == list(range(33))


def test_qnn_u3_structures():
    n, gates, npar, nfeat, obs = W.qnn_u3_gates(False)
    assert (n, npar, nfeat, len(obs)) == (1, 6, 1, 1)
    assert [g.kind for g in gates] == ["u3", "ry", "u3"]
    n, gates, npar, nfeat, obs = W.qnn_u3_gates(True)
    assert (n, npar, nfeat, len(obs)) == (2, 8, 1, 2)
    slots = sorted(p for g in gates if g.param >= 0 for p in range(g.param, g.param + W.ANGLE_SPAN.get(g.kind, 1)))
    assert slots == list(range(8))


def test_trotter_step_structure():
    n, steps, J, h, dt = 6, 3, 1.0, 1.2, 0.1
    g = W.tfim_trotter_gates(n, steps, J, h, dt)
    per_step = 2 * n + n            # two RX half layers, n bonds (periodic)
    assert len(g) == steps * per_step
    rx = [x for x in g if x.kind == "rx"]
    rzz = [x for x in g if x.kind == "rzz"]
    assert all(math.isclose(x.angle, -h * dt) for x in rx)
    assert all(math.isclose(x.angle, -2 * J * dt) for x in rzz)
    assert sorted(tuple(sorted(x.wires)) for x in rzz[:n]) == sorted([(i, i + 1) for i in range(n - 1)] + [(0, n - 1)])


def test_random_circuits_over_every_kind_are_well_formed():
    for seed in range(200):
        n, gates, angles = W.random_circuit(seed, nmin=3, nmax=9, kinds=W.GATE_KINDS)
        used = 0
        for g in gates:
            assert len(set(g.wires)) == len(g.wires) and all(0 <= w < n for w in g.wires)
            if g.kind in W.THREE_QUBIT:
                assert len(g.wires) == 3
            elif g.kind in W.TWO_QUBIT:
                assert len(g.wires) == 2
            if g.kind in W.PARAMETRIC:
                assert g.param == used
                used += W.ANGLE_SPAN.get(g.kind, 1)
        assert used == len(angles)
        assert np.all((angles >= 0) & (angles < 2 * math.pi))


def test_circuit_infers_parameter_count_with_u3_spans():
    import paper_2512_18995_gb300 as dq
    c = dq.Circuit(3, [W.Gate("ry", (0,), param=0), W.Gate("u3", (1,), param=1), W.Gate("rx", (2,), data=4),
                       W.Gate("u3", (2,), data=0)])
    assert c.nparams == 4 and c.nfeatures == 5
    assert c._arr[1].kind == 16 and list(c._arr[1].wires) == [1, -1, -1]
    t = dq.Circuit(3, [W.Gate("ccx", (0, 2, 1)), W.Gate("depolarizing", (1,), angle=0.1)])
    assert list(t._arr[0].wires) == [0, 2, 1] and t.nparams == 0
