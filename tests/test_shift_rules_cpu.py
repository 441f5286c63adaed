"""The shift rules behind the Hessian and the density-matrix gradients.

Both entry points differentiate by evaluating the circuit at shifted angles.
Here the oracle serves only as an evaluator; the rules themselves are fixed by
the mathematics (Wierichs, Izaac, Wang, Lin, "General parameter-shift rules
for quantum gradients", Quantum 6, 677 (2022)):

* exp(-i t G) with generator eigenvalue differences in {0, +-1} (RX, RY, RZ,
  RXX, RYY, RZZ, P, CP and each of U3's three angles) makes the loss a
  trigonometric polynomial of frequency 1 in t, and
  f'(t) = [f(t + pi/2) - f(t - pi/2)] / 2;
* the controlled rotations have generator |1><1| (x) P / 2 with differences
  1/2 and 1, and need the four-term rule
  f'(t) = c1 [f(t + pi/2) - f(t - pi/2)] - c2 [f(t + 3pi/2) - f(t - 3pi/2)];
  the two-term rule is wrong for them;
* noise channels do not depend on t, so on mixed states the loss is the same
  kind of polynomial and the same rules hold;
* with a parameter shared by several gates the loss is L~(A theta), A the 0/1
  map from parameters to angle occurrences, so H = A^T H~ A.
"""
import math

import numpy as np
import pytest

import workloads as W
from workloads import Gate

FOUR_TERM = ("crx", "cry", "crz")


def four_term_coefficients():
    """c1, c2 from the frequency conditions: sum_j c_j 2 sin(w s_j) = w for
    w in {1/2, 1} with shifts s = pi/2 (weight c1) and 3pi/2 (weight -c2)."""
    s1, s2 = math.pi / 2, 3 * math.pi / 2
    a = np.array([[2 * math.sin(w * s1), -2 * math.sin(w * s2)] for w in (0.5, 1.0)])
    return np.linalg.solve(a, np.array([0.5, 1.0]))


def rule(kind):
    """(shift, weight) pairs of the exact first-derivative rule for an angle of
    a gate of this kind."""
    if kind in FOUR_TERM:
        c1, c2 = four_term_coefficients()
        h = math.pi / 2
        return [(h, c1), (-h, -c1), (3 * h, -c2), (-3 * h, c2)]
    return [(math.pi / 2, 0.5), (-math.pi / 2, -0.5)]


def occurrences(gates):
    """Circuit with one virtual parameter per angle occurrence; returns it, the
    occurrence -> parameter map and the gate kind of each occurrence."""
    vg, occ, kinds = [], [], []
    for g in gates:
        if g.param >= 0:
            vg.append(g._replace(param=len(occ)))
            for s in range(W.ANGLE_SPAN.get(g.kind, 1)):
                occ.append(g.param + s)
                kinds.append(g.kind)
        else:
            vg.append(g)
    return vg, np.array(occ, dtype=np.int64), kinds


def trainable_circuit(n, depth, rng, kinds):
    gates, np_ = [], 0
    for _ in range(depth):
        k = kinds[rng.integers(len(kinds))]
        nw = 3 if k in W.THREE_QUBIT else 2 if k in W.TWO_QUBIT else 1
        wires = tuple(int(w) for w in rng.choice(n, size=nw, replace=False))
        if k in W.PARAMETRIC:
            gates.append(Gate(k, wires, param=np_))
            np_ += W.ANGLE_SPAN.get(k, 1)
        else:
            gates.append(Gate(k, wires))
    return gates, np_


def test_four_term_coefficients_closed_form():
    c1, c2 = four_term_coefficients()
    assert abs(c1 - (math.sqrt(2) + 1) / (4 * math.sqrt(2))) < 1e-15
    assert abs(c2 - (math.sqrt(2) - 1) / (4 * math.sqrt(2))) < 1e-15


def test_controlled_rotation_needs_four_terms(oracle_mod):
    """H on the control, CRY(t): <X_control> = cos(t / 2) (the control's
    coherence is <0|RY(t)|0>), so f' = -sin(t/2) / 2.  The four-term rule gives
    it; the two-term rule gives -sin(t/2) / sqrt2."""
    gates = [Gate("h", (0,)), Gate("cry", (0, 1), param=0)]
    obs = [[W.pauli_term(1.0, {0: "X"})]]

    def f(t):
        return oracle_mod.expect(2, oracle_mod.run(2, gates, np.array([t])), obs)[0, 0]

    for t in (0.3, 1.7, -2.4):
        assert abs(f(t) - math.cos(t / 2)) < 1e-14
        four = sum(w * f(t + s) for s, w in rule("cry"))
        two = sum(w * f(t + s) for s, w in rule("ry"))
        assert abs(four + math.sin(t / 2) / 2) < 1e-14
        assert abs(two + math.sin(t / 2) / math.sqrt(2)) < 1e-14


@pytest.mark.parametrize("seed", [3, 8])
def test_rules_reproduce_adjoint_gradients(oracle_mod, seed):
    """Every parametric kind, every occurrence: the rule of its kind applied to
    the expectation equals the adjoint gradient to rounding."""
    n = 4
    rng = np.random.default_rng(seed)
    kinds = tuple(sorted(W.PARAMETRIC)) + ("h", "cnot", "ccx", "swap")
    gates, P = trainable_circuit(n, 40, rng, kinds)
    vg, occ, okind = occurrences(gates)
    t = rng.uniform(-math.pi, math.pi, size=occ.size)
    obs = [W.obs_tfim_open(n, 0.7), [W.pauli_term(0.5, {0: "Y", 1: "Z", 3: "X"})]]
    w = np.array([[1.0, -0.4]])
    _, g, _ = oracle_mod.adjoint(n, vg, obs, t, row_weights=w)

    def loss(tv):
        return float(np.sum(w * oracle_mod.expect(n, oracle_mod.run(n, vg, tv), obs)))

    for v in range(occ.size):
        e = np.zeros(occ.size)
        e[v] = 1.0
        got = sum(wt * loss(t + s * e) for s, wt in rule(okind[v]))
        assert abs(got - g[v]) < 1e-12, (okind[v], v)


def test_shift_hessian_folds_to_the_oracle_hessian(oracle_mod):
    """H~ rows from shifted adjoint gradients over virtual occurrences, folded
    with the parameter map (parameters shared by several gates), against the
    oracle's product-rule Hessian; batch rows, encoded data and row weights."""
    n, batch = 3, 2
    rng = np.random.default_rng(5)
    kinds = ("rx", "ry", "rz", "crx", "cry", "crz", "cp", "p", "rxx", "rzz", "h", "cnot")
    gates, _ = trainable_circuit(n, 18, rng, kinds)
    # share: parameter p -> p mod 5; two encoded gates
    gates = [g._replace(param=g.param % 5) if g.param >= 0 else g for g in gates]
    gates += [Gate("ry", (0,), data=0), Gate("crz", (2, 1), data=1), Gate("u3", (1,), param=5)]
    P = 8
    params = rng.uniform(-3, 3, size=P)
    data = rng.uniform(-3, 3, size=(batch, 2))
    obs = [W.obs_tfim_open(n, 0.5), [W.pauli_term(1.0, {0: "Y", 2: "X"})]]
    w = rng.normal(size=(batch, 2))
    vg, occ, okind = occurrences(gates)
    V = occ.size
    Ht = np.zeros((V, V))
    for v in range(V):
        for s, wt in rule(okind[v]):
            tv = params[occ].copy()
            tv[v] += s
            _, gv, _ = oracle_mod.adjoint(n, vg, obs, tv, data, batch=batch, row_weights=w)
            Ht[v] += wt * gv
    A = np.zeros((V, P))
    A[np.arange(V), occ] = 1.0
    H = A.T @ Ht @ A
    ref = oracle_mod.hessian(n, gates, obs, params, data, batch=batch, row_weights=w)
    np.testing.assert_allclose(H, ref, atol=1e-11)
    np.testing.assert_allclose(H, H.T, atol=1e-11)


def test_rules_hold_on_noisy_density_circuits(oracle_mod):
    """Channels between the gates: the rule of each kind against central
    differences of the mixed-state expectation."""
    n = 3
    rng = np.random.default_rng(12)
    kinds = ("rx", "ry", "crx", "cry", "crz", "u3", "rzz", "cp", "cnot")
    gates, P = trainable_circuit(n, 12, rng, kinds)
    noisy = []
    for i, g in enumerate(gates):
        noisy.append(g)
        ch = W.NOISE_KINDS[i % len(W.NOISE_KINDS)]
        noisy.append(Gate(ch, (int(rng.integers(n)),), angle=float(rng.uniform(0.05, 0.3))))
    vg, occ, okind = occurrences(noisy)
    t = rng.uniform(-math.pi, math.pi, size=occ.size)
    obs = [W.obs_tfim_open(n, 0.5)]

    def f(tv):
        return oracle_mod.density(n, vg, obs, tv)[0][0, 0]

    h = 1e-5
    for v in range(occ.size):
        e = np.zeros(occ.size)
        e[v] = 1.0
        got = sum(wt * f(t + s * e) for s, wt in rule(okind[v]))
        fd = (f(t + h * e) - f(t - h * e)) / (2 * h)
        assert abs(got - fd) < 1e-8, (okind[v], v)
