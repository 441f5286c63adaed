"""Pin of the oracle's conventions against numbers the paper prints.

The paper's illustrative QubitCircuit example (Sec. "Quantum Computing with
Qubits", API Overview) prints, for a 3-qubit circuit whose three trainable
RY angles were drawn at random, five numbers: the probability of wire 0 being
|0>, the expectation of X(x)Z(x)X and its gradient with respect to the three
angles.  The angles themselves are not printed, but three unknowns cannot fit
five rounded numbers by accident: the oracle, with this repository's readings
(wire 0 the most significant bit, R_Y(t) = exp(-i t Y / 2), the CNOT ring
0->1, 1->2, 2->0, data feature q encoded on wire q), must find angles that
reproduce all five within the printing's rounding -- and the alternative
readings must not.  The printed values are in tests/golden/qubitcircuit_example.json.
"""
import itertools
import json
import math
import os

import numpy as np
import pytest

import workloads as W
from workloads import Gate

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "qubitcircuit_example.json")


def example_gates(ring=((0, 1), (1, 2), (2, 0)), cx=(0, 2)):
    gates = [Gate("h", (0,)), Gate("cnot", (0, 1)), Gate("cnot", cx)]
    gates += [Gate("ry", (q,), data=q) for q in range(3)]
    gates += [Gate("cnot", w) for w in ring]
    gates += [Gate("ry", (q,), param=q) for q in range(3)]
    return gates


XZX = [[W.pauli_term(1.0, {0: "X", 1: "Z", 2: "X"})]]


def best_fit(oracle_mod, fx, gates, obs=XZX, data_sign=1.0, wire0_bit="msb", stop_at=None):
    """Smallest max-abs residual over the five printed numbers found from a
    grid of starting angles."""
    from scipy.optimize import least_squares
    pr = fx["printed"]
    target = np.r_[pr["gradient"], pr["expectation"], pr["wire0_probability"]["0"]]
    data = data_sign * np.array([fx["data"]])

    def model(t):
        e, g, _ = oracle_mod.adjoint(3, gates, obs, t, data, batch=1)
        p = np.abs(oracle_mod.run(3, gates, t, data, batch=1)[0]) ** 2
        p0 = p[:4].sum() if wire0_bit == "msb" else p[0::2].sum()
        return np.r_[g, e[0, 0], p0]

    best, arg = np.inf, None
    for x0 in itertools.product(np.linspace(-3.0, 3.0, 5), repeat=3):
        r = least_squares(lambda t: model(t) - target, np.array(x0), xtol=1e-13, ftol=1e-13, gtol=1e-13)
        res = np.abs(model(r.x) - target).max()
        if res < best:
            best, arg = res, r.x
        if stop_at is not None and best <= stop_at:
            break
    return best, arg


@pytest.fixture(scope="module")
def fx():
    return json.load(open(GOLDEN))


def test_printed_example_fits_within_rounding(oracle_mod, fx):
    tol = fx["rounding"] * 1.1
    res, theta = best_fit(oracle_mod, fx, example_gates(), stop_at=tol)
    assert res <= tol, res
    # the printed shot counts are a plausible binomial draw at that probability
    p0 = fx["printed"]["wire0_probability"]["0"]
    n0 = fx["printed"]["wire0_counts_of_1000_shots"]["0"]
    assert abs(n0 - 1000 * p0) <= 4 * math.sqrt(1000 * p0 * (1 - p0))
    assert abs(fx["printed"]["wire0_probability"]["1"] - (1 - p0)) <= fx["rounding"]


ALTERNATIVES = {
    "wire 0 as the least significant bit": dict(wire0_bit="lsb"),
    "ring with reversed CNOT directions": dict(gates=example_gates(ring=((1, 0), (2, 1), (0, 2)))),
    "ring in descending order": dict(gates=example_gates(ring=((2, 0), (1, 2), (0, 1)))),
    "controlled X with wire 2 as control": dict(gates=example_gates(cx=(2, 0))),
    "rotation sign exp(+i t Y / 2)": dict(data_sign=-1.0),
    "basis string read as Z X Z": dict(obs=[[W.pauli_term(1.0, {0: "Z", 1: "X", 2: "Z"})]]),
}


@pytest.mark.parametrize("name", list(ALTERNATIVES))
def test_alternative_readings_do_not_fit(oracle_mod, fx, name):
    kw = dict(ALTERNATIVES[name])
    gates = kw.pop("gates", example_gates())
    res, _ = best_fit(oracle_mod, fx, gates, **kw)
    assert res > 100 * fx["rounding"], (name, res)
