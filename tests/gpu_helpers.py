"""Shared pieces of the GPU parity tests: tolerances, conversions and the
factorised 30-qubit workload whose exact result the oracle can assemble from
three 10-qubit pieces."""
import json
import os

import numpy as np
import torch

import workloads as W

# Tolerances of the parity bar: amplitudes max-abs 1e-5 (c64) / 1e-12
# (c128); expectations and gradients 1e-4 relative (c64) / 1e-12 (c128).
# The relative error of element i is |got_i - ref_i| / max(|ref_i|, ||ref||_inf):
# elements near zero are judged on the size of the largest element of the
# same result, nothing looser.  Only a result that is analytically zero
# (||ref||_inf within FP64 rounding of zero on the quantity's natural scale)
# is judged on that natural scale instead, and the record says so.
AMP_TOL = {torch.complex64: 1e-5, torch.complex128: 1e-12}
REL_TOL = {torch.complex64: 1e-4, torch.complex128: 1e-12}

# Every checked result's error, kept for the per-result error report that
# tests/conftest.py writes when DQ_PARITY_LOG names a file.
RECORDS = []


def _record(kind, what, dtype, max_abs, max_rel, size, note=""):
    RECORDS.append({"test": os.environ.get("PYTEST_CURRENT_TEST", "").split(" ")[0], "kind": kind,
                    "what": what, "dtype": str(dtype).replace("torch.", ""), "n": int(size),
                    "max_abs": float(max_abs), "max_rel": None if max_rel is None else float(max_rel),
                    "note": note})


def assert_amps(got, ref, dtype, what="state"):
    got = np.asarray(got)
    err = float(np.max(np.abs(got - ref))) if got.size else 0.0
    _record("amplitudes", what, dtype, err, None, got.size)
    assert err <= AMP_TOL[dtype], f"{what}: max-abs error {err:.3e} > {AMP_TOL[dtype]}"
    return err


def obs_scale(observables):
    return max(sum(abs(t[0]) for t in o) for o in observables) if observables else 1.0


def assert_rel(got, ref, dtype, what="value", zero_scale=None):
    """Element-wise relative check against max(|ref_i|, ||ref||_inf).

    `zero_scale` is the quantity's natural scale (sum of |coefficients| for an
    expectation, times the row weights for a gradient); it is used only when
    the whole reference is zero to FP64 rounding on that scale, where a
    relative error has no meaning."""
    got = np.asarray(got, dtype=np.float64).reshape(-1)
    ref = np.asarray(ref, dtype=np.float64).reshape(-1)
    if ref.size == 0:
        return 0.0
    top = float(np.max(np.abs(ref)))
    note = ""
    if zero_scale is not None and top <= 1e-13 * zero_scale:
        top, note = float(zero_scale), "analytically zero: judged on the natural scale"
    scale = np.maximum(np.abs(ref), top)
    scale = np.where(scale == 0, 1.0, scale)
    diff = np.abs(got - ref)
    rel = diff / scale
    worst = float(np.max(rel))
    _record("relative", what, dtype, float(np.max(diff)), worst, ref.size, note)
    assert worst <= REL_TOL[dtype], f"{what}: relative error {worst:.3e} > {REL_TOL[dtype]} at {int(np.argmax(rel))}"
    return worst


def write_records(path):
    with open(path, "a") as f:
        for r in RECORDS:
            f.write(json.dumps(r) + "\n")
    RECORDS.clear()


def np_state(t):
    return t.detach().cpu().numpy().astype(np.complex128)


def dev(x, dtype=torch.float64):
    if x is None:
        return None
    return torch.as_tensor(np.ascontiguousarray(x), dtype=dtype, device="cuda")


# ---------------------------------------------------------------------------
# factorised 30-qubit workload
# ---------------------------------------------------------------------------
def factorised_c5(n=30, groups=3, layers=10):
    """QFT then `layers` of RY/RZ with CNOT rings inside `groups` interleaved
    wire groups.  QFT|0...0> is the uniform state |+>^n exactly, and the
    rings never couple groups, so the final state is a product over groups."""
    rings = W.interleaved_rings(n, groups)
    wl = W.config_c5(n, layers, ring=rings)
    return wl, rings


def group_circuit(n, rings, gi, full_gates):
    """The group's own circuit on local wires: H on every wire (|+>), then
    the group's gates of the ansatz part with global parameter indices."""
    wires = rings[gi]
    local = {w: j for j, w in enumerate(wires)}
    gates = [W.Gate("h", (j,)) for j in range(len(wires))]
    nqft = len(W.qft_gates(n))
    for g in full_gates[nqft:]:
        if all(w in local for w in g.wires):
            gates.append(g._replace(wires=tuple(local[w] for w in g.wires)))
    return gates


def factorised_reference(oracle, n, rings, wl):
    """Exact <H_TFIM>, its gradient (600) and per-group states."""
    params = wl.params
    states, zexp = {}, np.zeros(n)
    xexp = np.zeros(n)
    for gi, wires in enumerate(rings):
        m = len(wires)
        gates = group_circuit(n, rings, gi, wl.gates)
        st = oracle.run(m, gates, params)[0]
        states[gi] = st
        obs = [W.obs_z(j) for j in range(m)] + [[W.pauli_term(1.0, {j: "X"})] for j in range(m)]
        e = oracle.expect(m, st[None], obs)[0]
        for j, w in enumerate(wires):
            zexp[w] = e[j]
            xexp[w] = e[m + j]
    energy = sum(zexp[i] * zexp[i + 1] for i in range(n - 1)) + 0.5 * xexp.sum()
    grad = np.zeros(params.size)
    for gi, wires in enumerate(rings):
        m = len(wires)
        local = {w: j for j, w in enumerate(wires)}
        terms = []
        for w in wires:
            c = 0.0
            if w - 1 >= 0:
                c += zexp[w - 1]
            if w + 1 < n:
                c += zexp[w + 1]
            terms.append(W.pauli_term(c, {local[w]: "Z"}))
            terms.append(W.pauli_term(0.5, {local[w]: "X"}))
        gates = group_circuit(n, rings, gi, wl.gates)
        _, gp, _ = oracle.adjoint(m, gates, [terms], params)
        grad += gp
    return energy, grad, states


def factorised_amplitude(n, rings, states, b):
    amp = 1.0 + 0j
    for gi, wires in enumerate(rings):
        m = len(wires)
        loc = 0
        for j, w in enumerate(wires):
            loc |= ((b >> (n - 1 - w)) & 1) << (m - 1 - j)
        amp *= states[gi][loc]
    return amp
