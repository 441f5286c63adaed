"""Dense blocks chosen by the planner (forward-only calls, complex64): runs of
at least eight consecutive gates on the six lowest-order wires are multiplied
into one 64 x 64 unitary on the device and applied by the tensor-core kernel
(the evolution U_n ... U_1 |psi_0> with a run of the U_j multiplied together,
Sec. "Quantum Computing with Qubits", Background).  Gates on other wires that
commute with a run move past it; everything else runs as tile passes."""
import math

import numpy as np
import pytest
import torch

import oracle
import workloads as W
from tests.gpu_helpers import assert_rel, dev, np_state, obs_scale

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("CUDA GPU required", allow_module_level=True)

import paper_2512_18995_gb300 as dq  # noqa: E402
from paper_2512_18995_gb300 import build as dqbuild  # noqa: E402

dqbuild.build()

# three-pass TF32 products: 1e-5 max-abs for a normalised state (the dense
# block's tolerance reading, as for dq_apply_dense)
DENSE_AMP_TOL = 1e-5


def low_block(n, layers, first_param, rng, pidx=True):
    """A brick of gates on wires n-6 .. n-1 (the six lowest-order qubits):
    RY/RZ on each, a CNOT chain, a CZ, a CRY, a SWAP and a fixed RX."""
    w = list(range(n - 6, n))
    g, p = [], first_param
    for _ in range(layers):
        for q in w:
            g.append(W.Gate("ry", (q,), param=p) if pidx else W.Gate("ry", (q,), angle=float(rng.uniform(0, 6))))
            p += pidx
            g.append(W.Gate("rz", (q,), angle=float(rng.uniform(0, 6))))
        for a, b in zip(w[:-1], w[1:]):
            g.append(W.Gate("cnot", (a, b)))
        g += [W.Gate("cz", (w[0], w[3])), W.Gate("cry", (w[5], w[1]), angle=0.7), W.Gate("swap", (w[2], w[4])),
              W.Gate("rx", (w[1],), angle=1.3)]
    return g, p


def planner_circuit(n, rng):
    """Tile-pass gates on all wires, two low-wire runs separated by a gate
    that couples a high and a low wire, high-wire gates interleaved with the
    runs (they commute and move past them), and an encoded RY on a low wire
    (its angle depends on the row, so it cannot join a run)."""
    g = W.hea_layers(n, 1)
    p = 2 * n
    run1, p = low_block(n, 2, p, rng)
    for i, gate in enumerate(run1):            # interleave gates on the high wires
        g.append(gate)
        if i % 7 == 3:
            g.append(W.Gate("rx", (i % (n - 6),), angle=0.1 * i))
    g.append(W.Gate("cnot", (0, n - 1)))       # ends the run: acts on a high and a low wire
    run2, p = low_block(n, 1, p, rng, pidx=False)
    g += run2
    g.append(W.Gate("ry", (n - 2,), data=0))   # row-dependent angle on a low wire
    g += W.hea_layers(n, 1, first_param=p)
    p += 2 * n
    return g, p


def run_forward(ctx, circ, params, data, batch, n, obs, mode):
    ctx.set_option(dq.OPT_DENSE_BLOCKS, mode)
    st = torch.empty((batch, 1 << n), dtype=torch.complex64, device="cuda")
    ctx.set_tracing(True)
    e, _, _, _ = ctx.forward_grad(circ, params, dq.Observables(obs), batch, torch.complex64, data=data,
                                  want_grad=False, state_out=st)
    torch.cuda.synchronize()
    names = set(ctx.trace())
    ctx.set_tracing(False)
    ctx.check()
    return st, e, names


@pytest.mark.parametrize("n,batch", [(15, 2), (19, 1)])
def test_planner_dense_blocks_match_oracle(n, batch):
    ctx = dq.Context(0)
    ctx.set_path(dq.PATH_FUSED)
    try:
        rng = np.random.default_rng(900 + n)
        gates, npar = planner_circuit(n, rng)
        params = rng.uniform(0, 2 * math.pi, npar)
        data = rng.uniform(-math.pi, math.pi, (batch, 1))
        circ = dq.Circuit(n, gates, nparams=npar, nfeatures=1)
        obs = [W.obs_sum_z(n), [W.pauli_term(0.5, {n - 1: "X", n - 3: "Y"})]]
        ref = oracle.run(n, gates, params, data, batch=batch)
        e_ref = oracle.expect(n, ref, obs)
        for mode, want in ((1, True), (0, False)):
            st, e, names = run_forward(ctx, circ, dev(params), dev(data), batch, n, obs, mode)
            assert ("k_dense" in names) == want and ("k_dense_compose" in names) == want, (mode, names)
            err = np.max(np.abs(np_state(st) - ref))
            assert err <= DENSE_AMP_TOL, (mode, err)
            assert_rel(e.cpu().numpy(), e_ref, torch.complex64, f"expectations (dense mode {mode})",
                       zero_scale=obs_scale(obs))
        # dq_apply_circuit takes the same segments
        ctx.set_option(dq.OPT_DENSE_BLOCKS, 1)
        st = torch.empty((batch, 1 << n), dtype=torch.complex64, device="cuda")
        ctx.state_init(st, n)
        ctx.set_tracing(True)
        ctx.apply_circuit(circ, dev(params), st, data=dev(data))
        torch.cuda.synchronize()
        assert "k_dense" in set(ctx.trace())
        ctx.set_tracing(False)
        assert np.max(np.abs(np_state(st) - ref)) <= DENSE_AMP_TOL
        # automatic: the autotuner measures both and picks one; results hold either way
        ctx.set_option(dq.OPT_DENSE_BLOCKS, 2)
        tune_state = torch.empty((batch, 1 << n), dtype=torch.complex64, device="cuda")
        ctx.plan_autotune(circ, tune_state)
        st, e, names = run_forward(ctx, circ, dev(params), dev(data), batch, n, obs, 2)
        assert np.max(np.abs(np_state(st) - ref)) <= DENSE_AMP_TOL
        assert_rel(e.cpu().numpy(), e_ref, torch.complex64, "expectations (autotuned)", zero_scale=obs_scale(obs))
    finally:
        ctx.set_option(dq.OPT_DENSE_BLOCKS, 2)
        ctx.close()


def test_gradient_calls_run_gate_by_gate():
    """With dense blocks forced on, a gradient call still runs every gate on
    its own (the reverse sweep needs each generator) and matches the oracle."""
    n, batch = 15, 2
    ctx = dq.Context(0)
    ctx.set_path(dq.PATH_FUSED)
    try:
        rng = np.random.default_rng(15)
        gates, npar = planner_circuit(n, rng)
        params = rng.uniform(0, 2 * math.pi, npar)
        data = rng.uniform(-math.pi, math.pi, (batch, 1))
        obs = [W.obs_tfim_open(n, 0.5)]
        circ = dq.Circuit(n, gates, nparams=npar, nfeatures=1)
        ctx.set_option(dq.OPT_DENSE_BLOCKS, 1)
        ctx.set_tracing(True)
        e, gp, gd, _ = ctx.forward_grad(circ, dev(params), dq.Observables(obs), batch, torch.complex64,
                                        data=dev(data))
        torch.cuda.synchronize()
        names = set(ctx.trace())
        ctx.set_tracing(False)
        assert "k_dense" not in names, names
        e_ref, gp_ref, gd_ref = oracle.adjoint(n, gates, obs, params, data, batch=batch)
        assert_rel(e.cpu().numpy(), e_ref, torch.complex64, "expectations", zero_scale=obs_scale(obs))
        assert_rel(gp.cpu().numpy(), gp_ref, torch.complex64, "grad params", zero_scale=batch * obs_scale(obs))
        assert_rel(gd.cpu().numpy(), gd_ref, torch.complex64, "grad data", zero_scale=obs_scale(obs))
    finally:
        ctx.set_option(dq.OPT_DENSE_BLOCKS, 2)
        ctx.close()


def test_no_run_no_dense_block():
    """Low-wire gates that alternate with gates coupling a high and a low
    wire never form an eight-gate run: no dense block, even when forced."""
    n = 16
    gates = []
    for i in range(12):
        gates += [W.Gate("ry", (n - 1 - i % 3,), param=i), W.Gate("cnot", (i % 5, n - 1 - i % 3)),
                  W.Gate("rz", (i % 7,), angle=0.3 * i)]
    circ = dq.Circuit(n, gates, nparams=12)
    ctx = dq.Context(0)
    ctx.set_path(dq.PATH_FUSED)
    try:
        params = np.linspace(0.2, 5.0, 12)
        st, e, names = run_forward(ctx, circ, dev(params), None, 1, n, [W.obs_z(0)], 1)
        assert "k_dense" not in names
        assert np.max(np.abs(np_state(st) - oracle.run(n, gates, params))) <= 1e-5
    finally:
        ctx.set_option(dq.OPT_DENSE_BLOCKS, 2)
        ctx.close()
