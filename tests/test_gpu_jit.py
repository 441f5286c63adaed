"""Run-time specialised kernels (DQ_OPT_JIT): each forward or reverse tile
pass's ops, or a whole-row program, compiled into direct handler calls.  The
arithmetic per element is the interpreter's, so states agree with the
interpreting kernel to rounding and with the oracle within the parity
tolerances, on every gate kind, both precisions, controls on register, lane,
warp and block bits, controlled-phase fans, parity-diagonal ops,
row-dependent angles, the diagonal-observable epilogue and the adjoint
gradients."""
import math

import numpy as np
import pytest
import torch

import oracle
import workloads as W
from tests.gpu_helpers import assert_amps, assert_rel, dev, np_state, obs_scale
from tests.test_gpu_parity import edge_gates, random_gates

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("CUDA GPU required", allow_module_level=True)

import paper_2512_18995_gb300 as dq  # noqa: E402
from paper_2512_18995_gb300 import build as dqbuild  # noqa: E402

dqbuild.build()


@pytest.fixture(scope="module")
def ctx():
    c = dq.Context(0)
    c.set_path(dq.PATH_FUSED)
    yield c
    c.set_option(dq.OPT_JIT, 2)
    c.close()


def forward(ctx, circ, params, data, batch, dt, n, obs, jit):
    ctx.set_option(dq.OPT_JIT, jit)
    st = torch.empty((batch, 1 << n), dtype=dt, device="cuda")
    ctx.set_tracing(True)
    e, _, _, _ = ctx.forward_grad(circ, params, dq.Observables(obs), batch, dt, data=data, want_grad=False,
                                  state_out=st)
    torch.cuda.synchronize()
    names = set(ctx.trace())
    ctx.set_tracing(False)
    ctx.check()
    return st, e, names


@pytest.mark.parametrize("dtype", [torch.complex64, torch.complex128])
@pytest.mark.parametrize("n,batch", [(15, 2), (18, 1)])
def test_jit_random_circuits_match_oracle_and_interpreter(ctx, dtype, n, batch):
    rng = np.random.default_rng(1300 + n)
    gates, npar = random_gates(n, 6 * n, rng, nfeat=3)
    gates = edge_gates(n) + W.qft_gates(n) + gates + [W.Gate("rzz", (1, n - 2), angle=0.4)]
    params = rng.uniform(-4, 4, npar)
    data = rng.uniform(-3, 3, (batch, 3))
    circ = dq.Circuit(n, gates, nparams=npar, nfeatures=3)
    obs = [W.obs_sum_z(n), [W.pauli_term(0.3, {0: "Z", n - 1: "Z"})]]
    st1, e1, names1 = forward(ctx, circ, dev(params), dev(data), batch, dtype, n, obs, 1)
    st0, e0, names0 = forward(ctx, circ, dev(params), dev(data), batch, dtype, n, obs, 0)
    assert "k_tile_fwd_jit" in names1 and "k_tile_fwd" not in names1, names1
    assert "k_tile_fwd_jit" not in names0, names0
    ref = oracle.run(n, gates, params, data, batch=batch)
    assert_amps(np_state(st1), ref, dtype, "specialised passes")
    assert_rel(e1.cpu().numpy(), oracle.expect(n, ref, obs), dtype, "expectations (specialised)",
               zero_scale=obs_scale(obs))
    # the same arithmetic as the interpreter: agreement to rounding
    tol = 1e-6 if dtype == torch.complex64 else 1e-13
    assert float((st1 - st0).abs().max()) <= tol


def test_jit_headline_workload(ctx):
    """The 20-qubit ansatz with the tuned shape, specialised vs oracle."""
    wl = W.config_c2()
    circ = dq.Circuit(wl.n, wl.gates, nparams=wl.nparams)
    st = torch.empty((1, 1 << wl.n), dtype=torch.complex64, device="cuda")
    ctx.plan_autotune(circ, st)
    s1, e1, names = forward(ctx, circ, dev(wl.params), None, 1, torch.complex64, wl.n, wl.observables, 1)
    assert "k_tile_fwd_jit" in names
    ref = oracle.run(wl.n, wl.gates, wl.params)
    assert_amps(np_state(s1), ref, torch.complex64, "C2 specialised state")
    assert_rel(e1.cpu().numpy(), oracle.expect(wl.n, ref, wl.observables), torch.complex64, "C2 <sum Z>",
               zero_scale=obs_scale(wl.observables))


def test_jit_forward_then_adjoint(ctx):
    """A gradient call: specialised forward and reverse passes (the observable
    passes interpreted); gradients against the oracle (QFT fans + ansatz)."""
    n = 17
    wl = W.config_c5(n)
    circ = dq.Circuit(n, wl.gates, nparams=wl.nparams)
    ctx.set_option(dq.OPT_JIT, 1)
    ctx.set_tracing(True)
    e, gp, _, _ = ctx.forward_grad(circ, dev(wl.params), dq.Observables(wl.observables), 1, torch.complex64)
    torch.cuda.synchronize()
    names = set(ctx.trace())
    assert "k_tile_fwd_jit" in names and "k_tile_adj_jit" in names and "k_tile_adj" not in names, names
    ctx.set_tracing(False)
    e_ref, gp_ref, _ = oracle.adjoint(n, wl.gates, wl.observables, wl.params)
    assert_rel(e.cpu().numpy(), e_ref, torch.complex64, "TFIM energy (specialised forward)")
    assert_rel(gp.cpu().numpy(), gp_ref, torch.complex64, "TFIM gradient (specialised forward)")


def test_jit_under_graph_replay(ctx):
    n, batch = 16, 3
    gates = W.encode_layer(n) + W.hea_layers(n, 2)
    circ = dq.Circuit(n, gates, nparams=4 * n, nfeatures=n)
    rng = np.random.default_rng(16)
    params = dev(rng.uniform(0, 6, 4 * n))
    data = dev(rng.uniform(-3, 3, (batch, n)))
    st = torch.empty((batch, 1 << n), dtype=torch.complex64, device="cuda")
    ctx.set_option(dq.OPT_JIT, 1)
    ctx.set_graphs(True)
    try:
        for call in range(3):
            params.copy_(dev(rng.uniform(0, 6, 4 * n)))
            ctx.state_init(st, n)
            ctx.apply_circuit(circ, params, st, data=data)
            torch.cuda.synchronize()
            ref = oracle.run(n, gates, params.cpu().numpy(), data.cpu().numpy(), batch=batch)
            assert_amps(np_state(st), ref, torch.complex64, f"call {call}")
    finally:
        ctx.set_graphs(False)


@pytest.mark.parametrize("dtype", [torch.complex64, torch.complex128])
@pytest.mark.parametrize("ppr", [False, True])
def test_jit_gradients_random_circuits(ctx, dtype, ppr):
    """Specialised reverse passes on random circuits over every kind, shared
    or per-row parameters, data gradients: against the oracle."""
    n, batch = 15, 2
    rng = np.random.default_rng(1500 + ppr)
    gates, npar = random_gates(n, 6 * n, rng, nfeat=2)
    params = rng.uniform(-4, 4, size=(batch, npar) if ppr else npar)
    data = rng.uniform(-3, 3, size=(batch, 2))
    obs = [W.obs_tfim_open(n, 0.5), [(0.7, 1, (1 << n) - 1), (-0.4, 0, 1)]]
    w = rng.normal(size=(batch, 2))
    circ = dq.Circuit(n, gates, nparams=npar, nfeatures=2)
    ctx.set_option(dq.OPT_JIT, 1)
    ctx.set_tracing(True)
    e, gp, gd, _ = ctx.forward_grad(circ, dev(params), dq.Observables(obs), batch, dtype, data=dev(data),
                                    row_weights=dev(w), params_per_row=ppr)
    torch.cuda.synchronize()
    names = set(ctx.trace())
    ctx.set_tracing(False)
    assert "k_tile_adj_jit" in names, names
    e_ref, gp_ref, gd_ref = oracle.adjoint(n, gates, obs, params, data, batch=batch, params_per_row=ppr,
                                           row_weights=w)
    gscale = float(np.abs(w).max(axis=1).sum()) * obs_scale(obs)
    assert_rel(e.cpu().numpy(), e_ref, dtype, "expectations", zero_scale=obs_scale(obs))
    assert_rel(gp.cpu().numpy(), gp_ref, dtype, "grad params (specialised reverse)", zero_scale=gscale)
    assert_rel(gd.cpu().numpy(), gd_ref, dtype, "grad data (specialised reverse)", zero_scale=gscale)


@pytest.mark.parametrize("dtype", [torch.complex64, torch.complex128])
@pytest.mark.parametrize("ppr", [False, True])
def test_jit_whole_row_kernel(ctx, dtype, ppr):
    """The whole-row kernel with the row program compiled in (forward,
    expectations, lambda and the reverse sweep in one kernel): random
    circuits over every kind with parity-diagonal ops, SWAPs, encoded
    features, shared or per-row parameters and a ragged batch, against the
    oracle and the interpreting kernel."""
    n, batch = 10, 37
    rng = np.random.default_rng(1700 + ppr)
    gates, npar = random_gates(n, 8 * n, rng, nfeat=2)
    gates += [W.Gate("rzz", (2, 7), angle=0.6), W.Gate("swap", (0, n - 1)), W.Gate("rxx", (3, 5), angle=1.1)]
    params = rng.uniform(-4, 4, size=(batch, npar) if ppr else npar)
    data = rng.uniform(-3, 3, size=(batch, 2))
    obs = [W.obs_tfim_open(n, 0.5), [(0.7, 1, (1 << n) - 1), (-0.4, 0, 1)]]
    w = rng.normal(size=(batch, 2))
    circ = dq.Circuit(n, gates, nparams=npar, nfeatures=2)
    out = {}
    for jit in (1, 0):
        ctx.set_option(dq.OPT_JIT, jit)
        st = torch.empty((batch, 1 << n), dtype=dtype, device="cuda")
        ctx.set_tracing(True)
        e, gp, gd, _ = ctx.forward_grad(circ, dev(params), dq.Observables(obs), batch, dtype, data=dev(data),
                                        row_weights=dev(w), params_per_row=ppr, state_out=st)
        torch.cuda.synchronize()
        names = set(ctx.trace())
        ctx.set_tracing(False)
        ctx.check()
        assert ("k_rows_jit" in names) == (jit == 1) and ("k_rows" in names) == (jit == 0), names
        out[jit] = (st, e, gp, gd)
    st, e, gp, gd = out[1]
    ref = oracle.run(n, gates, params, data, batch=batch, params_per_row=ppr)
    assert_amps(np_state(st), ref, dtype, "whole-row kernel (specialised)")
    e_ref, gp_ref, gd_ref = oracle.adjoint(n, gates, obs, params, data, batch=batch, params_per_row=ppr,
                                           row_weights=w)
    gscale = float(np.abs(w).max(axis=1).sum()) * obs_scale(obs)
    assert_rel(e.cpu().numpy(), e_ref, dtype, "expectations (specialised rows)", zero_scale=obs_scale(obs))
    assert_rel(gp.cpu().numpy(), gp_ref, dtype, "grad params (specialised rows)", zero_scale=gscale)
    assert_rel(gd.cpu().numpy(), gd_ref, dtype, "grad data (specialised rows)", zero_scale=gscale)
    tol = 1e-5 if dtype == torch.complex64 else 1e-12
    assert float((out[1][0] - out[0][0]).abs().max()) <= tol


def test_jit_whole_row_autotuned(ctx):
    """DQ_OPT_JIT = 2: dq_plan_autotune times the whole-row kernel both ways
    and keeps one; results hold either way, and a later tile tuning of the
    same plan keeps the choice."""
    wl = W.config_c3(batch=256)
    circ = dq.Circuit(wl.n, wl.gates, nparams=wl.nparams, nfeatures=wl.nfeatures)
    ctx.set_option(dq.OPT_JIT, 2)
    st = torch.empty((wl.batch, 1 << wl.n), dtype=torch.complex64, device="cuda")
    ctx.plan_autotune(circ, st)
    ctx.set_tracing(True)
    e, gp, gd, _ = ctx.forward_grad(circ, dev(wl.params), dq.Observables(wl.observables), wl.batch, torch.complex64,
                                    data=dev(wl.data))
    torch.cuda.synchronize()
    names = set(ctx.trace())
    ctx.set_tracing(False)
    assert ("k_rows_jit" in names) != ("k_rows" in names), names
    e_ref, gp_ref, gd_ref = oracle.adjoint(wl.n, wl.gates, wl.observables, wl.params, wl.data, batch=wl.batch)
    scale = obs_scale(wl.observables)
    assert_rel(e.cpu().numpy(), e_ref, torch.complex64, "expectations (autotuned rows)", zero_scale=scale)
    assert_rel(gp.cpu().numpy(), gp_ref, torch.complex64, "grad params (autotuned rows)", zero_scale=wl.batch * scale)
    assert_rel(gd.cpu().numpy(), gd_ref, torch.complex64, "grad data (autotuned rows)", zero_scale=scale)


def test_pinned_tile_shape():
    """dq_plan_set_tile: a pinned shape with specialised passes is what later
    forward calls run (DQ_OPT_JIT = 2, no tuning), reported by plan_tuned,
    with results against the oracle; shapes out of range or without a
    schedule are refused."""
    n = 17
    rng = np.random.default_rng(1717)
    gates, npar = random_gates(n, 5 * n, rng)
    params = rng.uniform(-4, 4, npar)
    circ = dq.Circuit(n, gates, nparams=npar)
    obs = [W.obs_sum_z(n)]
    ctx = dq.Context(0)
    ctx.set_path(dq.PATH_FUSED)
    try:
        ctx.set_option(dq.OPT_JIT, 2)
        ctx.plan_set_tile(circ, 11, 5, 4, jit=True)
        assert ctx.plan_tuned(circ) == (11, 5, 4)
        st, e, names = forward(ctx, circ, dev(params), None, 1, torch.complex64, n, obs, 2)
        assert "k_tile_fwd_jit" in names, names
        ref = oracle.run(n, gates, params)
        assert_amps(np_state(st), ref, torch.complex64, "pinned shape, specialised")
        ctx.plan_set_tile(circ, 12, 5, 3, jit=False)
        st, e, names = forward(ctx, circ, dev(params), None, 1, torch.complex64, n, obs, 2)
        assert "k_tile_fwd_jit" not in names and ctx.plan_tuned(circ) == (12, 5, 3), names
        assert_amps(np_state(st), ref, torch.complex64, "pinned shape, interpreted")
        for bad in ((4, 5, 4), (12, 5, 9), (12, 11, 4), (16, 5, 2)):
            with pytest.raises(dq.DQError) as ei:
                ctx.plan_set_tile(circ, *bad)
            assert ei.value.status == 1, bad
        lib = dq.load_library()   # the C check of the jit flag (the binding passes a bool)
        assert lib.dq_plan_set_tile(ctx.h, circ.ref(), 0, 11, 5, 4, 2) == 1
    finally:
        ctx.set_option(dq.OPT_JIT, 2)
        ctx.close()


CACHE_CHILD = r"""
import os, sys, time, json
import numpy as np, torch
sys.path.insert(0, os.getcwd())
import workloads as W, paper_2512_18995_gb300 as dq
n = 10
gates = W.hea_layers(n, 2) + [W.Gate("rzz", (1, 8), angle=0.4)]
circ = dq.Circuit(n, gates, nparams=4 * n)
ctx = dq.Context(0)
ctx.set_path(dq.PATH_FUSED)
ctx.set_option(dq.OPT_JIT, 1)
params = torch.linspace(0.1, 3.0, 4 * n, dtype=torch.float64, device="cuda")
ctx.set_tracing(True)
t0 = time.time()
e, gp, _, _ = ctx.forward_grad(circ, params, dq.Observables([W.obs_sum_z(n)]), 3, torch.complex64)
torch.cuda.synchronize()
dt = time.time() - t0
names = sorted(ctx.trace())
ctx.check()
print("RESULT", json.dumps({"s": dt, "names": names, "e": float(e[0, 0]), "g": gp.cpu().tolist()}))
"""


def test_compiled_program_cache(tmp_path):
    """Specialised programs are kept on disk (DQ_JIT_CACHE): the first process
    compiles and writes the cubin, a second process with the same circuit
    loads it (no new file) and gets identical results."""
    import json
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, DQ_JIT_CACHE=str(tmp_path))
    runs = []
    for _ in range(2):
        r = subprocess.run([sys.executable, "-c", CACHE_CHILD], cwd=root, env=env, capture_output=True, text=True,
                           timeout=600)
        line = [x for x in r.stdout.splitlines() if x.startswith("RESULT ")]
        assert r.returncode == 0 and line, r.stdout[-2000:] + r.stderr[-2000:]
        runs.append((json.loads(line[0][7:]), sorted(p.name for p in tmp_path.iterdir())))
    (first, files1), (second, files2) = runs
    assert "k_rows_jit" in first["names"] and "k_rows_jit" in second["names"], first["names"]
    assert len(files1) == 1 and files1[0].endswith(".cubin") and files2 == files1
    assert first["e"] == second["e"] and first["g"] == second["g"]


@pytest.mark.parametrize("jit", [0, 1])
def test_two_rows_per_cta(jit):
    """DQ_OPT_ROWS_PER_CTA = 2: the CTA's two halves run two rows of the
    whole-row kernel in step (interpreting or specialised), a ragged batch
    leaves the last CTA's second half without a row; expectations, shared and
    per-row gradients and the states against the oracle and against one row
    per CTA."""
    n, batch = 10, 37
    rng = np.random.default_rng(2100 + jit)
    gates, npar = random_gates(n, 6 * n, rng, nfeat=2)
    gates += [W.Gate("rzz", (2, 7), angle=0.6), W.Gate("swap", (0, n - 1))]
    params = rng.uniform(-4, 4, npar)
    data = rng.uniform(-3, 3, size=(batch, 2))
    obs = [W.obs_tfim_open(n, 0.5), [(0.7, 1, (1 << n) - 1), (-0.4, 0, 1)]]
    w = rng.normal(size=(batch, 2))
    circ = dq.Circuit(n, gates, nparams=npar, nfeatures=2)
    ctx = dq.Context(0)
    ctx.set_path(dq.PATH_FUSED)
    ctx.set_option(dq.OPT_JIT, jit)
    out = {}
    try:
        for rpc in (2, 1):
            ctx.set_option(dq.OPT_ROWS_PER_CTA, rpc)
            st = torch.empty((batch, 1 << n), dtype=torch.complex64, device="cuda")
            ctx.set_tracing(True)
            e, gp, gd, _ = ctx.forward_grad(circ, dev(params), dq.Observables(obs), batch, torch.complex64,
                                            data=dev(data), row_weights=dev(w), state_out=st)
            torch.cuda.synchronize()
            names = set(ctx.trace())
            ctx.set_tracing(False)
            ctx.check()
            assert ("k_rows_jit" if jit else "k_rows") in names, names
            out[rpc] = (st, e, gp, gd)
        st, e, gp, gd = out[2]
        ref = oracle.run(n, gates, params, data, batch=batch)
        assert_amps(np_state(st), ref, torch.complex64, "two rows per CTA")
        e_ref, gp_ref, gd_ref = oracle.adjoint(n, gates, obs, params, data, batch=batch, row_weights=w)
        gscale = float(np.abs(w).max(axis=1).sum()) * obs_scale(obs)
        assert_rel(e.cpu().numpy(), e_ref, torch.complex64, "expectations (two rows per CTA)", zero_scale=obs_scale(obs))
        assert_rel(gp.cpu().numpy(), gp_ref, torch.complex64, "grad params (two rows per CTA)", zero_scale=gscale)
        assert_rel(gd.cpu().numpy(), gd_ref, torch.complex64, "grad data (two rows per CTA)", zero_scale=gscale)
        # the same rows as one row per CTA (only the FP64 fold order of the shared sums differs)
        assert torch.equal(out[2][0], out[1][0]) and torch.equal(out[2][1], out[1][1])
        assert torch.equal(out[2][3], out[1][3])
        assert float((out[2][2] - out[1][2]).abs().max()) <= 1e-12 * max(1.0, float(out[1][2].abs().max()))
        with pytest.raises(dq.DQError):
            ctx.set_option(dq.OPT_ROWS_PER_CTA, 3)
    finally:
        ctx.close()
