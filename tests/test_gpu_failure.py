"""Failure detection without a GPU fault, and the FP64 norm reduction.

* A device-side bounded wait that runs out (a barrier nothing arrives on, no
  copy in flight, the context's wait limit lowered to 1 ms) surfaces as
  DQ_ERR_TIMEOUT from the next check, and the context keeps working.
* A caller-attached workspace one byte smaller than a call needs gives
  DQ_ERR_OOM before anything is launched; the exact size then works.
* dq_state_norm: <psi|psi> per row with FP64 accumulation, against FP64 sums
  of the same amplitudes, and the norm drift of an FP32 evolution."""
import math
import re

import numpy as np
import pytest
import torch

import oracle
import workloads as W
from tests.gpu_helpers import assert_amps, assert_rel, dev, np_state

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("CUDA GPU required", allow_module_level=True)

import paper_2512_18995_gb300 as dq  # noqa: E402
from paper_2512_18995_gb300 import build as dqbuild  # noqa: E402

dqbuild.build()

DQ_ERR_INVALID_ARG, DQ_ERR_OOM, DQ_ERR_TIMEOUT = 1, 3, 5


def test_bounded_wait_expiry_surfaces_as_timeout():
    ctx = dq.Context(0)
    try:
        ctx.set_option(dq.OPT_WAIT_LIMIT_US, 1000)
        ctx.selftest_wait_expiry()
        with pytest.raises(dq.DQError) as ei:
            ctx.check()
        assert ei.value.status == DQ_ERR_TIMEOUT
        ctx.check()                                   # the flag was cleared
        ctx.set_option(dq.OPT_WAIT_LIMIT_US, 2000000)
        # the context still computes correctly (tile path with bounded waits)
        n = 16
        gates = W.hea_layers(n, 2)
        params = np.linspace(0.1, 3.0, 4 * n)
        st = torch.empty((1, 1 << n), dtype=torch.complex64, device="cuda")
        ctx.set_path(dq.PATH_FUSED)
        ctx.state_init(st, n)
        ctx.apply_circuit(dq.Circuit(n, gates, nparams=4 * n), dev(params), st)
        ctx.check()
        assert_amps(np_state(st), oracle.run(n, gates, params), torch.complex64)
    finally:
        ctx.close()


@pytest.mark.parametrize("bad", [0, -5, 60000001])
def test_wait_limit_out_of_range_is_rejected(bad):
    ctx = dq.Context(0)
    try:
        with pytest.raises(dq.DQError) as ei:
            ctx.set_option(dq.OPT_WAIT_LIMIT_US, bad)
        assert ei.value.status == DQ_ERR_INVALID_ARG
        with pytest.raises(dq.DQError):
            ctx.set_option(99, 1)
    finally:
        ctx.close()


def test_workspace_one_byte_short_is_oom():
    ctx = dq.Context(0)
    ctx.ensure_workspace = lambda *a, **k: None        # the binding must not resize what the test attaches
    n, batch = 16, 2
    gates = W.encode_layer(n) + W.hea_layers(n, 1)
    circ = dq.Circuit(n, gates, nparams=2 * n, nfeatures=n)
    obs = dq.Observables([W.obs_tfim_open(n, 0.5)])
    rng = np.random.default_rng(16)
    params = dev(rng.uniform(0, 6, 2 * n))
    data = dev(rng.uniform(-3, 3, (batch, n)))
    e = torch.full((batch, 1), 7.0, dtype=torch.float64, device="cuda")
    gp = torch.full((2 * n,), 7.0, dtype=torch.float64, device="cuda")
    gd = torch.full((batch, n), 7.0, dtype=torch.float64, device="cuda")
    ws = torch.empty(64 << 20, dtype=torch.uint8, device="cuda")

    def attach(nbytes):
        ctx._check(ctx.lib.dq_ctx_set_workspace(ctx.h, None, 0), "detach")
        ctx._check(ctx.lib.dq_ctx_set_workspace(ctx.h, ws.data_ptr(), int(nbytes)), "attach")

    def call():
        return ctx.forward_grad(circ, params, obs, batch, torch.complex64, data=data, expect_out=e,
                                grad_params=gp, grad_data=gd)

    try:
        ctx.set_path(dq.PATH_FUSED)
        attach(64)
        with pytest.raises(dq.DQError) as ei:
            call()
        assert ei.value.status == DQ_ERR_OOM
        need = int(re.search(r"than the (\d+) bytes needed", str(ei.value)).group(1))
        assert 64 < need <= ws.numel()
        attach(need - 1)
        l0 = ctx.launch_count
        with pytest.raises(dq.DQError) as ei:
            call()
        assert ei.value.status == DQ_ERR_OOM
        torch.cuda.synchronize()
        assert ctx.launch_count == l0, "nothing may be launched when the workspace is short"
        assert bool((e == 7.0).all()) and bool((gp == 7.0).all()) and bool((gd == 7.0).all())
        attach(need)
        call()
        torch.cuda.synchronize()
        ctx.check()
        e_ref, gp_ref, gd_ref = oracle.adjoint(n, gates, [W.obs_tfim_open(n, 0.5)], params.cpu().numpy(),
                                               data.cpu().numpy(), batch=batch)
        assert_rel(e.cpu().numpy(), e_ref, torch.complex64, "expectations (exact workspace)")
        assert_rel(gp.cpu().numpy(), gp_ref, torch.complex64, "grad params (exact workspace)")
        assert_rel(gd.cpu().numpy(), gd_ref, torch.complex64, "grad data (exact workspace)")
    finally:
        ctx._check(ctx.lib.dq_ctx_set_workspace(ctx.h, None, 0), "detach")
        ctx.close()


@pytest.mark.parametrize("dtype,n,batch", [(torch.complex64, 1, 3), (torch.complex64, 12, 5),
                                           (torch.complex64, 22, 2), (torch.complex128, 0, 2),
                                           (torch.complex128, 9, 7), (torch.complex128, 20, 1)])
def test_state_norm_fp64(dtype, n, batch):
    ctx = dq.Context(0)
    try:
        g = torch.Generator(device="cuda").manual_seed(100 + n)
        st = torch.randn((batch, 1 << n), dtype=dtype, device="cuda", generator=g) * 0.37
        got = ctx.state_norm(st, n).cpu().numpy()
        ref = (np.abs(st.cpu().numpy().astype(np.complex128)) ** 2).sum(axis=1)
        tol = 1e-13 if dtype == torch.complex128 else 1e-6     # products and 8-term runs in the state's precision
        assert np.max(np.abs(got - ref) / ref) <= tol
        assert ctx.state_norm(st[:0].reshape(0, 1 << n), n).numel() == 0
    finally:
        ctx.close()


def test_norm_drift_of_fp32_evolution():
    """The 17-qubit QFT + 10-layer ansatz (1073 gates) in complex64: the norm
    drifts by FP32 rounding only (|<psi|psi> - 1| well below the amplitude
    tolerance), and the FP64 norm of the complex128 run is 1 to 1e-12."""
    n = 17
    wl = W.config_c5(n)
    circ = dq.Circuit(n, wl.gates, nparams=wl.nparams)
    ctx = dq.Context(0)
    try:
        for dt, tol in ((torch.complex64, 1e-5), (torch.complex128, 1e-12)):
            st = torch.empty((1, 1 << n), dtype=dt, device="cuda")
            ctx.state_init(st, n)
            ctx.apply_circuit(circ, dev(wl.params), st)
            drift = abs(float(ctx.state_norm(st, n).item()) - 1.0)
            assert drift <= tol, (dt, drift)
    finally:
        ctx.close()


BOUNDS_CHILD = r"""
import os, sys
import numpy as np, torch
sys.path.insert(0, os.getcwd())
from paper_2512_18995_gb300 import build as b
b.build(debug=True)
import paper_2512_18995_gb300 as dq
from paper_2512_18995_gb300 import _lib
import oracle, workloads as W
assert _lib.LIB_PATH.endswith("libdq_debug.so"), _lib.LIB_PATH
ctx = dq.Context(0)
ctx.selftest_bounds()
try:
    ctx.check()
    raise SystemExit("the failing check was not reported")
except dq.DQError as e:
    assert e.status == 4 and "bounds check" in str(e) and "k_norm.cu" in str(e), str(e)
ctx.check()   # cleared
rng = np.random.default_rng(7)
def run(path, n, gates, npar, nfeat, batch, dtype, obs, tol):
    ctx.set_path(path)
    params = rng.uniform(-3, 3, npar)
    data = rng.uniform(-3, 3, (batch, nfeat)) if nfeat else None
    circ = dq.Circuit(n, gates, nparams=npar, nfeatures=nfeat)
    e, gp, gd, _ = ctx.forward_grad(circ, torch.tensor(params, device="cuda"), dq.Observables(obs), batch, dtype,
                                    data=None if data is None else torch.tensor(data, device="cuda"))
    ctx.check()   # no index outside its buffer
    e_ref, gp_ref, gd_ref = oracle.adjoint(n, gates, obs, params, data, batch=batch)
    scale = sum(abs(t[0]) for o in obs for t in o)
    err = max(np.max(np.abs(e.cpu().numpy() - e_ref)), np.max(np.abs(gp.cpu().numpy() - gp_ref)) / batch)
    assert err <= tol * scale, (path, n, err)
# per-gate path, complex128: swaps, controlled rotations, a parity-diagonal gate, X/Y terms
n = 9
g = W.encode_layer(n) + W.hea_layers(n, 2, first_param=0) + [W.Gate("swap", (1, 7)), W.Gate("crx", (0, 5), angle=0.4),
                                                           W.Gate("rzz", (2, 6), param=4 * n)]
obs = [W.obs_tfim_open(n, 0.5), [W.pauli_term(0.3, {0: "X", 4: "Y"})]]
run(dq.PATH_PLAIN, n, g, 4 * n + 1, n, 3, torch.complex128, obs, 1e-10)
# whole-row kernel (fused, 10 qubits, complex64)
n = 10
g = W.encode_layer(n) + W.hea_layers(n, 2) + [W.Gate("rzz", (1, 8), angle=0.3)]
run(dq.PATH_FUSED, n, g, 4 * n, n, 5, torch.complex64, [W.obs_tfim_open(n, 0.5)], 1e-4)
# tile passes: forward, observable and reverse passes (16 qubits, complex64)
n = 16
g = W.qft_gates(n) + W.hea_layers(n, 2)
run(dq.PATH_FUSED, n, g, 4 * n, 0, 1, torch.complex64, [W.obs_tfim_open(n, 0.5)], 1e-4)
ctx.close()
print("bounds ok")
"""


def test_bounds_checking_build():
    """The bounds-checking build (libdq_debug.so, DQ_DEBUG_BOUNDS): a check
    that fails on purpose (no memory touched) is reported by the next
    check() with its source site, then the per-gate, whole-row and tile
    paths run with every checked index inside its buffer and match the
    oracle.  The normal build refuses the self-test."""
    import os
    import subprocess
    import sys
    ctx = dq.Context(0)
    try:
        with pytest.raises(dq.DQError) as ei:
            ctx.selftest_bounds()
        assert ei.value.status == 2
    finally:
        ctx.close()
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, DQ_DEBUG_BOUNDS="1")
    r = subprocess.run([sys.executable, "-c", BOUNDS_CHILD], cwd=root, env=env, capture_output=True, text=True,
                       timeout=900)
    assert r.returncode == 0 and "bounds ok" in r.stdout, r.stdout[-3000:] + r.stderr[-3000:]
