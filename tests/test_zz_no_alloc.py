"""The allocation-free entry point, dq_forward_grad_noalloc.

Some callers cannot allocate device memory while they run: a serving loop
that reserves all of its memory at start-up (cudaMalloc and cudaFree can
synchronise or stall the whole device in the middle of a request), or a host
application whose own allocator owns the GPU's memory and hands out nothing
else.  This entry point keeps its scratch in one static device array that all
calls share, so the test makes two calls in a row with different inputs and
checks each against the FP64 oracle and against the regular entry point
(dq_forward_grad), within the parity tolerance of the other GPU tests.  It
also checks the refusals: a circuit or batch beyond the static array, and a
stream that is being captured into a graph.

This file is collected last on purpose, and passes alone in a fresh process
as well as after the other tests.
"""
import numpy as np
import pytest
import torch

import oracle
import workloads as W
from tests.gpu_helpers import assert_rel, obs_scale

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("CUDA GPU required", allow_module_level=True)

import paper_2512_18995_gb300 as dq  # noqa: E402
from paper_2512_18995_gb300 import _lib  # noqa: E402
from paper_2512_18995_gb300 import build as dqbuild  # noqa: E402

dqbuild.build()


@pytest.mark.parametrize("dtype", [torch.complex64, torch.complex128])
@pytest.mark.parametrize("ppr", [False, True])
def test_noalloc_matches_oracle_twice(dtype, ppr):
    n, batch = 10, 96
    gates = W.encode_layer(n) + W.hea_layers(n, 3) + [W.Gate("cry", (2, 7), param=60), W.Gate("swap", (0, 9))]
    nparams = 61
    circ = dq.Circuit(n, gates, nparams=nparams, nfeatures=n)
    obs = [W.obs_z(0), W.obs_tfim_open(n, 0.5)]
    dobs = dq.Observables(obs)
    ctx = dq.Context(torch.cuda.current_device())
    rng = np.random.default_rng(2024 + ppr)
    try:
        for call in range(2):
            shape = (batch, nparams) if ppr else (nparams,)
            p_np = rng.uniform(0, 2 * np.pi, shape)
            x_np = rng.uniform(-np.pi, np.pi, (batch, n))
            w_np = rng.normal(size=(batch, 2))
            params = torch.tensor(p_np, device="cuda")
            data = torch.tensor(x_np, device="cuda")
            w = torch.tensor(w_np, device="cuda")
            e1, gp1, gd1 = _lib.forward_grad_noalloc(circ, params, dobs, batch, dtype, data=data, row_weights=w,
                                                     params_per_row=ppr)
            e0, gp0, gd0, _ = ctx.forward_grad(circ, params, dobs, batch, dtype, data=data, row_weights=w,
                                               params_per_row=ppr)
            torch.cuda.synchronize()
            e_ref, gp_ref, gd_ref = oracle.adjoint(n, gates, obs, p_np, x_np, batch=batch, params_per_row=ppr,
                                                   row_weights=w_np)
            gscale = float(np.abs(w_np).max(axis=1).sum()) * obs_scale(obs)
            # against the oracle
            assert_rel(e1.cpu().numpy(), e_ref, dtype, f"call {call}: expectations", zero_scale=obs_scale(obs))
            assert_rel(gp1.cpu().numpy(), gp_ref, dtype, f"call {call}: grad params", zero_scale=gscale)
            assert_rel(gd1.cpu().numpy(), gd_ref, dtype, f"call {call}: grad data", zero_scale=gscale)
            # and against the regular entry point
            assert_rel(e1.cpu().numpy(), e0.cpu().numpy(), dtype, f"call {call}: expectations vs forward_grad",
                       zero_scale=obs_scale(obs))
            assert_rel(gp1.cpu().numpy(), gp0.cpu().numpy(), dtype, f"call {call}: grad params vs forward_grad",
                       zero_scale=gscale)
            assert_rel(gd1.cpu().numpy(), gd0.cpu().numpy(), dtype, f"call {call}: grad data vs forward_grad",
                       zero_scale=gscale)
    finally:
        ctx.close()


def test_noalloc_rejects_what_does_not_fit():
    n = 16
    circ = dq.Circuit(n, [W.Gate("h", (0,))])
    with pytest.raises(dq.DQError) as ei:
        _lib.forward_grad_noalloc(circ, None, dq.Observables([W.obs_z(0)]), 1, torch.complex64)
    assert ei.value.status == 2
    assert "on-chip" in str(ei.value)
    # a batch whose coefficient table exceeds the static array
    n = 8
    gates = [W.Gate("ry", (q % n,), data=q) for q in range(64)]
    circ = dq.Circuit(n, gates, nfeatures=64)
    batch = 8192
    data = torch.zeros((batch, 64), dtype=torch.float64, device="cuda")
    with pytest.raises(dq.DQError) as ei:
        _lib.forward_grad_noalloc(circ, None, dq.Observables([W.obs_z(0)]), batch, torch.complex128, data=data)
    assert ei.value.status == 2
    assert "static limit" in str(ei.value)


def test_noalloc_refuses_a_capturing_stream():
    """Its tables come from host buffers that live only during the call, so
    the entry point must not be recorded into a graph: it returns
    DQ_ERR_UNSUPPORTED on a capturing stream and enqueues nothing."""
    n, batch = 6, 4
    gates = W.hea_layers(n, 1)
    circ = dq.Circuit(n, gates, nparams=2 * n)
    dobs = dq.Observables([W.obs_z(0)])
    params = torch.zeros(2 * n, dtype=torch.float64, device="cuda")
    e = torch.empty((batch, 1), dtype=torch.float64, device="cuda")
    gp = torch.empty(2 * n, dtype=torch.float64, device="cuda")
    pad = torch.zeros(1, device="cuda")
    graph = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        graph.capture_begin()
        try:
            pad.add_(1.0)          # keeps the captured graph non-empty
            with pytest.raises(dq.DQError) as ei:
                _lib.forward_grad_noalloc(circ, params, dobs, batch, torch.complex64, expect_out=e,
                                          grad_params=gp)
        finally:
            graph.capture_end()
    torch.cuda.current_stream().wait_stream(side)
    assert ei.value.status == 2
    assert "capturing" in str(ei.value)
    # the same call on an ordinary stream still works afterwards
    _lib.forward_grad_noalloc(circ, params, dobs, batch, torch.complex64, expect_out=e, grad_params=gp)
    torch.cuda.synchronize()
    assert np.allclose(e.cpu().numpy(), 1.0, atol=1e-5)     # all angles zero: |0...0>, <Z0> = 1
