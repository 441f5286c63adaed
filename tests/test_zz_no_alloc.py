"""The allocation-free entry point against the regular one.

dq_forward_grad_noalloc serves callers that may not allocate device memory
at call time (for example serving loops that reserve everything at start-up,
because cudaMalloc and cudaFree can stall the whole device, or hosts whose
own allocator owns the GPU's memory).  Its scratch is a static device array
shared by all calls, so the test makes two calls in a row with different
inputs and checks each against dq_forward_grad, within the parity tolerance
of the other GPU tests.  This file is collected last on purpose.
"""
import numpy as np
import pytest
import torch

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
def test_noalloc_matches_forward_grad_twice(dtype, ppr):
    n, batch = 10, 96
    gates = W.encode_layer(n) + W.hea_layers(n, 3) + [W.Gate("cry", (2, 7), param=60), W.Gate("swap", (0, 9))]
    nparams = 61
    circ = dq.Circuit(n, gates, nparams=nparams, nfeatures=n)
    obs = [W.obs_z(0), W.obs_tfim_open(n, 0.5)]
    dobs = dq.Observables(obs)
    ctx = dq.Context(torch.cuda.current_device())
    rng = np.random.default_rng(2024 + ppr)
    tol_dtype = dtype
    for call in range(2):
        shape = (batch, nparams) if ppr else (nparams,)
        params = torch.tensor(rng.uniform(0, 2 * np.pi, shape), device="cuda")
        data = torch.tensor(rng.uniform(-np.pi, np.pi, (batch, n)), device="cuda")
        w = torch.tensor(rng.normal(size=(batch, 2)), device="cuda")
        e0, gp0, gd0, _ = ctx.forward_grad(circ, params, dobs, batch, dtype, data=data, row_weights=w,
                                           params_per_row=ppr)
        e1, gp1, gd1 = _lib.forward_grad_noalloc(circ, params, dobs, batch, dtype, data=data, row_weights=w,
                                                 params_per_row=ppr)
        torch.cuda.synchronize()
        floor = float(w.abs().max(dim=1).values.sum()) * obs_scale(obs)
        assert_rel(e1.cpu().numpy(), e0.cpu().numpy(), tol_dtype, f"call {call}: expectations", obs_scale(obs))
        assert_rel(gp1.cpu().numpy(), gp0.cpu().numpy(), tol_dtype, f"call {call}: grad params", floor)
        assert_rel(gd1.cpu().numpy(), gd0.cpu().numpy(), tol_dtype, f"call {call}: grad data", floor)
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
