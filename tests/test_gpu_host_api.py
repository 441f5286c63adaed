"""GPU parity of dq_forward_host (the forward path with host buffers: inputs
copied in, expectations copied back, the stream synchronised) against the
FP64 oracle: pinned and pageable buffers, graphs on and off, repeated calls
whose pinned parameters change in place between calls (replays of one CUDA
graph must read the new values), several rows, the 20-qubit ansatz of the
headline workload, and the rejection of circuits with encoded data."""
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
from paper_2512_18995_gb300 import build as dqbuild  # noqa: E402

dqbuild.build()

DTYPES = {"c64": torch.complex64, "c128": torch.complex128}


@pytest.fixture(scope="module")
def ctx():
    c = dq.Context(0)
    yield c
    c.close()


def reference(n, gates, params, observables):
    return oracle.expect(n, oracle.run(n, gates, params), observables)[0]


@pytest.mark.parametrize("dtype", sorted(DTYPES))
@pytest.mark.parametrize("pinned", [True, False])
@pytest.mark.parametrize("graphs", [True, False])
@pytest.mark.parametrize("n,layers,batch", [(6, 2, 1), (13, 3, 2), (16, 2, 1)])
def test_forward_host_matches_oracle(ctx, dtype, pinned, graphs, n, layers, batch):
    dt = DTYPES[dtype]
    gates = W.hea_layers(n, layers)
    nparams = 2 * n * layers
    circ = dq.Circuit(n, gates, nparams=nparams)
    observables = [W.obs_sum_z(n), W.obs_tfim_open(n, 0.7), W.obs_z(n - 1)]
    obs = dq.Observables(observables)
    ctx.set_graphs(graphs)
    try:
        p = torch.empty(nparams, dtype=torch.float64)
        e = torch.empty((batch, len(observables)), dtype=torch.float64)
        if pinned:
            p, e = p.pin_memory(), e.pin_memory()
        # four calls with new values written into the same host buffers: the
        # second captures the call's graph, later ones replay it
        for k in range(4):
            vals = W.uniform_array(1000 * n + 10 * layers + k, nparams, -np.pi, np.pi)
            p.copy_(torch.from_numpy(vals))
            e.fill_(np.nan)
            out = ctx.forward_host(circ, p, obs, batch, dt, expect_out=e)
            assert out.data_ptr() == e.data_ptr()
            ctx.check()
            ref = reference(n, gates, vals, observables)
            got = e.numpy()
            for r in range(batch):
                assert_rel(got[r], ref, dt, f"call {k} row {r}", zero_scale=obs_scale(observables))
    finally:
        ctx.set_graphs(False)


def test_forward_host_headline_workload(ctx):
    """The 20-qubit, 8-layer ansatz (480 gates) with <sum Z>, graphs on,
    pinned buffers, as the end-to-end benchmark calls it."""
    wl = W.config_c2()
    circ = dq.Circuit(wl.n, wl.gates, nparams=wl.nparams)
    obs = dq.Observables(wl.observables)
    ref = oracle.expect(wl.n, oracle.run(wl.n, wl.gates, wl.params), wl.observables)[0]
    ctx.set_graphs(True)
    try:
        p = torch.tensor(wl.params, dtype=torch.float64).pin_memory()
        e = torch.empty((1, 1), dtype=torch.float64).pin_memory()
        for _ in range(3):
            e.fill_(np.nan)
            ctx.forward_host(circ, p, obs, 1, torch.complex64, expect_out=e)
            assert_rel(e.numpy()[0], ref, torch.complex64, "c2 <sum Z>", zero_scale=obs_scale(wl.observables))
    finally:
        ctx.set_graphs(False)


def test_forward_host_rejections(ctx):
    obs = dq.Observables([W.obs_z(0)])
    enc = dq.Circuit(3, [W.Gate("ry", (0,), data=0), W.Gate("rx", (1,), param=0)])
    with pytest.raises(dq.DQError) as err:
        ctx.forward_host(enc, torch.zeros(1, dtype=torch.float64), obs, 1)
    assert err.value.status == 2     # DQ_ERR_UNSUPPORTED
    circ = dq.Circuit(3, [W.Gate("rx", (1,), param=0)])
    with pytest.raises(dq.DQError):          # device tensors are not host buffers
        ctx.forward_host(circ, torch.zeros(1, dtype=torch.float64, device="cuda"), obs, 1)
    with pytest.raises(dq.DQError):          # too few parameters
        ctx.forward_host(circ, torch.zeros(0, dtype=torch.float64), obs, 1)
    e = torch.zeros((0, 1), dtype=torch.float64)
    assert ctx.forward_host(circ, torch.zeros(1, dtype=torch.float64), obs, 0, expect_out=e) is e
