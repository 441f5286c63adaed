"""Parity in the headline benchmark's own launch configuration: the 20-qubit,
8-layer ansatz (480 gates, 320 parameters) on the autotuned fused schedule
with CUDA-graph replay and an L2 flush between steps, called exactly as
bench.py times it.  Every step -- issued directly, captured, then replayed --
must give the oracle's final state and <sum Z>.  (Named to run last.)"""
import pytest
import torch

import oracle
import workloads as W
from tests.gpu_helpers import assert_amps, assert_rel, np_state, obs_scale

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("CUDA GPU required", allow_module_level=True)

import paper_2512_18995_gb300 as dq  # noqa: E402
from paper_2512_18995_gb300 import build as dqbuild  # noqa: E402

dqbuild.build()


def test_c2_autotuned_graph_replay_matches_oracle():
    wl = W.config_c2()
    n = wl.n
    ref = oracle.run(n, wl.gates, wl.params)
    e_ref = oracle.expect(n, ref, wl.observables)
    ctx = dq.Context(0)
    try:
        circ = dq.Circuit(n, wl.gates, nparams=wl.nparams)
        obs = dq.Observables(wl.observables)
        params = torch.tensor(wl.params, dtype=torch.float64, device="cuda")
        state = torch.empty((1, 1 << n), dtype=torch.complex64, device="cuda")
        expect = torch.empty((1, 1), dtype=torch.float64, device="cuda")
        flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")
        ctx.plan_autotune(circ, state)
        ctx.set_graphs(True)
        for step in range(5):
            flush.zero_()
            state.zero_()                      # the step itself must write the whole state
            ctx.forward_grad(circ, params, obs, 1, torch.complex64, want_grad=False, state_out=state,
                             expect_out=expect)
            torch.cuda.synchronize()
            ctx.check()
            assert_amps(np_state(state), ref, torch.complex64, f"step {step}: state")
            assert_rel(expect.cpu().numpy(), e_ref, torch.complex64, f"step {step}: <sum Z>",
                       zero_scale=obs_scale(wl.observables))
    finally:
        ctx.set_graphs(False)
        ctx.close()
