"""The persistent multi-pass forward kernel (k_tile_multi) for states that
stay in L2: every forward tile pass in one launch, the passes separated by a
bounded grid barrier.  It must give exactly what one launch per pass gives
(same arithmetic in the same order on every tile), and match the oracle."""
import math

import numpy as np
import pytest
import torch

import oracle
import workloads as W
from tests.gpu_helpers import assert_amps, assert_rel, dev, np_state, obs_scale

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
    c.set_option(dq.OPT_MULTIPASS, 1)
    c.close()


def run(ctx, circ, params, data, batch, dt, n, obs, multi):
    ctx.set_option(dq.OPT_MULTIPASS, int(multi))
    st = torch.empty((batch, 1 << n), dtype=dt, device="cuda")
    ctx.set_tracing(True)
    e, _, _, _ = ctx.forward_grad(circ, params, dq.Observables(obs), batch, dt, data=data, want_grad=False,
                                  state_out=st)
    torch.cuda.synchronize()
    names = set(ctx.trace())
    ctx.set_tracing(False)
    ctx.check()
    return st, e, names


CASES = [
    # n, batch, layers, dtype, with parity-diagonal gates (RZZ), encoded data
    (15, 3, 3, torch.complex64, False, True),
    (18, 2, 4, torch.complex64, True, True),
    (20, 1, 12, torch.complex64, False, False),     # more passes than one launch holds: chunked
    (20, 2, 3, torch.complex64, True, True),
    (17, 1, 4, torch.complex128, True, False),
    (19, 2, 3, torch.complex128, False, True),
]


@pytest.mark.parametrize("n,batch,layers,dt,pd,enc", CASES)
def test_multipass_equals_per_pass_launches_and_oracle(ctx, n, batch, layers, dt, pd, enc):
    rng = np.random.default_rng(700 + n + layers)
    gates = (W.encode_layer(n) if enc else []) + W.hea_layers(n, layers)
    if pd:
        gates += [W.Gate("rzz", (q, (q + 5) % n), angle=0.3 + 0.1 * q) for q in range(0, n, 2)]
        gates += W.hea_layers(n, 1, first_param=2 * n * layers)
    npar = 2 * n * (layers + (1 if pd else 0))
    params = rng.uniform(0, 2 * math.pi, size=npar)
    data = rng.uniform(-math.pi, math.pi, size=(batch, n)) if enc else None
    circ = dq.Circuit(n, gates, nparams=npar, nfeatures=n if enc else 0)
    obs = [W.obs_sum_z(n), [W.pauli_term(0.7, {0: "Z", n - 1: "Z"})]]
    st1, e1, names1 = run(ctx, circ, dev(params), dev(data), batch, dt, n, obs, True)
    st0, e0, names0 = run(ctx, circ, dev(params), dev(data), batch, dt, n, obs, False)
    assert "k_tile_multi" in names1 and "k_tile_fwd" not in names1, names1
    assert "k_tile_fwd" in names0 and "k_tile_multi" not in names0, names0
    assert torch.equal(st1, st0), "multi-pass and per-pass states differ"
    assert torch.equal(e1, e0), "multi-pass and per-pass expectations differ"
    ref = oracle.run(n, gates, params, data, batch=batch)
    assert_amps(np_state(st1), ref, dt, "multi-pass state")
    assert_rel(e1.cpu().numpy(), oracle.expect(n, ref, obs), dt, "multi-pass expectations",
               zero_scale=obs_scale(obs))


def test_multipass_only_for_l2_resident_states(ctx):
    """A 26-qubit complex64 state (512 MiB) keeps one launch per pass."""
    n = 26
    gates = W.hea_layers(n, 1)
    circ = dq.Circuit(n, gates, nparams=2 * n)
    params = dev(np.linspace(0.1, 2.0, 2 * n))
    st, e, names = run(ctx, circ, params, None, 1, torch.complex64, n, [W.obs_z(0)], True)
    assert "k_tile_fwd" in names and "k_tile_multi" not in names, names
    del st
    torch.cuda.empty_cache()


def test_multipass_under_graph_replay(ctx):
    """The captured launch (barrier reset + persistent kernel) replays with
    the values written in place between calls."""
    n, batch = 20, 1
    wl = W.config_c2()
    circ = dq.Circuit(n, wl.gates, nparams=wl.nparams)
    obs = dq.Observables(wl.observables)
    ctx.set_option(dq.OPT_MULTIPASS, 1)
    params = dev(wl.params)
    st = torch.empty((batch, 1 << n), dtype=torch.complex64, device="cuda")
    e = torch.empty((batch, 1), dtype=torch.float64, device="cuda")
    rng = np.random.default_rng(3)
    ctx.set_graphs(True)
    try:
        for call in range(4):
            p = rng.uniform(0, 2 * math.pi, size=wl.nparams)
            params.copy_(dev(p))
            ctx.forward_grad(circ, params, obs, batch, torch.complex64, want_grad=False, state_out=st, expect_out=e)
            torch.cuda.synchronize()
            ctx.check()
            ref = oracle.run(n, wl.gates, p)
            assert_amps(np_state(st), ref, torch.complex64, f"call {call} state")
            assert_rel(e.cpu().numpy(), oracle.expect(n, ref, wl.observables), torch.complex64,
                       f"call {call} <sum Z>", zero_scale=obs_scale(wl.observables))
    finally:
        ctx.set_graphs(False)
