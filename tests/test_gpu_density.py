"""GPU parity of mixed-state evolution (dq_density_forward) against the
oracle's density-matrix simulator, which applies U rho U^dagger column by
column and row by row and channels as Kraus sums -- nothing like the
library's vectorised 2n-qubit lowering: random circuits over every gate kind
with bit-flip, phase-flip, depolarizing and amplitude-damping channels,
encoded data rows, both dtypes, both paths (on-chip rows for small n, tiles
for the 18- and 22-qubit vectors of 9 and 11 qubits)."""
import numpy as np
import pytest
import torch

import oracle
import workloads as W
from tests.gpu_helpers import assert_amps, assert_rel, dev, obs_scale

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("CUDA GPU required", allow_module_level=True)

import paper_2512_18995_gb300 as dq  # noqa: E402
from paper_2512_18995_gb300 import build as dqbuild  # noqa: E402

dqbuild.build()

PATHS = {"plain": dq.PATH_PLAIN, "fused": dq.PATH_FUSED}
DTYPES = {"c64": torch.complex64, "c128": torch.complex128}
KINDS = W.GATE_KINDS + W.NOISE_KINDS


@pytest.fixture(scope="module")
def ctx():
    c = dq.Context(0)
    yield c
    c.close()


def noisy_gates(n, depth, rng, nfeat):
    gates, npar = [], 0
    while len(gates) < depth:
        k = KINDS[rng.integers(len(KINDS))]
        nw = 3 if k in W.THREE_QUBIT else (2 if k in W.TWO_QUBIT else 1)
        if n < nw:
            continue
        wires = tuple(int(w) for w in rng.choice(n, size=nw, replace=False))
        if k in W.NOISE_KINDS:
            pmax = 0.75 if k == "depolarizing" else 1.0
            gates.append(W.Gate(k, wires, angle=float(rng.uniform(0, pmax))))
            continue
        span = W.ANGLE_SPAN.get(k, 1)
        if k in W.PARAMETRIC:
            u = rng.random()
            if nfeat >= span and u < 0.25:
                gates.append(W.Gate(k, wires, data=int(rng.integers(nfeat - span + 1))))
            elif span == 1 and u < 0.4:
                gates.append(W.Gate(k, wires, angle=float(rng.uniform(-4, 4))))
            else:
                gates.append(W.Gate(k, wires, param=npar))
                npar += span
        else:
            gates.append(W.Gate(k, wires))
    return gates, max(npar, 1)


@pytest.mark.parametrize("path", sorted(PATHS))
@pytest.mark.parametrize("dtype", sorted(DTYPES))
@pytest.mark.parametrize("n,batch,depth", [(1, 2, 10), (2, 3, 20), (3, 2, 30), (5, 3, 40), (7, 2, 50), (9, 1, 50),
                                           (11, 1, 40)])
def test_density_matches_oracle(ctx, path, dtype, n, batch, depth):
    ctx.set_path(PATHS[path])
    dt = DTYPES[dtype]
    rng = np.random.default_rng(1300 + 7 * n + batch)
    gates, npar = noisy_gates(n, depth, rng, nfeat=3)
    params = rng.uniform(-4, 4, size=npar)
    data = rng.uniform(-3, 3, size=(batch, 3))
    obs = [W.obs_tfim_open(n, 0.5) if n > 1 else W.obs_z(0), [(0.6, (1 << n) - 1, 1), (-0.3, 0, (1 << n) - 1)]]
    circ = dq.Circuit(n, gates, nparams=npar, nfeatures=3)
    e, rho = ctx.density_forward(circ, dev(params), dq.Observables(obs), batch, dt, data=dev(data), want_rho=True)
    e_ref, rho_ref = oracle.density(n, gates, obs, params, data, batch=batch)
    assert_amps(rho.cpu().numpy().astype(np.complex128), rho_ref, dt, "rho")
    assert_rel(e.cpu().numpy(), e_ref, dt, "expectations", zero_scale=obs_scale(obs))


def test_noiseless_density_equals_outer_product(ctx):
    """Without channels the vectorised evolution is |psi><psi| of the
    state-vector path (both on the GPU), at 8 qubits."""
    ctx.set_path(dq.PATH_AUTO)
    n = 8
    rng = np.random.default_rng(4)
    gates, npar = noisy_gates(n, 60, rng, nfeat=0)
    gates = [g for g in gates if g.kind not in W.NOISE_KINDS]
    params = rng.uniform(-4, 4, size=npar)
    circ = dq.Circuit(n, gates, nparams=npar)
    _, rho = ctx.density_forward(circ, dev(params), None, 1, torch.complex128, want_rho=True)
    st = torch.empty((1, 1 << n), dtype=torch.complex128, device="cuda")
    ctx.state_init(st, n)
    ctx.apply_circuit(circ, dev(params), st)
    psi = st[0]
    torch.testing.assert_close(rho[0], torch.outer(psi, psi.conj()), atol=1e-12, rtol=0)


def test_density_rejects_bad_arguments(ctx):
    st = torch.zeros((1, 4), dtype=torch.complex64, device="cuda")
    noisy = dq.Circuit(2, [W.Gate("bitflip", (0,), angle=0.1)])
    with pytest.raises(dq.DQError, match="density"):
        ctx.apply_circuit(noisy, None, st)
    with pytest.raises(dq.DQError, match="probability"):
        ctx.density_forward(dq.Circuit(2, [W.Gate("depolarizing", (0,), angle=0.8)]), None, None)
    with pytest.raises(dq.DQError, match="fixed probability"):
        ctx.density_forward(dq.Circuit(2, [W.Gate("ampdamp", (0,), param=0)], nparams=1),
                            dev(np.array([0.1])), None)
    with pytest.raises(dq.DQError, match="17"):
        ctx.density_forward(dq.Circuit(18, [W.Gate("h", (0,))]), None, None)


def fd_density_grad(n, gates, obs, params, data, w, h=1e-5):
    """Central differences of the oracle's weighted expectation sum."""
    def loss(pv):
        e, _ = oracle.density(n, gates, obs, pv, data, batch=data.shape[0])
        return float(np.sum(w * e))
    g = np.zeros(params.size)
    for i in range(params.size):
        d = np.zeros(params.size)
        d[i] = h
        g[i] = (loss(params + d) - loss(params - d)) / (2 * h)
    return g


@pytest.mark.parametrize("dtype", sorted(DTYPES))
@pytest.mark.parametrize("n,batch,depth", [(1, 2, 12), (3, 2, 30), (4, 3, 36), (6, 1, 40)])
def test_density_gradients_match_finite_differences(ctx, dtype, n, batch, depth):
    """Shift-rule gradients of noisy circuits (every parametric kind,
    including the four-term controlled rotations, U3 and shared parameters)
    against central differences of the oracle."""
    ctx.set_path(dq.PATH_AUTO)
    dt = DTYPES[dtype]
    rng = np.random.default_rng(2300 + 5 * n + batch)
    gates, npar = noisy_gates(n, depth, rng, nfeat=3)
    if npar > 1:
        gates.append(W.Gate("rx", (0,), param=0))   # parameter 0 used twice
    params = rng.uniform(-3, 3, size=npar)
    data = rng.uniform(-3, 3, size=(batch, 3))
    obs = [W.obs_tfim_open(n, 0.5) if n > 1 else W.obs_z(0), [(0.6, (1 << n) - 1, 1)]]
    w = rng.normal(size=(batch, 2))
    circ = dq.Circuit(n, gates, nparams=npar, nfeatures=3)
    e, g = ctx.density_grad(circ, dev(params), dq.Observables(obs), data=dev(data), row_weights=dev(w), dtype=dt)
    e_ref, _ = oracle.density(n, gates, obs, params, data, batch=batch)
    g_ref = fd_density_grad(n, gates, obs, params, data, w)
    assert_rel(e.cpu().numpy(), e_ref, dt, "expectations", zero_scale=obs_scale(obs))
    scale = float(np.abs(w).max(axis=1).sum()) * obs_scale(obs)
    err = np.max(np.abs(g.cpu().numpy() - g_ref)) / scale
    assert err <= (1e-4 if dt == torch.complex64 else 1e-8), f"gradient error {err:.3e} (relative to {scale:.3f})"


def test_density_gradients_in_chunks(ctx):
    """A memory bound of one occurrence per batched call gives the same gradient."""
    n = 5
    rng = np.random.default_rng(9)
    gates, npar = noisy_gates(n, 40, rng, nfeat=0)
    params = rng.uniform(-3, 3, size=npar)
    obs = [W.obs_tfim_open(n, 0.5)]
    circ = dq.Circuit(n, gates, nparams=npar)
    _, g1 = ctx.density_grad(circ, dev(params), dq.Observables(obs), dtype=torch.complex128)
    _, g2 = ctx.density_grad(circ, dev(params), dq.Observables(obs), dtype=torch.complex128, max_bytes=1 << 12)
    torch.testing.assert_close(g1, g2, atol=1e-12, rtol=0)


def test_density_autograd(ctx):
    """density_expectation through torch autograd: d(sum w * E)/dparams equals
    dq_density_grad with the same weights."""
    n, batch = 4, 3
    rng = np.random.default_rng(12)
    gates, npar = noisy_gates(n, 30, rng, nfeat=2)
    circ = dq.Circuit(n, gates, nparams=npar, nfeatures=2)
    obs = dq.Observables([W.obs_tfim_open(n, 0.5)])
    p = torch.tensor(rng.uniform(-3, 3, size=npar), device="cuda", requires_grad=True)
    x = dev(rng.uniform(-3, 3, size=(batch, 2)))
    w = dev(rng.normal(size=(batch, 1)))
    e = dq.density_expectation(circ, p, obs, data=x, dtype=torch.complex128, context=ctx)
    (e * w).sum().backward()
    _, g = ctx.density_grad(circ, p.detach(), obs, data=x, row_weights=w, dtype=torch.complex128)
    torch.testing.assert_close(p.grad, g, atol=1e-12, rtol=0)
