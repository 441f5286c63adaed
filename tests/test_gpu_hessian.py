"""GPU parity of the Hessian (dq_hessian: two- and four-term shift rules on
batched adjoint gradients) against the oracle's product-rule Hessian, which
differentiates the circuit gate by gate and shares nothing with the shift
rules: random circuits over every parametric kind with a parameter used by
several gates, encoded data rows and row weights, both dtypes, both paths,
the on-chip and tiled sizes, chunked batches, and the paper's data
re-uploading QNN."""
import numpy as np
import pytest
import torch

import oracle
import workloads as W
from tests.gpu_helpers import assert_rel, dev, obs_scale

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("CUDA GPU required", allow_module_level=True)

import paper_2512_18995_gb300 as dq  # noqa: E402
from paper_2512_18995_gb300 import build as dqbuild  # noqa: E402

dqbuild.build()

PATHS = {"plain": dq.PATH_PLAIN, "fused": dq.PATH_FUSED}
DTYPES = {"c64": torch.complex64, "c128": torch.complex128}
KINDS = ("h", "rx", "ry", "rz", "cnot", "cp", "p", "u3", "rxx", "ryy", "rzz", "crx", "cry", "crz", "ccx", "cz")


@pytest.fixture(scope="module")
def ctx():
    c = dq.Context(0)
    yield c
    c.close()


def hess_gates(n, depth, rng, nfeat):
    gates, npar = [], 0
    while len(gates) < depth:
        k = KINDS[rng.integers(len(KINDS))]
        nw = 3 if k in W.THREE_QUBIT else (2 if k in W.TWO_QUBIT else 1)
        if n < nw:
            continue
        wires = tuple(int(w) for w in rng.choice(n, size=nw, replace=False))
        span = W.ANGLE_SPAN.get(k, 1)
        if k in W.PARAMETRIC:
            u = rng.random()
            if nfeat >= span and u < 0.2:
                gates.append(W.Gate(k, wires, data=int(rng.integers(nfeat - span + 1))))
            elif span == 1 and u < 0.3:
                gates.append(W.Gate(k, wires, angle=float(rng.uniform(-3, 3))))
            elif span == 1 and npar > 0 and u < 0.4:
                gates.append(W.Gate(k, wires, param=int(rng.integers(npar))))   # a shared parameter
            else:
                gates.append(W.Gate(k, wires, param=npar))
                npar += span
        else:
            gates.append(W.Gate(k, wires))
    return gates, max(npar, 1)


def hscale(obs, w):
    return obs_scale(obs) * (float(np.abs(w).sum()) if w is not None else 1.0)


@pytest.mark.parametrize("path", sorted(PATHS))
@pytest.mark.parametrize("dtype", sorted(DTYPES))
@pytest.mark.parametrize("n,batch,depth", [(2, 1, 12), (3, 3, 20), (5, 2, 28), (12, 2, 30), (16, 1, 26)])
def test_hessian_matches_product_rule(ctx, path, dtype, n, batch, depth):
    ctx.set_path(PATHS[path])
    dt = DTYPES[dtype]
    rng = np.random.default_rng(700 + 17 * n + batch)
    gates, npar = hess_gates(n, depth, rng, nfeat=3)
    params = rng.uniform(-3, 3, size=npar)
    data = rng.uniform(-3, 3, size=(batch, 3))
    obs = [W.obs_tfim_open(n, 0.5) if n > 1 else W.obs_z(0), [(0.6, 1, (1 << n) - 1)]]
    w = rng.normal(size=(batch, 2))
    circ = dq.Circuit(n, gates, nparams=npar, nfeatures=3)
    H, g = ctx.hessian(circ, dev(params), dq.Observables(obs), data=dev(data), row_weights=dev(w), dtype=dt)
    Href = oracle.hessian(n, gates, obs, params, data, batch=batch, row_weights=w)
    _, gref, _ = oracle.adjoint(n, gates, obs, params, data, batch=batch, row_weights=w)
    assert_rel(H.cpu().numpy(), Href, dt, "hessian", zero_scale=hscale(obs, w))
    assert_rel(g.cpu().numpy(), gref, dt, "gradient", zero_scale=hscale(obs, w))


def test_hessian_in_chunks(ctx):
    """A memory bound that admits one occurrence per batched call gives the
    same Hessian as one call."""
    ctx.set_path(dq.PATH_FUSED)
    n, batch = 14, 2
    rng = np.random.default_rng(5)
    gates, npar = hess_gates(n, 30, rng, nfeat=2)
    params = rng.uniform(-3, 3, size=npar)
    data = rng.uniform(-3, 3, size=(batch, 2))
    obs = [W.obs_tfim_open(n, 0.5)]
    circ = dq.Circuit(n, gates, nparams=npar, nfeatures=2)
    H1, _ = ctx.hessian(circ, dev(params), dq.Observables(obs), data=dev(data), dtype=torch.complex128)
    H2, _ = ctx.hessian(circ, dev(params), dq.Observables(obs), data=dev(data), dtype=torch.complex128,
                        max_bytes=1 << 16)
    Href = oracle.hessian(n, gates, obs, params, data, batch=batch)
    assert_rel(H1.cpu().numpy(), Href, torch.complex128, "hessian", zero_scale=obs_scale(obs) * batch)
    assert_rel(H2.cpu().numpy(), Href, torch.complex128, "hessian (chunked)", zero_scale=obs_scale(obs) * batch)


@pytest.mark.parametrize("dtype", sorted(DTYPES))
def test_hessian_qnn_u3(ctx, dtype):
    """The residual data re-uploading QNN (U3 layers, controlled encoded RY)
    over 200 data rows: Hessian of the summed expectations."""
    ctx.set_path(dq.PATH_AUTO)
    dt = DTYPES[dtype]
    n, gates, npar, nfeat, obs = W.qnn_u3_gates(True)
    batch = 200
    params = W.uniform_array(91, npar, -np.pi, np.pi)
    data = W.uniform_array(92, batch * nfeat, -1.0, 1.0).reshape(batch, nfeat)
    circ = dq.Circuit(n, gates, nparams=npar, nfeatures=nfeat)
    H, _ = ctx.hessian(circ, dev(params), dq.Observables(obs), data=dev(data), dtype=dt, want_grad=False)
    Href = oracle.hessian(n, gates, obs, params, data, batch=batch)
    assert_rel(H.cpu().numpy(), Href, dt, "hessian", zero_scale=float(batch * len(obs)))


def test_hessian_without_trainable_occurrences(ctx):
    """A circuit whose parameters are unused gives a zero Hessian."""
    circ = dq.Circuit(3, [W.Gate("h", (0,)), W.Gate("rx", (1,), angle=0.3)], nparams=2)
    H, g = ctx.hessian(circ, dev(np.array([0.1, 0.2])), dq.Observables([W.obs_z(1)]))
    assert torch.count_nonzero(H) == 0 and torch.count_nonzero(g) == 0


def test_hessian_full_size_properties(ctx):
    """20 qubits (beyond the oracle's product rule): the Hessian is symmetric
    and each row matches central differences of the library's own adjoint
    gradient (complex128; the gradient itself is checked against the oracle
    elsewhere)."""
    ctx.set_path(dq.PATH_AUTO)
    n = 20
    gates = W.hea_layers(n, 1)[:2 * n] + [W.Gate("rzz", (0, 7), param=2 * n), W.Gate("cry", (3, 11), param=2 * n + 1),
                                         W.Gate("u3", (5,), param=2 * n + 2)] + W.hea_layers(n, 1)[2 * n:]
    npar = 2 * n + 5
    rng = np.random.default_rng(20)
    params = rng.uniform(-3, 3, size=npar)
    obs = [W.obs_tfim_open(n, 0.5)]
    circ = dq.Circuit(n, gates, nparams=npar)
    dobs = dq.Observables(obs)
    H, g = ctx.hessian(circ, dev(params), dobs, dtype=torch.complex128)
    H = H.cpu().numpy()
    scale = obs_scale(obs)
    assert np.max(np.abs(H - H.T)) <= 1e-10 * scale
    h = 1e-5
    for j in (0, n, 2 * n, 2 * n + 1, 2 * n + 3):
        e = np.zeros(npar)
        e[j] = h
        _, gp, _, _ = ctx.forward_grad(circ, dev(params + e), dobs, 1, torch.complex128)
        _, gm, _, _ = ctx.forward_grad(circ, dev(params - e), dobs, 1, torch.complex128)
        fd = (gp - gm).cpu().numpy() / (2 * h)
        assert np.max(np.abs(H[j] - fd)) <= 1e-6 * scale, j
