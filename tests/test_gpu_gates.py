"""GPU parity of the wider gate set -- the phase shift P, U3, the two-qubit
rotations RXX / RYY / RZZ and the Toffoli gate CCX -- against the FP64 oracle,
which implements each of them from its own definition (the library lowers the
composite kinds to products of its kernel-level gates).  Covers the paper's
QCNN and data re-uploading QNN examples with encoded inputs and their
gradients, a Trotterised TFIM evolution on the tiled path, the uneven-batch
kernel, and both dtypes on the plain and fused paths."""
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

PATHS = {"plain": dq.PATH_PLAIN, "fused": dq.PATH_FUSED}
DTYPES = {"c64": torch.complex64, "c128": torch.complex128}
WIDE = ("h", "p", "u3", "rxx", "ryy", "rzz", "ccx", "cnot", "ry", "rz", "cry")


@pytest.fixture(scope="module")
def ctx():
    c = dq.Context(0)
    yield c
    c.close()


def wide_gates(n, depth, rng, nfeat=0):
    """Random gates weighted towards the wider kinds; U3 takes three slots."""
    gates, npar = [], 0
    while len(gates) < depth:
        k = WIDE[rng.integers(len(WIDE))]
        nw = 3 if k in W.THREE_QUBIT else (2 if k in W.TWO_QUBIT else 1)
        if n < nw:
            continue
        wires = tuple(int(w) for w in rng.choice(n, size=nw, replace=False))
        span = W.ANGLE_SPAN.get(k, 1)
        if k in W.PARAMETRIC:
            u = rng.random()
            if nfeat >= span and u < 0.3:
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
@pytest.mark.parametrize("n,batch", [(3, 4), (6, 9), (11, 3), (14, 2), (17, 2), (20, 1)])
def test_wide_gate_states(ctx, path, dtype, n, batch):
    ctx.set_path(PATHS[path])
    dt = DTYPES[dtype]
    rng = np.random.default_rng(5000 + 13 * n + batch)
    gates, npar = wide_gates(n, 6 * n + 12, rng, nfeat=4)
    params = rng.uniform(-4, 4, size=npar)
    data = rng.uniform(-3, 3, size=(batch, 4))
    circ = dq.Circuit(n, gates, nparams=npar, nfeatures=4)
    st = torch.empty((batch, 1 << n), dtype=dt, device="cuda")
    ctx.state_init(st, n)
    ctx.apply_circuit(circ, dev(params), st, data=dev(data))
    assert_amps(np_state(st), oracle.run(n, gates, params, data, batch=batch), dt)


@pytest.mark.parametrize("path", sorted(PATHS))
@pytest.mark.parametrize("dtype", sorted(DTYPES))
@pytest.mark.parametrize("ppr", [False, True])
@pytest.mark.parametrize("n,batch", [(2, 3), (5, 17), (12, 4), (16, 2), (18, 2)])
def test_wide_gate_gradients(ctx, path, dtype, ppr, n, batch):
    ctx.set_path(PATHS[path])
    dt = DTYPES[dtype]
    rng = np.random.default_rng(6000 + 11 * n + batch + ppr)
    gates, npar = wide_gates(n, 5 * n + 10, rng, nfeat=3)
    params = rng.uniform(-4, 4, size=(batch, npar) if ppr else npar)
    data = rng.uniform(-3, 3, size=(batch, 3))
    obs = [W.obs_tfim_open(n, 0.5) if n > 1 else W.obs_z(0), [(0.8, 1, (1 << n) - 1), (-0.3, 0, 1)]]
    w = rng.normal(size=(batch, 2))
    circ = dq.Circuit(n, gates, nparams=npar, nfeatures=3)
    e, gp, gd, _ = ctx.forward_grad(circ, dev(params), dq.Observables(obs), batch, dt, data=dev(data),
                                    row_weights=dev(w), params_per_row=ppr)
    e_ref, gp_ref, gd_ref = oracle.adjoint(n, gates, obs, params, data, batch=batch, params_per_row=ppr,
                                           row_weights=w)
    gscale = float(np.abs(w).max(axis=1).sum()) * obs_scale(obs)
    assert_rel(e.cpu().numpy(), e_ref, dt, "expectations", zero_scale=obs_scale(obs))
    assert_rel(gp.cpu().numpy(), gp_ref, dt, "grad params", zero_scale=gscale)
    assert_rel(gd.cpu().numpy(), gd_ref, dt, "grad data", zero_scale=gscale)


@pytest.mark.parametrize("path", sorted(PATHS))
def test_qcnn_batch(ctx, path):
    """The paper's 12-qubit QCNN on 1024 rows of 21 encoded features in
    [-pi, pi] (the tanh-scaled pooled image features of the example, here
    synthetic), <Z_0> per row and gradients of the batch sum with respect to
    the 33 parameters and to every feature."""
    ctx.set_path(PATHS[path])
    gates, npar, nfeat = W.qcnn_gates(12)
    batch = 1024
    params = W.uniform_array(71, npar, 0.0, 2 * np.pi)
    data = W.uniform_array(72, batch * nfeat, -np.pi, np.pi).reshape(batch, nfeat)
    obs = [W.obs_z(0)]
    circ = dq.Circuit(12, gates, nparams=npar, nfeatures=nfeat)
    e, gp, gd, _ = ctx.forward_grad(circ, dev(params), dq.Observables(obs), batch, torch.complex64,
                                    data=dev(data))
    rows = np.arange(0, batch, 8)
    e_ref, _, gd_ref = oracle.adjoint(12, gates, obs, params, data[rows], batch=rows.size)
    _, gp_ref, _ = oracle.adjoint(12, gates, obs, params, data, batch=batch)
    assert_rel(e.cpu().numpy()[rows], e_ref, torch.complex64, "expectations", zero_scale=1.0)
    assert_rel(gp.cpu().numpy(), gp_ref, torch.complex64, "grad params", zero_scale=float(batch))
    assert_rel(gd.cpu().numpy()[rows], gd_ref, torch.complex64, "grad data", zero_scale=1.0)


@pytest.mark.parametrize("residual", [False, True])
@pytest.mark.parametrize("dtype", sorted(DTYPES))
def test_qnn_u3_reuploading(ctx, residual, dtype):
    """The data re-uploading QNNs (U3 layers around an encoded RY, and the
    residual two-qubit version with a controlled encoded RY) through the
    autograd function: expectations, d/dparams and d/dx."""
    ctx.set_path(dq.PATH_AUTO)
    dt = DTYPES[dtype]
    n, gates, npar, nfeat, obs = W.qnn_u3_gates(residual)
    batch = 500
    params = W.uniform_array(81, npar, -np.pi, np.pi)
    data = W.uniform_array(82, batch * nfeat, -1.0, 1.0).reshape(batch, nfeat)
    circ = dq.Circuit(n, gates, nparams=npar, nfeatures=nfeat)
    p = torch.tensor(params, device="cuda", requires_grad=True)
    x = torch.tensor(data, device="cuda", requires_grad=True)
    e = dq.expectation(circ, p, dq.Observables(obs), data=x, dtype=dt, context=ctx)
    e.sum().backward()
    e_ref, gp_ref, gd_ref = oracle.adjoint(n, gates, obs, params, data, batch=batch)
    assert_rel(e.detach().cpu().numpy(), e_ref, dt, "expectations", zero_scale=1.0)
    assert_rel(p.grad.cpu().numpy(), gp_ref, dt, "grad params", zero_scale=float(batch * len(obs)))
    assert_rel(x.grad.cpu().numpy(), gd_ref, dt, "grad data", zero_scale=float(len(obs)))


@pytest.mark.parametrize("path", sorted(PATHS))
@pytest.mark.parametrize("n", [12, 19])
def test_tfim_trotter_evolution(ctx, path, n):
    """Second-order Trotter steps of the periodic TFIM (RX and RZZ with fixed
    angles), on the tiled path at 19 qubits: the state and <H>."""
    ctx.set_path(PATHS[path])
    steps = 6
    gates = W.tfim_trotter_gates(n, steps)
    circ = dq.Circuit(n, gates, nparams=0)
    H = [[W.pauli_term(-1.0, {i: "Z", (i + 1) % n: "Z"}) for i in range(n)]
         + [W.pauli_term(-1.2, {i: "X"}) for i in range(n)]]
    st = torch.empty((1, 1 << n), dtype=torch.complex64, device="cuda")
    ctx.state_init(st, n)
    ctx.apply_circuit(circ, None, st)
    ref = oracle.run(n, gates)
    assert_amps(np_state(st), ref, torch.complex64)
    e = ctx.expect(n, dq.Observables(H), st)
    assert_rel(e.cpu().numpy(), oracle.expect(n, ref, H), torch.complex64, "energy", zero_scale=obs_scale(H))


@pytest.mark.parametrize("path", sorted(PATHS))
def test_uneven_batch_wide_gate_set(ctx, path):
    """Uneven batch (one persistent launch) of random circuits over every
    kind, per-circuit parameters (U3 owns three), against the oracle."""
    ctx.set_path(PATHS[path])
    circs = [W.random_circuit(9000 + c, nmin=3, nmax=14, kinds=W.GATE_KINDS) for c in range(96)]
    obs = [W.obs_zz01_x0()]
    dcs = [dq.Circuit(n, g, nparams=len(a)) for n, g, a in circs]
    params = np.concatenate([a for _, _, a in circs])
    offs = np.cumsum([0] + [len(a) for _, _, a in circs])
    e, gp = ctx.batch_forward_grad(dcs, dev(params), dq.Observables(obs), torch.complex64)
    e = e.cpu().numpy()
    gp = gp.cpu().numpy()
    e_ref = []
    for i, (n, g, a) in enumerate(circs):
        er, gr, _ = oracle.adjoint(n, g, obs, a)
        e_ref.append(er[0, 0])
        assert_rel(gp[offs[i]:offs[i + 1]], gr, torch.complex64, f"circuit {i} gradient", zero_scale=obs_scale(obs))
    assert_rel(e.reshape(-1), e_ref, torch.complex64, "expectations of all circuits", zero_scale=obs_scale(obs))


def test_trotter_full_size_paths_agree(ctx):
    """26 qubits (512 MiB complex64, beyond the oracle): the fused passes with
    parity-diagonal RZZ and the per-gate path agree on sampled amplitudes and
    on <H>, and the state stays normalised."""
    n, steps = 26, 3
    gates = W.tfim_trotter_gates(n, steps)
    circ = dq.Circuit(n, gates, nparams=0)
    H = dq.Observables([[W.pauli_term(-1.0, {i: "Z", (i + 1) % n: "Z"}) for i in range(n)]
                        + [W.pauli_term(-1.2, {i: "X"}) for i in range(n)]])
    out = {}
    for name, path in (("fused", dq.PATH_FUSED), ("plain", dq.PATH_PLAIN)):
        ctx.set_path(path)
        st = torch.empty((1, 1 << n), dtype=torch.complex64, device="cuda")
        ctx.state_init(st, n)
        ctx.apply_circuit(circ, None, st)
        out[name] = (st, ctx.expect(n, H, st).cpu().numpy())
    ctx.set_path(dq.PATH_AUTO)
    a, b = out["fused"][0], out["plain"][0]
    idx = torch.randint(0, 1 << n, (4096,), generator=torch.Generator().manual_seed(26)).cuda()
    assert float((a[0, idx] - b[0, idx]).abs().max()) <= 1e-5
    assert abs(float(torch.linalg.vector_norm(a.to(torch.complex128))) - 1.0) <= 1e-4
    assert abs(out["fused"][1][0, 0] - out["plain"][1][0, 0]) <= 1e-4 * 2 * n * 1.2
    del out, a, b
    torch.cuda.empty_cache()
