"""GPU parity: the CUDA library (through its C ABI) against the FP64 oracle,
element by element, on seeded inputs -- random circuits over every gate kind
and wire position, ragged batches, both the plain per-gate path and the fused
paths, and the five workload configurations at full size (sampled outputs or
exact factorised references where the oracle cannot run the whole thing)."""
import math

import numpy as np
import pytest
import torch

import oracle
import workloads as W
from tests.gpu_helpers import (AMP_TOL, REL_TOL, assert_amps, assert_rel, dev, factorised_amplitude,
                               factorised_c5, factorised_reference, np_state, obs_scale)

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("CUDA GPU required", allow_module_level=True)

import paper_2512_18995_gb300 as dq  # noqa: E402
from paper_2512_18995_gb300 import build as dqbuild  # noqa: E402

dqbuild.build()

PATHS = {"plain": dq.PATH_PLAIN, "fused": dq.PATH_FUSED}
DTYPES = {"c64": torch.complex64, "c128": torch.complex128}


@pytest.fixture(scope="module")
def ctx():
    c = dq.Context(0)
    yield c
    c.close()


def random_gates(n, depth, rng, nfeat=0, kinds=None):
    """Random gates over every kind (U3 reads three consecutive parameter or
    feature slots and never takes a fixed angle)."""
    kinds = kinds or W.GATE_KINDS
    gates, npar = [], 0
    while len(gates) < depth:
        k = kinds[rng.integers(len(kinds))]
        if k in W.TWO_QUBIT or k in W.THREE_QUBIT:
            nw = 3 if k in W.THREE_QUBIT else 2
            if n < nw:
                continue
            wires = tuple(int(w) for w in rng.choice(n, size=nw, replace=False))
        else:
            wires = (int(rng.integers(n)),)
        span = W.ANGLE_SPAN.get(k, 1)
        if k in W.PARAMETRIC:
            u = rng.random()
            if nfeat >= span and u < 0.25:
                gates.append(W.Gate(k, wires, data=int(rng.integers(nfeat - span + 1))))
            elif span == 1 and u < 0.35:
                gates.append(W.Gate(k, wires, angle=float(rng.uniform(-4, 4))))
            else:
                gates.append(W.Gate(k, wires, param=npar))
                npar += span
        else:
            gates.append(W.Gate(k, wires))
    return gates, max(npar, 1)


def edge_gates(n):
    """Every kind on the extreme wires (bit 0 and bit n-1) and in both
    control/target orders."""
    g = []
    hi, lo = 0, n - 1          # wire 0 = top bit, wire n-1 = bit 0
    for q in sorted({hi, lo, n // 2}):
        for k in ("h", "x", "y", "z", "s"):
            g.append(W.Gate(k, (q,)))
        for k in ("rx", "ry", "rz"):
            g.append(W.Gate(k, (q,), angle=0.37 + q))
    if n >= 2:
        pairs = {(hi, lo), (lo, hi), (0, 1), (1, 0), (n - 2, n - 1), (n - 1, n - 2)}
        for a, b in sorted(pairs):
            for k in ("cnot", "cz", "swap"):
                g.append(W.Gate(k, (a, b)))
            for k in ("cp", "crx", "cry", "crz", "rxx", "ryy", "rzz"):
                g.append(W.Gate(k, (a, b), angle=1.1 + 0.1 * a))
    for q in sorted({hi, lo, n // 2}):
        g.append(W.Gate("p", (q,), angle=0.6 - q))
    if n >= 3:
        mid = n // 2 if n // 2 not in (hi, lo) else 1
        for c0, c1, t in ((hi, lo, mid), (lo, mid, hi), (mid, hi, lo), (n - 3, n - 2, n - 1), (2, 1, 0)):
            g.append(W.Gate("h", (t,)))
            g.append(W.Gate("ccx", (c0, c1, t)))
    return g


# ---------------------------------------------------------------------------
# random circuits: states
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("path", sorted(PATHS))
@pytest.mark.parametrize("dtype", sorted(DTYPES))
@pytest.mark.parametrize("n,batch", [(1, 1), (2, 3), (3, 5), (5, 33), (8, 7), (11, 3), (13, 2), (14, 3), (16, 2),
                                     (18, 1), (21, 2)])
def test_random_circuit_states(ctx, path, dtype, n, batch):
    ctx.set_path(PATHS[path])
    dt = DTYPES[dtype]
    rng = np.random.default_rng(1000 + 37 * n + batch)
    gates, npar = random_gates(n, 8 * n + 10, rng, nfeat=3)
    gates = edge_gates(n) + gates
    params = rng.uniform(-4, 4, size=npar)
    data = rng.uniform(-3, 3, size=(batch, 3))
    circ = dq.Circuit(n, gates, nparams=npar, nfeatures=3)
    st = torch.empty((batch, 1 << n), dtype=dt, device="cuda")
    ctx.state_init(st, n)
    ctx.apply_circuit(circ, dev(params), st, data=dev(data))
    ref = oracle.run(n, gates, params, data, batch=batch)
    assert_amps(np_state(st), ref, dt)


@pytest.mark.parametrize("dtype", sorted(DTYPES))
@pytest.mark.parametrize("n", [15, 19])
def test_tiled_path_after_autotune(ctx, dtype, n):
    """The fused tile path with the configuration the autotuner picks, on
    circuits with every kind, SWAPs, controls on low and high bits and long
    diagonal runs (a QFT block)."""
    ctx.set_path(dq.PATH_FUSED)
    dt = DTYPES[dtype]
    rng = np.random.default_rng(4242 + n)
    gates, npar = random_gates(n, 10 * n, rng)
    gates = edge_gates(n) + W.qft_gates(n) + gates
    params = rng.uniform(-4, 4, size=npar)
    circ = dq.Circuit(n, gates, nparams=npar)
    st = torch.empty((1, 1 << n), dtype=dt, device="cuda")
    ctx.plan_autotune(circ, st)
    ctx.state_init(st, n)
    ctx.apply_circuit(circ, dev(params), st)
    ctx.check()
    assert_amps(np_state(st), oracle.run(n, gates, params), dt)


@pytest.mark.parametrize("path", sorted(PATHS))
def test_apply_to_given_state_and_inverse(ctx, path):
    ctx.set_path(PATHS[path])
    n, batch = 9, 4
    rng = np.random.default_rng(5)
    gates, npar = random_gates(n, 80, rng)
    params = rng.uniform(-4, 4, size=npar)
    psi = rng.normal(size=(batch, 1 << n)) + 1j * rng.normal(size=(batch, 1 << n))
    psi /= np.linalg.norm(psi, axis=1, keepdims=True)
    st = torch.as_tensor(psi, dtype=torch.complex128, device="cuda").contiguous()
    ctx.apply_circuit(dq.Circuit(n, gates, nparams=npar), dev(params), st)
    ref = oracle.apply(n, gates, psi, params)
    assert_amps(np_state(st), ref, torch.complex128)


# ---------------------------------------------------------------------------
# expectations
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("path", sorted(PATHS))
@pytest.mark.parametrize("dtype", sorted(DTYPES))
@pytest.mark.parametrize("n,batch", [(1, 2), (3, 3), (7, 5), (12, 3), (15, 2)])
def test_expectations(ctx, path, dtype, n, batch):
    ctx.set_path(PATHS[path])
    dt = DTYPES[dtype]
    rng = np.random.default_rng(77 + n)
    N = 1 << n
    psi = rng.normal(size=(batch, N)) + 1j * rng.normal(size=(batch, N))
    psi /= np.linalg.norm(psi, axis=1, keepdims=True)
    obs = []
    for _ in range(3):
        obs.append([(float(rng.normal()), int(rng.integers(N)), int(rng.integers(N))) for _ in range(5)])
    obs.append(W.obs_tfim_open(n, 0.5) if n > 1 else W.obs_z(0))
    st = torch.as_tensor(psi, dtype=dt, device="cuda").contiguous()
    got = ctx.expect(n, dq.Observables(obs), st).cpu().numpy()
    ref = oracle.expect(n, np_state(st), obs)
    assert_rel(got, ref, dt, "expectations", zero_scale=obs_scale(obs))


# ---------------------------------------------------------------------------
# adjoint gradients
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("path", sorted(PATHS))
@pytest.mark.parametrize("dtype", sorted(DTYPES))
@pytest.mark.parametrize("ppr", [False, True])
@pytest.mark.parametrize("n,batch", [(1, 2), (4, 3), (9, 17), (12, 5), (15, 2), (18, 3)])
def test_adjoint_gradients(ctx, path, dtype, ppr, n, batch):
    ctx.set_path(PATHS[path])
    dt = DTYPES[dtype]
    rng = np.random.default_rng(300 + n + 7 * batch + ppr)
    gates, npar = random_gates(n, 6 * n + 12, rng, nfeat=2)
    params = rng.uniform(-4, 4, size=(batch, npar) if ppr else npar)
    data = rng.uniform(-3, 3, size=(batch, 2))
    obs = [W.obs_tfim_open(n, 0.5) if n > 1 else W.obs_z(0),
           [(0.7, 1 % (1 << n), (1 << n) - 1), (-0.4, 0, 1)]]
    w = rng.normal(size=(batch, 2))
    circ = dq.Circuit(n, gates, nparams=npar, nfeatures=2)
    dobs = dq.Observables(obs)
    st = torch.empty((batch, 1 << n), dtype=dt, device="cuda")
    ctx.state_init(st, n)
    ctx.apply_circuit(circ, dev(params), st, data=dev(data), params_per_row=ppr)
    keep = st.clone()
    gp, gd = ctx.adjoint_grad(circ, dev(params), dobs, st, data=dev(data), row_weights=dev(w),
                              params_per_row=ppr)
    assert torch.equal(st, keep), "state must be preserved without the clobber flag"
    e_ref, gp_ref, gd_ref = oracle.adjoint(n, gates, obs, params, data, batch=batch, params_per_row=ppr,
                                           row_weights=w)
    gscale = float(np.abs(w).max(axis=1).sum()) * obs_scale(obs)
    assert_rel(gp.cpu().numpy(), gp_ref, dt, "grad params", zero_scale=gscale)
    assert_rel(gd.cpu().numpy(), gd_ref, dt, "grad data", zero_scale=gscale)
    # the one-call path gives the same expectations and gradients
    e2, gp2, gd2, _ = ctx.forward_grad(circ, dev(params), dobs, batch, dt, data=dev(data), row_weights=dev(w),
                                       params_per_row=ppr)
    assert_rel(e2.cpu().numpy(), e_ref, dt, "expectations (forward_grad)", zero_scale=obs_scale(obs))
    assert_rel(gp2.cpu().numpy(), gp_ref, dt, "grad params (forward_grad)", zero_scale=gscale)
    assert_rel(gd2.cpu().numpy(), gd_ref, dt, "grad data (forward_grad)", zero_scale=gscale)


def test_clobber_flag_uses_state(ctx):
    ctx.set_path(dq.PATH_PLAIN)
    n, batch = 6, 2
    rng = np.random.default_rng(9)
    gates, npar = random_gates(n, 40, rng)
    params = rng.uniform(-3, 3, size=npar)
    circ = dq.Circuit(n, gates, nparams=npar)
    obs = [W.obs_sum_z(n)]
    st = torch.empty((batch, 1 << n), dtype=torch.complex128, device="cuda")
    ctx.state_init(st, n)
    ctx.apply_circuit(circ, dev(params), st)
    gp, _ = ctx.adjoint_grad(circ, dev(params), dq.Observables(obs), st, clobber=True)
    _, gp_ref, _ = oracle.adjoint(n, gates, obs, params, batch=batch)
    assert_rel(gp.cpu().numpy(), gp_ref, torch.complex128)


@pytest.mark.parametrize("dtype", sorted(DTYPES))
@pytest.mark.parametrize("n,batch", [(17, 2), (20, 1)])
def test_qft_controlled_phase_fans(ctx, dtype, n, batch):
    """QFT columns (runs of controlled phases sharing one qubit) on the tiled
    path are applied as fused fans: states against the oracle, from random
    product states so that every fan member's bit takes both values."""
    ctx.set_path(dq.PATH_FUSED)
    dt = DTYPES[dtype]
    rng = np.random.default_rng(n + 5)
    pre = [W.Gate("ry", (q,), angle=float(a)) for q, a in enumerate(rng.uniform(0, 2 * math.pi, size=n))]
    gates = pre + W.qft_gates(n) + [W.Gate("rz", (q,), angle=0.1 * q) for q in range(0, n, 3)]
    circ = dq.Circuit(n, gates)
    st = torch.empty((batch, 1 << n), dtype=dt, device="cuda")
    ctx.state_init(st, n)
    ctx.apply_circuit(circ, None, st)
    torch.cuda.synchronize()
    ctx.check()
    ref = oracle.run(n, gates, batch=batch)
    assert_amps(np_state(st), ref, dt, "QFT state")


@pytest.mark.parametrize("dtype", sorted(DTYPES))
@pytest.mark.parametrize("n,batch", [(17, 3), (20, 1)])
def test_diagonal_observables_in_last_forward_pass(ctx, dtype, n, batch):
    """Z-string observables measured by the last tiled forward pass (no
    separate observable pass), several observables and rows; a set with an
    X term takes the observable passes instead and must agree too."""
    ctx.set_path(dq.PATH_FUSED)
    dt = DTYPES[dtype]
    rng = np.random.default_rng(60 + n)
    gates = W.encode_layer(n) + W.hea_layers(n, 2)
    npar = 4 * n
    params = rng.uniform(0, 2 * math.pi, size=npar)
    data = rng.uniform(-math.pi, math.pi, size=(batch, n))
    circ = dq.Circuit(n, gates, nparams=npar, nfeatures=n)
    diag = [W.obs_sum_z(n), W.obs_z(0), [W.pauli_term(0.7, {1: "Z", n - 1: "Z"}), W.pauli_term(-0.2, {3: "Z"})]]
    mixed = diag + [W.obs_zz01_x0()]
    for obs in (diag, mixed):
        ref = oracle.expect(n, oracle.run(n, gates, params, data, batch=batch), obs)
        e, _, _, _ = ctx.forward_grad(circ, dev(params), dq.Observables(obs), batch, dt, data=dev(data),
                                      want_grad=False)
        torch.cuda.synchronize()
        ctx.check()
        assert_rel(e.cpu().numpy(), ref, dt, "expectations", zero_scale=obs_scale(obs))


@pytest.mark.parametrize("path", sorted(PATHS))
@pytest.mark.parametrize("n,batch", [(7, 3), (13, 2), (18, 1)])
def test_gradient_free_prefix(ctx, path, n, batch):
    """A parameter-free prefix (QFT) before the parametric layers: the reverse
    sweep stops at the first parametric gate; gradients, expectations and
    data gradients (when an encoding precedes the QFT) stay exact."""
    ctx.set_path(PATHS[path])
    rng = np.random.default_rng(40 + n)
    gates = W.encode_layer(n, wires=[0, n - 1]) + W.qft_gates(n) + W.hea_layers(n, 1)
    npar = 2 * n
    params = rng.uniform(0, 2 * math.pi, size=npar)
    data = rng.uniform(-math.pi, math.pi, size=(batch, 2))
    obs = [W.obs_tfim_open(n)]
    circ = dq.Circuit(n, gates, nparams=npar, nfeatures=2)
    exp_ref, gp_ref, gd_ref = oracle.adjoint(n, gates, obs, params, data=data, batch=batch)
    for with_data in (False, True):
        e, gp, gd, _ = ctx.forward_grad(circ, dev(params), dq.Observables(obs), batch, torch.complex64,
                                        data=dev(data), want_data_grad=with_data)
        assert (gd is not None) == with_data
        torch.cuda.synchronize()
        scale = obs_scale(obs)
        assert_rel(e.cpu().numpy(), exp_ref, torch.complex64, "expectation", zero_scale=scale)
        assert_rel(gp.cpu().numpy(), gp_ref, torch.complex64, "grad params", zero_scale=scale * batch)
        if with_data:
            assert_rel(gd.cpu().numpy(), gd_ref, torch.complex64, "grad data", zero_scale=scale)


# ---------------------------------------------------------------------------
# workload configurations
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("path", sorted(PATHS))
def test_config_c1_hea10_c128(ctx, path):
    ctx.set_path(PATHS[path])
    wl = W.config_c1()
    circ = dq.Circuit(wl.n, wl.gates, nparams=wl.nparams)
    st = torch.empty((1, 1 << wl.n), dtype=torch.complex128, device="cuda")
    e, _, _, _ = ctx.forward_grad(circ, dev(wl.params), dq.Observables(wl.observables), 1, torch.complex128,
                                  want_grad=False, state_out=st)
    ref = oracle.run(wl.n, wl.gates, wl.params)
    assert_amps(np_state(st), ref, torch.complex128)
    assert_rel(e.cpu().numpy(), oracle.expect(wl.n, ref, wl.observables), torch.complex128)


@pytest.mark.parametrize("path", sorted(PATHS))
def test_config_c2_hea20_c64(ctx, path):
    ctx.set_path(PATHS[path])
    wl = W.config_c2()
    circ = dq.Circuit(wl.n, wl.gates, nparams=wl.nparams)
    st = torch.empty((1, 1 << wl.n), dtype=torch.complex64, device="cuda")
    e, _, _, _ = ctx.forward_grad(circ, dev(wl.params), dq.Observables(wl.observables), 1, torch.complex64,
                                  want_grad=False, state_out=st)
    ref = oracle.run(wl.n, wl.gates, wl.params)
    assert_amps(np_state(st), ref, torch.complex64)
    assert_rel(e.cpu().numpy(), oracle.expect(wl.n, ref, wl.observables), torch.complex64)
    assert abs(torch.linalg.vector_norm(st.to(torch.complex128)).item() - 1.0) < 1e-5


@pytest.mark.parametrize("path", sorted(PATHS))
def test_config_c3_qml_batch(ctx, path):
    ctx.set_path(PATHS[path])
    wl = W.config_c3()
    circ = dq.Circuit(wl.n, wl.gates, nparams=wl.nparams, nfeatures=wl.nfeatures)
    e, gp, gd, _ = ctx.forward_grad(circ, dev(wl.params), dq.Observables(wl.observables), wl.batch,
                                    torch.complex64, data=dev(wl.data))
    e_ref, gp_ref, gd_ref = oracle.adjoint(wl.n, wl.gates, wl.observables, wl.params, wl.data, batch=wl.batch)
    assert_rel(e.cpu().numpy(), e_ref, torch.complex64, "per-sample <Z0>")
    assert_rel(gp.cpu().numpy(), gp_ref, torch.complex64, "grad params (batch sum)")
    assert_rel(gd.cpu().numpy(), gd_ref, torch.complex64, "grad data")


@pytest.mark.parametrize("path", sorted(PATHS))
def test_config_c4_uneven_batch(ctx, path):
    ctx.set_path(PATHS[path])
    circs = W.config_c4(1024)
    obs = [W.obs_zz01_x0()]
    dcs = [dq.Circuit(n, g, nparams=len(a)) for n, g, a in circs]
    params = np.concatenate([a for _, _, a in circs])
    offs = np.cumsum([0] + [len(a) for _, _, a in circs])
    e, gp = ctx.batch_forward_grad(dcs, dev(params), dq.Observables(obs), torch.complex64)
    e = e.cpu().numpy()
    gp = gp.cpu().numpy()
    # sampled circuits: every 16th plus every 16-qubit one
    pick = sorted(set(range(0, 1024, 16)) | {i for i, c in enumerate(circs) if c[0] == 16})
    # the expectations of the sampled circuits form one result vector; each
    # circuit's gradient is judged on its own largest element
    e_ref = []
    for i in pick:
        n, g, a = circs[i]
        er, gr, _ = oracle.adjoint(n, g, obs, a)
        e_ref.append(er[0, 0])
        assert_rel(gp[offs[i]:offs[i + 1]], gr, torch.complex64, f"circuit {i} gradient", zero_scale=obs_scale(obs))
    assert_rel(e[pick], e_ref, torch.complex64, "sampled circuits' expectations", zero_scale=obs_scale(obs))


@pytest.mark.parametrize("dtype", sorted(DTYPES))
def test_config_c4_autotuned_launch(ctx, dtype):
    """The uneven batch with its autotuned launch: the tuner's own outputs and
    a later call with the cached choice both match the oracle."""
    ctx.set_path(dq.PATH_FUSED)
    dt = DTYPES[dtype]
    circs = W.config_c4(256)
    obs = [W.obs_zz01_x0()]
    dcs = [dq.Circuit(n, g, nparams=len(a)) for n, g, a in circs]
    params = np.concatenate([a for _, _, a in circs])
    offs = np.cumsum([0] + [len(a) for _, _, a in circs])
    choice = ctx.batch_autotune(dcs, dev(params), dq.Observables(obs), dt)
    assert choice[0] in (10, 11, 12) and choice[1] in (128, 256, 512) and choice[2] in (2, 4, 8), choice
    assert choice[3] in (0, 64, 96, 128, 160), choice
    e, gp = ctx.batch_forward_grad(dcs, dev(params), dq.Observables(obs), dt)
    e = e.cpu().numpy()
    gp = gp.cpu().numpy()
    pick = sorted(set(range(0, 256, 8)) | {i for i, c in enumerate(circs) if c[0] >= 14})
    e_ref = []
    for i in pick:
        n, g, a = circs[i]
        er, gr, _ = oracle.adjoint(n, g, obs, a)
        e_ref.append(er[0, 0])
        assert_rel(gp[offs[i]:offs[i + 1]], gr, dt, f"circuit {i} gradient (tuned {choice})",
                   zero_scale=obs_scale(obs))
    assert_rel(e[pick], e_ref, dt, f"expectations (tuned {choice})", zero_scale=obs_scale(obs))


@pytest.mark.parametrize("path", sorted(PATHS))
@pytest.mark.parametrize("n", [14, 17])
def test_config_c5_structure_reduced(ctx, path, n):
    """QFT + 10 layers + TFIM at reduced n, compared in full with the oracle."""
    ctx.set_path(PATHS[path])
    wl = W.config_c5(n)
    circ = dq.Circuit(wl.n, wl.gates, nparams=wl.nparams)
    st = torch.empty((1, 1 << n), dtype=torch.complex64, device="cuda")
    e, gp, _, _ = ctx.forward_grad(circ, dev(wl.params), dq.Observables(wl.observables), 1, torch.complex64,
                                   state_out=st)
    e_ref, gp_ref, _ = oracle.adjoint(n, wl.gates, wl.observables, wl.params)
    assert_amps(np_state(st), oracle.run(n, wl.gates, wl.params), torch.complex64)
    assert_rel(e.cpu().numpy(), e_ref, torch.complex64, "TFIM energy")
    assert_rel(gp.cpu().numpy(), gp_ref, torch.complex64, "TFIM gradient")


@pytest.mark.parametrize("path", ["fused"])
def test_config_c5_full_size_factorised(ctx, path):
    """30 qubits, 1380 gates, 600 params, three resident vectors: the ring is
    split into three interleaved 10-qubit rings so the exact answer is a
    product the oracle computes from 10-qubit pieces."""
    ctx.set_path(PATHS[path])
    n = 30
    wl, rings = factorised_c5(n)
    energy, grad, states = factorised_reference(oracle, n, rings, wl)
    circ = dq.Circuit(n, wl.gates, nparams=wl.nparams)
    st = torch.empty((1, 1 << n), dtype=torch.complex64, device="cuda")
    e, gp, _, _ = ctx.forward_grad(circ, dev(wl.params), dq.Observables(wl.observables), 1, torch.complex64,
                                   state_out=st)
    assert_rel(e.cpu().numpy(), [energy], torch.complex64, "energy")
    assert_rel(gp.cpu().numpy(), grad, torch.complex64, "gradient")
    rng = np.random.default_rng(30)
    idx = np.concatenate([[0, (1 << n) - 1], rng.integers(0, 1 << n, size=400)])
    got = st.view(-1)[torch.as_tensor(idx, device="cuda")].cpu().numpy().astype(np.complex128)
    ref = np.array([factorised_amplitude(n, rings, states, int(b)) for b in idx])
    assert_amps(got, ref, torch.complex64, "sampled amplitudes")
    assert np.max(np.abs(got - ref)) <= 1e-3 * np.max(np.abs(ref))
    del st
    torch.cuda.empty_cache()


# ---------------------------------------------------------------------------
# autograd boundary
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("n,budget", [(10, None), (15, None), (15, 0)])
def test_autograd_function(ctx, n, budget):
    ctx.set_path(dq.PATH_AUTO)
    rng = np.random.default_rng(n)
    batch = 6
    gates = W.encode_layer(n) + W.hea_layers(n, 2)
    npar = 4 * n
    circ = dq.Circuit(n, gates, nparams=npar, nfeatures=n)
    obs = [W.obs_z(0), W.obs_tfim_open(n, 0.5)]
    params = torch.tensor(rng.uniform(0, 6, npar), device="cuda", requires_grad=True)
    data = torch.tensor(rng.uniform(-3, 3, (batch, n)), device="cuda", requires_grad=True)
    wts = torch.tensor(rng.normal(size=(batch, 2)), device="cuda")
    e = dq.expectation(circ, params, dq.Observables(obs), data=data, context=ctx, memory_budget=budget)
    (e * wts).sum().backward()
    e_ref, gp_ref, gd_ref = oracle.adjoint(n, gates, obs, params.detach().cpu().numpy(),
                                           data.detach().cpu().numpy(), batch=batch,
                                           row_weights=wts.cpu().numpy())
    assert_rel(e.detach().cpu().numpy(), e_ref, torch.complex64)
    assert_rel(params.grad.cpu().numpy(), gp_ref, torch.complex64)
    assert_rel(data.grad.cpu().numpy(), gd_ref, torch.complex64)


@pytest.mark.parametrize("n", [10, 15])
def test_autograd_backward_twice(ctx, n):
    """retain_graph=True and a second backward: the kept forward states are
    swept in place by the first backward, so the second must recompute and
    give the same gradients (both against the oracle)."""
    ctx.set_path(dq.PATH_AUTO)
    rng = np.random.default_rng(100 + n)
    batch = 4
    gates = W.encode_layer(n) + W.hea_layers(n, 2)
    npar = 4 * n
    circ = dq.Circuit(n, gates, nparams=npar, nfeatures=n)
    obs = [W.obs_tfim_open(n, 0.5)]
    params = torch.tensor(rng.uniform(0, 6, npar), device="cuda", requires_grad=True)
    data = torch.tensor(rng.uniform(-3, 3, (batch, n)), device="cuda", requires_grad=True)
    wts = torch.tensor(rng.normal(size=(batch, 1)), device="cuda")
    e = dq.expectation(circ, params, dq.Observables(obs), data=data, context=ctx, memory_budget=1 << 40)
    loss = (e * wts).sum()
    _, gp_ref, gd_ref = oracle.adjoint(n, gates, obs, params.detach().cpu().numpy(), data.detach().cpu().numpy(),
                                       batch=batch, row_weights=wts.cpu().numpy())
    gscale = float(wts.abs().sum()) * obs_scale(obs)
    for k in range(2):
        gp, gd = torch.autograd.grad(loss, (params, data), retain_graph=True)
        assert_rel(gp.cpu().numpy(), gp_ref, torch.complex64, f"backward {k}: grad params", zero_scale=gscale)
        assert_rel(gd.cpu().numpy(), gd_ref, torch.complex64, f"backward {k}: grad data", zero_scale=gscale)


# ---------------------------------------------------------------------------
# edge cases and validation
# ---------------------------------------------------------------------------
def test_empty_and_degenerate(ctx):
    ctx.set_path(dq.PATH_AUTO)
    st = torch.empty((0, 8), dtype=torch.complex64, device="cuda")
    ctx.apply_circuit(dq.Circuit(3, [W.Gate("h", (0,))]), None, st)       # batch 0: no-op
    st = torch.empty((2, 8), dtype=torch.complex64, device="cuda")
    ctx.state_init(st, 3)
    ctx.apply_circuit(dq.Circuit(3, []), None, st)                           # no gates
    ref = np.zeros((2, 8))
    ref[:, 0] = 1
    assert_amps(np_state(st), ref, torch.complex64)
    e, gp, _, _ = ctx.forward_grad(dq.Circuit(3, [], nparams=0), None, dq.Observables([W.obs_z(2)]), 2,
                                   torch.complex64)
    assert np.allclose(e.cpu().numpy(), 1.0)
    e = ctx.expect(3, dq.Observables([[]]), st)                              # empty observable
    assert np.allclose(e.cpu().numpy(), 0.0)


@pytest.mark.parametrize("bad", ["wire", "same", "kind", "param", "data_missing", "fixed_angle_param",
                                 "u3_fixed", "u3_span", "ccx_same", "ccx_wire", "dtype", "null_state",
                                 "misaligned"])
def test_invalid_arguments_are_rejected(ctx, bad):
    n = 4
    st = torch.empty((1, 16), dtype=torch.complex64, device="cuda")
    ctx.state_init(st, n)
    before = st.clone()
    params = dev(np.zeros(2))
    gates = [W.Gate("h", (0,))]
    circ_kw = {}
    state = st
    if bad == "wire":
        gates = [W.Gate("h", (4,))]
    elif bad == "same":
        gates = [W.Gate("cnot", (1, 1))]
    elif bad == "kind":
        gates = [(99, (0,), -1, -1, 0.0)]
    elif bad == "param":
        gates = [W.Gate("rx", (0,), param=5)]
        circ_kw = {"nparams": 2}
    elif bad == "data_missing":
        gates = [W.Gate("rx", (0,), data=0)]
        circ_kw = {"nfeatures": 1}
    elif bad == "fixed_angle_param":
        gates = [W.Gate("h", (0,), param=0)]
        circ_kw = {"nparams": 1}
    elif bad == "u3_fixed":
        gates = [W.Gate("u3", (0,), angle=0.5)]
    elif bad == "u3_span":
        gates = [W.Gate("u3", (0,), param=0)]
        circ_kw = {"nparams": 2}
    elif bad == "ccx_same":
        gates = [W.Gate("ccx", (0, 2, 0))]
    elif bad == "ccx_wire":
        gates = [W.Gate("ccx", (0, 1, 4))]
    circ = dq.Circuit(n, gates, **circ_kw)
    with pytest.raises(dq.DQError) as ei:
        if bad == "dtype":
            ctx.lib.dq_state_init(ctx.h, n, 1, 7, st.data_ptr(), None) and ctx._check(7 and 1, "x")
            ctx._check(ctx.lib.dq_state_init(ctx.h, n, 1, 7, st.data_ptr(), None), "state_init")
        elif bad == "null_state":
            ctx._check(ctx.lib.dq_apply_circuit(ctx.h, circ.ref(), None, 0, None, None, 1, 0, None), "apply")
        elif bad == "misaligned":
            ctx._check(ctx.lib.dq_apply_circuit(ctx.h, circ.ref(), None, 0, None, st.data_ptr() + 8, 1, 0, None),
                       "apply")
        else:
            ctx.apply_circuit(circ, params if bad != "data_missing" else params, state)
    assert ei.value.status == 1
    torch.cuda.synchronize()
    assert torch.equal(st, before), "nothing may be launched on invalid input"


def test_launch_counter_counts_kernels(ctx):
    ctx.set_path(dq.PATH_PLAIN)
    n = 8
    gates = [W.Gate("h", (q,)) for q in range(n)]
    st = torch.empty((1, 1 << n), dtype=torch.complex64, device="cuda")
    c0 = ctx.launch_count
    ctx.state_init(st, n)
    ctx.apply_circuit(dq.Circuit(n, gates), None, st)
    assert ctx.launch_count - c0 == 1 + 1 + n      # init, bind, one sweep per gate


@pytest.mark.parametrize("n,batch,want", [(12, 64, {"k_rows"}),
                                          (18, 2, {"k_tile_multi", "k_tile_obs", "k_tile_adj"}),
                                          (23, 1, {"k_tile_fwd", "k_tile_obs", "k_tile_adj"})])
def test_fused_path_runs_the_fused_kernels(ctx, n, batch, want):
    """The fused path must not fall back to per-gate sweeps silently: whole
    rows on chip, the persistent multi-pass forward for states that stay in
    L2 (2 x 2^18 complex64 = 4 MiB), one launch per forward pass above
    32 MiB (2^23 complex64 = 64 MiB)."""
    ctx.set_path(dq.PATH_FUSED)
    gates = W.encode_layer(n) + W.hea_layers(n, 2)
    circ = dq.Circuit(n, gates, nparams=4 * n, nfeatures=n)
    rng = np.random.default_rng(n)
    params = dev(rng.uniform(0, 6, 4 * n))
    data = dev(rng.uniform(-3, 3, (batch, n)))
    ctx.set_tracing(True)
    ctx.forward_grad(circ, params, dq.Observables([W.obs_tfim_open(n, 0.5)]), batch, torch.complex64, data=data)
    names = set(ctx.trace())
    ctx.set_tracing(False)
    assert want <= names, names
    assert "k_sweep" not in names and "k_adj" not in names


@pytest.mark.parametrize("n,batch,path", [(10, 32, "fused"), (18, 1, "fused"), (9, 3, "plain")])
def test_graph_replay_reads_current_values(ctx, n, batch, path):
    """Replayed graphs must see parameter and data values written in place
    between calls, and give what a fresh (non-graph) call gives."""
    ctx.set_path(PATHS[path])
    gates = W.encode_layer(n) + W.hea_layers(n, 2)
    circ = dq.Circuit(n, gates, nparams=4 * n, nfeatures=n)
    obs = dq.Observables([W.obs_tfim_open(n, 0.5)])
    rng = np.random.default_rng(7 + n)
    params = dev(rng.uniform(0, 6, 4 * n))
    data = dev(rng.uniform(-3, 3, (batch, n)))
    e = torch.empty((batch, 1), dtype=torch.float64, device="cuda")
    gp = torch.empty(4 * n, dtype=torch.float64, device="cuda")
    gd = torch.empty((batch, n), dtype=torch.float64, device="cuda")
    ctx.set_graphs(True)
    try:
        for call in range(4):
            params.copy_(dev(rng.uniform(0, 6, 4 * n)))
            data.copy_(dev(rng.uniform(-3, 3, (batch, n))))
            ctx.forward_grad(circ, params, obs, batch, torch.complex64, data=data, expect_out=e, grad_params=gp,
                             grad_data=gd)
            torch.cuda.synchronize()
            e_ref, gp_ref, gd_ref = oracle.adjoint(n, gates, [W.obs_tfim_open(n, 0.5)], params.cpu().numpy(),
                                                   data.cpu().numpy(), batch=batch)
            assert_rel(e.cpu().numpy(), e_ref, torch.complex64, f"call {call} expectation", zero_scale=obs_scale([W.obs_tfim_open(n, 0.5)]))
            fl = batch * obs_scale([W.obs_tfim_open(n, 0.5)])
            assert_rel(gp.cpu().numpy(), gp_ref, torch.complex64, f"call {call} grad params", zero_scale=fl)
            assert_rel(gd.cpu().numpy(), gd_ref, torch.complex64, f"call {call} grad data", zero_scale=fl)
    finally:
        ctx.set_graphs(False)


def test_tracing_inside_replayed_graphs(ctx):
    """With graph replay and tracing both on, every call's kernels are
    counted once (first call issued directly, later ones from the traced
    graph) with positive device times, and results stay exact."""
    ctx.set_path(dq.PATH_FUSED)
    n = 18
    rng = np.random.default_rng(18)
    gates = W.hea_layers(n, 2)
    params = rng.uniform(0, 2 * math.pi, size=4 * n)
    obs = [W.obs_sum_z(n)]
    circ = dq.Circuit(n, gates, nparams=4 * n)
    o = dq.Observables(obs)
    p = dev(params)
    e = torch.empty((1, 1), dtype=torch.float64, device="cuda")
    st = torch.empty((1, 1 << n), dtype=torch.complex64, device="cuda")
    ref = oracle.expect(n, oracle.run(n, gates, params), obs)
    ctx.set_graphs(True)
    try:
        ctx.forward_grad(circ, p, o, 1, torch.complex64, want_grad=False, state_out=st, expect_out=e)
        torch.cuda.synchronize()
        per_call = ctx.launch_count
        ctx.set_tracing(True)
        l0 = ctx.launch_count
        for _ in range(5):
            ctx.forward_grad(circ, p, o, 1, torch.complex64, want_grad=False, state_out=st, expect_out=e)
        tr = ctx.trace()
        per_call = (ctx.launch_count - l0) // 5
        ctx.set_tracing(False)
    finally:
        ctx.set_graphs(False)
    assert per_call > 0
    assert sum(c for c, _ in tr.values()) == 5 * per_call
    assert all(ms > 0 for _, ms in tr.values())
    assert_rel(e.cpu().numpy(), ref, torch.complex64, "expectation", zero_scale=obs_scale(obs))
