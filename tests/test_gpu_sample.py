"""GPU parity of shot sampling (dq_sample) against the oracle's inversion of
the cumulative distribution: identical outcomes for the same uniforms except
where a target lies within rounding of a cumulative boundary (there either
neighbour is valid and the test checks validity), the built-in splitmix64
stream against the shared generator, marginal packing, zero-probability
outcomes, a chi-square check of the Born rule and a 28-qubit state checked
shot by shot against an independent cumulative sum."""
import numpy as np
import pytest
import torch

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("CUDA GPU required", allow_module_level=True)

import paper_2512_18995_gb300 as dq  # noqa: E402
from paper_2512_18995_gb300 import build as dqbuild  # noqa: E402

dqbuild.build()

DTYPES = {"c64": torch.complex64, "c128": torch.complex128}
# Cumulative sums of the two sides add in different orders; a target closer
# than this (relative to the row total) to a boundary may go either way.
BOUNDARY_TOL = 1e-12


@pytest.fixture(scope="module")
def ctx():
    c = dq.Context(0)
    yield c
    c.close()


def rand_states(rng, batch, n, dt, zero_every=0):
    st = rng.normal(size=(batch, 1 << n)) + 1j * rng.normal(size=(batch, 1 << n))
    if zero_every:
        st[:, ::zero_every] = 0
    t = torch.tensor(st, dtype=dt, device="cuda")
    return t, t.cpu().numpy().astype(np.complex128)


def check_outcomes(got, ref, states, u):
    """Equal outcomes, or (near a boundary) a valid outcome for the target."""
    got = np.asarray(got)
    bad = np.argwhere(got != ref)
    for r, s in bad:
        p = states[r].real ** 2 + states[r].imag ** 2
        c = np.cumsum(p)
        z = c[-1]
        t = u[r, s] * z
        i = int(got[r, s])
        lo = c[i - 1] if i > 0 else 0.0
        assert p[i] > 0, f"row {r} shot {s}: drew zero-probability outcome {i}"
        assert lo - BOUNDARY_TOL * z <= t <= c[i] + BOUNDARY_TOL * z, \
            f"row {r} shot {s}: outcome {i} (oracle {ref[r, s]}) invalid for target {t}"
    assert bad.shape[0] <= max(2, got.size // 100000), f"{bad.shape[0]} outcomes differ"


@pytest.mark.parametrize("dtype", sorted(DTYPES))
@pytest.mark.parametrize("n,batch,shots", [(1, 3, 100), (3, 2, 500), (7, 5, 300), (8, 1, 1000), (9, 3, 700),
                                           (12, 64, 50), (18, 2, 4000), (19, 1, 3000), (21, 2, 2000)])
def test_sampling_matches_oracle(ctx, dtype, n, batch, shots):
    dt = DTYPES[dtype]
    rng = np.random.default_rng(40 + 3 * n + batch)
    t, st = rand_states(rng, batch, n, dt, zero_every=3 if n > 2 else 0)
    u = W.uniform_array(500 + n, batch * shots, 0.0, 1.0).reshape(batch, shots)
    got = ctx.sample(n, t, shots, uniforms=torch.tensor(u, device="cuda")).cpu().numpy()
    ctx.check()
    ref = oracle.sample(n, st, u)
    check_outcomes(got, ref, st, u)


@pytest.mark.parametrize("n", [5, 14, 20])
def test_seeded_stream_equals_given_uniforms(ctx, n):
    """With no uniforms the kernel draws output k of the splitmix64 stream of
    the seed, the same numbers the shared input generator produces."""
    batch, shots, seed = 3, 1000, 0x1234567 + n
    rng = np.random.default_rng(n)
    t, _ = rand_states(rng, batch, n, torch.complex64)
    u = W.uniform_array(seed, batch * shots, 0.0, 1.0)
    a = ctx.sample(n, t, shots, seed=seed)
    b = ctx.sample(n, t, shots, uniforms=torch.tensor(u, device="cuda"))
    assert torch.equal(a, b)


@pytest.mark.parametrize("n,wires", [(6, [0]), (6, [5, 1, 3]), (13, [12, 0, 7, 2]), (17, list(range(17)))])
def test_marginal_outcomes(ctx, n, wires):
    batch, shots = 2, 2000
    rng = np.random.default_rng(n + len(wires))
    t, st = rand_states(rng, batch, n, torch.complex64)
    u = W.uniform_array(900 + n, batch * shots, 0.0, 1.0).reshape(batch, shots)
    ud = torch.tensor(u, device="cuda")
    full = ctx.sample(n, t, shots, uniforms=ud).cpu().numpy()
    part = ctx.sample(n, t, shots, uniforms=ud, wires=wires).cpu().numpy()
    proj = np.zeros_like(full)
    for q in sorted(wires):
        proj = (proj << 1) | ((full >> (n - 1 - q)) & 1)
    assert (part == proj).all()
    assert (part == oracle.sample(n, st, u, wires=wires)).mean() > 0.999


def test_born_rule_chi_square(ctx):
    """One million shots of a 6-qubit state: chi-square against |psi|^2 at
    the 0.1% level (fixed seed), and no impossible outcome."""
    from scipy.stats import chi2
    n, shots = 6, 1_000_000
    rng = np.random.default_rng(66)
    t, st = rand_states(rng, 1, n, torch.complex128, zero_every=5)
    p = st[0].real ** 2 + st[0].imag ** 2
    p /= p.sum()
    out = ctx.sample(n, t, shots, seed=2025).cpu().numpy()[0]
    counts = np.bincount(out, minlength=1 << n)
    assert counts[p == 0].sum() == 0
    nz = p > 0
    stat = float(np.sum((counts[nz] - shots * p[nz]) ** 2 / (shots * p[nz])))
    assert stat < chi2.ppf(0.999, int(nz.sum()) - 1)


def test_degenerate_rows(ctx):
    """Basis states give their index; a row of zeros gives 2^n - 1; an empty
    request launches nothing."""
    n = 10
    t = torch.zeros((3, 1 << n), dtype=torch.complex64, device="cuda")
    t[0, 0] = 1
    t[1, 777] = -1j
    out = ctx.sample(n, t, 64, seed=1).cpu().numpy()
    assert (out[0] == 0).all() and (out[1] == 777).all() and (out[2] == (1 << n) - 1).all()
    assert ctx.sample(n, t, 0).numel() == 0


def test_full_size_shots_are_valid(ctx):
    """28 qubits (2 GiB complex64): 4096 shots, each checked against a
    cumulative sum taken independently (torch, FP64 on the device)."""
    n, shots = 28, 4096
    gen = torch.Generator(device="cuda").manual_seed(28)
    t = torch.randn((1, 1 << n), dtype=torch.complex64, device="cuda", generator=gen)
    u = W.uniform_array(2828, shots, 0.0, 1.0)
    out = ctx.sample(n, t, shots, uniforms=torch.tensor(u, device="cuda"))[0]
    ctx.check()
    p = t[0].real.double() ** 2 + t[0].imag.double() ** 2
    c = torch.cumsum(p, 0)
    del p
    z = float(c[-1])
    idx = out.long()
    hi = c[idx].cpu().numpy()
    lo = torch.where(idx > 0, c[(idx - 1).clamp(min=0)], torch.zeros_like(c[idx])).cpu().numpy()
    target = u * z
    assert (lo - 1e-11 * z <= target).all() and (target <= hi + 1e-11 * z).all()
    assert (hi > lo).all(), "a zero-probability outcome was drawn"
    del c, t
    torch.cuda.empty_cache()


def test_sampling_rejects_bad_arguments(ctx):
    t = torch.zeros((1, 16), dtype=torch.complex64, device="cuda")
    with pytest.raises(dq.DQError, match="wire_mask"):
        ctx.sample(4, t, 10, wires=[4])
    with pytest.raises(ValueError):
        ctx.sample(4, t, 10, uniforms=torch.zeros(3, dtype=torch.float64, device="cuda"))


def test_measure_counts(ctx):
    """measure() returns bitstring counts whose total is the shot count and
    whose keys follow the selected wires (first listed wire leftmost)."""
    n = 3
    st = torch.zeros((1, 8), dtype=torch.complex64, device="cuda")
    st[0, 0b101] = 1.0
    c = dq.measure(st, n, 100, context=ctx)[0]
    assert c == {"101": 100}
    c = dq.measure(st, n, 50, wires=[2, 0], context=ctx)[0]
    assert c == {"11": 50}
    st2 = torch.full((1, 8), 8 ** -0.5, dtype=torch.complex64, device="cuda")
    c = dq.measure(st2, n, 4000, seed=3, context=ctx)[0]
    assert sum(c.values()) == 4000 and len(c) == 8
