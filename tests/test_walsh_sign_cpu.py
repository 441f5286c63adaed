"""The sign factorisation behind the Z-string sums of the forward epilogue and
the observable passes, checked exhaustively on small cases (CPU): a thread t
of a CTA of 2^lb threads holds the tile amplitudes l = t + i 2^lb, and under a
Z string with tile mask s

    sum_i (-1)^parity(l_i & s) p_i = (-1)^parity(t & s) * W[s >> lb],

where W is the Walsh-Hadamard transform of the thread's values,
W[h] = sum_i (-1)^popc(i & h) p_i, computed in place by butterflies.  The
expectation of a Pauli Z string (API Overview: expectations of Pauli-string
observables) is the signed sum of the probabilities |psi_l|^2."""
import numpy as np


def parity(x: int) -> int:
    return bin(x).count("1") & 1


def butterfly_wht(v):
    """In-place Walsh-Hadamard transform by butterflies, as the kernels do it."""
    v = list(v)
    st = 1
    while st < len(v):
        for i in range(len(v)):
            if not i & st:
                a0, a1 = v[i], v[i | st]
                v[i], v[i | st] = a0 + a1, a0 - a1
        st <<= 1
    return v


def test_butterflies_compute_the_hadamard_transform():
    rng = np.random.default_rng(1)
    for m in (1, 2, 3, 4):
        n = 1 << m
        p = rng.random(n)
        hadamard = np.array([[(-1) ** parity(h & i) for i in range(n)] for h in range(n)])
        np.testing.assert_allclose(butterfly_wht(p), hadamard @ p, rtol=0, atol=1e-12)


def test_signed_sum_factorises_over_thread_and_register_bits():
    rng = np.random.default_rng(2)
    for m in (3, 4):          # 8 values a thread (observable passes), 16 (forward epilogue, M = 4)
        for lb in (0, 1, 3, 5):
            k = lb + m
            p = rng.random(1 << k)
            for s in range(1 << k):
                for t in range(1 << lb):
                    vals = [p[t + (i << lb)] for i in range(1 << m)]
                    direct = sum((-1) ** parity((t + (i << lb)) & s) * v for i, v in enumerate(vals))
                    w = butterfly_wht(vals)
                    factored = (-1) ** parity(t & s) * w[(s >> lb) & ((1 << m) - 1)]
                    assert abs(direct - factored) < 1e-12, (m, lb, s, t)


def test_gathered_weights_give_each_amplitudes_diagonal_factor():
    """The lambda side: sum over Z terms j of w_j (-1)^parity(l_i & s_j) equals
    the transform of the weights gathered per s_j >> lb, each signed by
    parity(t & s_j)."""
    rng = np.random.default_rng(3)
    m, lb = 3, 4
    k = lb + m
    for _ in range(50):
        terms = [(int(rng.integers(1 << k)), float(rng.normal())) for _ in range(int(rng.integers(1, 12)))]
        for t in range(1 << lb):
            gathered = [0.0] * (1 << m)
            for s, wgt in terms:
                gathered[s >> lb] += (-1) ** parity(t & s) * wgt
            d = butterfly_wht(gathered)
            for i in range(1 << m):
                direct = sum(wgt * (-1) ** parity((t + (i << lb)) & s) for s, wgt in terms)
                assert abs(d[i] - direct) < 1e-12
