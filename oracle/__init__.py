"""FP64 CPU oracle -- TEST INFRASTRUCTURE ONLY.

Python side of the plain C reference simulator in ``oracle.c``.  Only the
test-suite, the package smoke check and the benchmark's CPU-baseline leg may
import this module; the library's product path never does, and this module
imports nothing from the library.

Inputs are the plain descriptions from :mod:`workloads` (gate tuples, numpy
arrays, Pauli terms as ``(coeff, xmask, zmask)`` by wire).  States are numpy
``complex128`` arrays of shape ``(batch, 2**n)`` with wire 0 as the most
significant index bit.

Parity: pinned -- see ``tests/test_oracle_pins.py`` (closed forms, unitarity,
brute-force dense Kronecker products for n <= 8, parameter-shift and central
finite differences).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_default = None

# The oracle's own gate codes (order of the enum in oracle.c).
_KIND = {k: i for i, k in enumerate(
    ["h", "x", "y", "z", "s", "rx", "ry", "rz",
     "cnot", "cz", "cp", "swap", "crx", "cry", "crz",
     "p", "u3", "rxx", "ryy", "rzz", "ccx", "bitflip", "phaseflip", "depolarizing", "ampdamp"])}


def compile_source(src: str, out: str) -> str:
    """Compile an oracle source file into a shared library (gcc, OpenMP)."""
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fopenmp", "-fPIC",
           "-shared", src, "-o", tmp, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, out)
    return out


def build(force: bool = False) -> str:
    """Compile ``oracle.c`` into ``liboracle.so`` next to it."""
    if not force and os.path.exists(_LIB_PATH) and \
            os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
        return _LIB_PATH
    return compile_source(_SRC, _LIB_PATH)


def _bind(path):
    lib = ctypes.CDLL(path)
    P = ctypes.c_void_p
    I = ctypes.c_int
    lib.oracle_num_threads.restype = I
    lib.oracle_gate_block.argtypes = [I, ctypes.c_double, P]
    gate_args = [I, I, P, P, P, P, P, P, P, P, I, I, P, I]
    lib.oracle_run.argtypes = gate_args + [I, P]
    lib.oracle_apply.argtypes = gate_args + [I, I, P]
    lib.oracle_expect.argtypes = [I, P, P, P, P, I, I, P, P]
    lib.oracle_adjoint.argtypes = gate_args + [I, P, P, P, P, I, P, P, P, P]
    lib.oracle_apply_dense.argtypes = [I, I, P, I, P]
    lib.oracle_hessian.argtypes = [I, I, P, P, P, P, P, P, P, P, I, P, I, I, P, P, P, P, I, P, P]
    lib.oracle_density.argtypes = [I, I, P, P, P, P, P, P, P, P, I, P, I, I, P, P, P, P, I, P, P]
    lib.oracle_sample.argtypes = [I, I, P, ctypes.c_int64, P, ctypes.c_uint64, P]
    return lib


def _load():
    global _default
    with _lock:
        if _default is None:
            build()
            _default = _bind(_LIB_PATH)
    return _default


def num_threads() -> int:
    return _load().oracle_num_threads()


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


class _Gates:
    """Gate list as the flat arrays the C side reads."""

    def __init__(self, gates):
        g = list(gates)
        self.count = len(g)
        self.kind = np.array([_KIND[x.kind] for x in g] or [0], dtype=np.int32)
        self.w0 = np.array([x.wires[0] for x in g] or [0], dtype=np.int32)
        self.w1 = np.array([x.wires[1] if len(x.wires) > 1 else -1 for x in g] or [0], dtype=np.int32)
        self.w2 = np.array([x.wires[2] if len(x.wires) > 2 else -1 for x in g] or [0], dtype=np.int32)
        self.pidx = np.array([x.param for x in g] or [0], dtype=np.int32)
        self.didx = np.array([x.data for x in g] or [0], dtype=np.int32)
        self.angle = np.array([x.angle for x in g] or [0.0], dtype=np.float64)

    def args(self, n, params, params_per_row, data):
        params = np.ascontiguousarray(params, dtype=np.float64) if params is not None else np.zeros(1)
        nparams = params.shape[-1] if params.ndim else 1
        if data is not None:
            data = np.ascontiguousarray(data, dtype=np.float64)
            nfeat = data.shape[-1]
        else:
            nfeat = 0
        self._keep = (params, data)
        return [n, self.count, _ptr(self.kind), _ptr(self.w0), _ptr(self.w1), _ptr(self.w2), _ptr(self.pidx),
                _ptr(self.didx), _ptr(self.angle), _ptr(params), int(nparams),
                int(bool(params_per_row)), _ptr(data), int(nfeat)]


class _Obs:
    def __init__(self, observables):
        obs = [list(o) for o in observables]
        terms = [t for o in obs for t in o]
        self.coeff = np.array([t[0] for t in terms] or [0.0], dtype=np.float64)
        self.x = np.array([t[1] for t in terms] or [0], dtype=np.uint64)
        self.z = np.array([t[2] for t in terms] or [0], dtype=np.uint64)
        offs = [0]
        for o in obs:
            offs.append(offs[-1] + len(o))
        self.offsets = np.array(offs, dtype=np.int32)
        self.nobs = len(obs)


def run(n, gates, params=None, data=None, batch=1, params_per_row=False, lib=None):
    """Final states (batch, 2**n) complex128 from |0...0>."""
    lib = lib or _load()
    g = _Gates(gates)
    out = np.empty((batch, 1 << n), dtype=np.complex128)
    lib.oracle_run(*g.args(n, params, params_per_row, data), int(batch), _ptr(out))
    return out


def apply(n, gates, states, params=None, data=None, params_per_row=False, dagger=False, lib=None):
    """Apply the gate list (or its inverse) to given states, returning a copy."""
    lib = lib or _load()
    g = _Gates(gates)
    st = np.array(states, dtype=np.complex128, copy=True).reshape(-1, 1 << n)
    lib.oracle_apply(*g.args(n, params, params_per_row, data), st.shape[0], int(bool(dagger)), _ptr(st))
    return st


def expect(n, states, observables, lib=None):
    """(batch, nobs) expectations of Pauli-sum observables."""
    lib = lib or _load()
    st = np.ascontiguousarray(states, dtype=np.complex128).reshape(-1, 1 << n)
    o = _Obs(observables)
    out = np.empty((st.shape[0], o.nobs), dtype=np.float64)
    lib.oracle_expect(n, _ptr(o.coeff), _ptr(o.x), _ptr(o.z), _ptr(o.offsets), o.nobs,
                      st.shape[0], _ptr(st), _ptr(out))
    return out


def adjoint(n, gates, observables, params=None, data=None, batch=1, params_per_row=False,
            row_weights=None, lib=None):
    """Adjoint gradients.  Returns (expect (batch, nobs), grad_params, grad_data).

    grad_params has shape (nparams,) summed over rows for shared params, or
    (batch, nparams) when ``params_per_row``; grad_data is (batch, nfeat) or
    None when there is no encoded data."""
    lib = lib or _load()
    g = _Gates(gates)
    o = _Obs(observables)
    args = g.args(n, params, params_per_row, data)
    nparams, nfeat = args[10], args[13]
    exp = np.empty((batch, o.nobs), dtype=np.float64)
    gp = np.zeros((batch, nparams) if params_per_row else (nparams,), dtype=np.float64)
    gd = np.zeros((batch, nfeat), dtype=np.float64) if nfeat else None
    rw = None
    if row_weights is not None:
        rw = np.ascontiguousarray(row_weights, dtype=np.float64).reshape(batch, o.nobs)
    lib.oracle_adjoint(*args, int(batch), _ptr(o.coeff), _ptr(o.x), _ptr(o.z), _ptr(o.offsets),
                       o.nobs, _ptr(rw), _ptr(exp), _ptr(gp), _ptr(gd))
    return exp, gp, gd


def apply_dense(n, nw, unitary, states, lib=None):
    """(I (x) U) on the nw lowest-order wires of every row; returns a copy."""
    lib = lib or _load()
    u = np.ascontiguousarray(unitary, dtype=np.complex128).reshape(1 << nw, 1 << nw)
    st = np.array(states, dtype=np.complex128, copy=True).reshape(-1, 1 << n)
    lib.oracle_apply_dense(int(n), int(nw), _ptr(u), st.shape[0], _ptr(st))
    return st


def hessian(n, gates, observables, params, data=None, batch=1, row_weights=None, lib=None):
    """(nparams, nparams) Hessian of sum_row sum_o w[row, o] E[row, o] with
    respect to the shared parameters, by the product rule (one forward run
    per pair of parameter occurrences -- small cases only)."""
    lib = lib or _load()
    g = _Gates(gates)
    o = _Obs(observables)
    params = np.ascontiguousarray(params, dtype=np.float64)
    nparams = params.size
    if data is not None:
        data = np.ascontiguousarray(data, dtype=np.float64).reshape(batch, -1)
        nfeat = data.shape[1]
    else:
        nfeat = 0
    rw = None
    if row_weights is not None:
        rw = np.ascontiguousarray(row_weights, dtype=np.float64).reshape(batch, o.nobs)
    out = np.zeros((nparams, nparams), dtype=np.float64)
    lib.oracle_hessian(int(n), g.count, _ptr(g.kind), _ptr(g.w0), _ptr(g.w1), _ptr(g.w2), _ptr(g.pidx),
                       _ptr(g.didx), _ptr(g.angle), _ptr(params), int(nparams), _ptr(data), int(nfeat),
                       int(batch), _ptr(o.coeff), _ptr(o.x), _ptr(o.z), _ptr(o.offsets), o.nobs, _ptr(rw),
                       _ptr(out))
    return out


def density(n, gates, observables=None, params=None, data=None, batch=1, lib=None):
    """Mixed-state evolution from |0><0| (gates and noise channels):
    (expectations (batch, nobs) or None, rho (batch, 2**n, 2**n) complex128)."""
    lib = lib or _load()
    g = _Gates(gates)
    params = np.ascontiguousarray(params, dtype=np.float64) if params is not None else np.zeros(1)
    if data is not None:
        data = np.ascontiguousarray(data, dtype=np.float64).reshape(batch, -1)
        nfeat = data.shape[1]
    else:
        nfeat = 0
    o = _Obs(observables or [])
    exp = np.empty((batch, o.nobs), dtype=np.float64) if observables else None
    rho = np.empty((batch, 1 << n, 1 << n), dtype=np.complex128)
    lib.oracle_density(int(n), g.count, _ptr(g.kind), _ptr(g.w0), _ptr(g.w1), _ptr(g.w2), _ptr(g.pidx),
                       _ptr(g.didx), _ptr(g.angle), _ptr(params), int(params.size), _ptr(data), int(nfeat),
                       int(batch), _ptr(o.coeff), _ptr(o.x), _ptr(o.z), _ptr(o.offsets), o.nobs, _ptr(exp),
                       _ptr(rho))
    return exp, rho


def sample(n, states, uniforms, wires=None, lib=None):
    """(batch, shots) int64 outcomes from |psi|^2 by inversion of the
    cumulative distribution, one per uniform in ``uniforms`` (batch, shots);
    ``wires``: packed bits of those wires (lowest wire most significant)."""
    lib = lib or _load()
    st = np.ascontiguousarray(states, dtype=np.complex128).reshape(-1, 1 << n)
    u = np.ascontiguousarray(uniforms, dtype=np.float64).reshape(st.shape[0], -1)
    mask = 0
    for q in (wires or []):
        mask |= 1 << int(q)
    out = np.empty(u.shape, dtype=np.int64)
    lib.oracle_sample(int(n), st.shape[0], _ptr(st), int(u.shape[1]), _ptr(u), ctypes.c_uint64(mask), _ptr(out))
    return out


def load_library(path: str):
    """Bind another build of the oracle (used to check that the pins reject
    deliberately mutated sources)."""
    return _bind(path)


def gate_block(kind: str, angle: float = 0.0, lib=None) -> np.ndarray:
    """The oracle's 2x2 target block for ``kind`` (complex128)."""
    out = np.empty(8, dtype=np.float64)
    (lib or _load()).oracle_gate_block(_KIND[kind], float(angle), _ptr(out))
    return (out[0::2] + 1j * out[1::2]).reshape(2, 2)
