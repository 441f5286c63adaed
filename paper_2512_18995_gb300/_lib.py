"""ctypes binding of libdq (include/dq.h).

Argument marshalling only: every step of the hot path runs in the CUDA
library.  PyTorch supplies device memory (states, parameters, outputs, the
workspace) and the current CUDA stream.  If ``libdq.so`` cannot be loaded the
import fails loudly; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from typing import Iterable, List, Optional, Sequence, Tuple

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
# DQ_DEBUG_BOUNDS=1 selects the bounds-checking build (build.build(debug=True))
LIB_PATH = os.path.join(_HERE, "libdq_debug.so" if os.environ.get("DQ_DEBUG_BOUNDS") == "1" else "libdq.so")

# dq_status
DQ_OK = 0
STATUS = {0: "DQ_OK", 1: "DQ_ERR_INVALID_ARG", 2: "DQ_ERR_UNSUPPORTED", 3: "DQ_ERR_OOM",
          4: "DQ_ERR_CUDA", 5: "DQ_ERR_TIMEOUT"}
DQ_C64, DQ_C128 = 0, 1
PATH_AUTO, PATH_PLAIN, PATH_FUSED = 0, 1, 2
OPT_MULTIPASS, OPT_WAIT_LIMIT_US, OPT_DENSE_BLOCKS, OPT_JIT, OPT_ROWS_PER_CTA = 1, 2, 3, 4, 5
ADJ_CLOBBER_STATE = 1

KIND = {k: i for i, k in enumerate(
    ["h", "x", "y", "z", "s", "rx", "ry", "rz", "cnot", "cz", "cp", "swap", "crx", "cry", "crz",
     "p", "u3", "rxx", "ryy", "rzz", "ccx", "bitflip", "phaseflip", "depolarizing", "ampdamp"])}
# consecutive angle slots a gate reads from params / data (U3: theta, phi, lam)
ANGLE_SPAN = {"u3": 3}


class DQError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class dq_gate(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("wires", ctypes.c_int32 * 3), ("param_idx", ctypes.c_int32),
                ("data_idx", ctypes.c_int32), ("angle", ctypes.c_double)]


class dq_circuit(ctypes.Structure):
    _fields_ = [("nqubits", ctypes.c_int32), ("ngates", ctypes.c_int32), ("gates", ctypes.POINTER(dq_gate)),
                ("nparams", ctypes.c_int32), ("nfeatures", ctypes.c_int32)]


class dq_pauli_term(ctypes.Structure):
    _fields_ = [("coeff", ctypes.c_double), ("xmask", ctypes.c_uint64), ("zmask", ctypes.c_uint64)]


class dq_observables(ctypes.Structure):
    _fields_ = [("nobs", ctypes.c_int32), ("term_offsets", ctypes.POINTER(ctypes.c_int32)),
                ("terms", ctypes.POINTER(dq_pauli_term))]


# kernel-level kinds of lowered circuits beyond the public ones (dq_lowered_op)
LOWERED_BLOCK, LOWERED_CBLOCK = 64, 65
KIND_NAME = {**{i: k for k, i in KIND.items()}, LOWERED_BLOCK: "block", LOWERED_CBLOCK: "cblock"}


class dq_lowered_op(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("wires", ctypes.c_int32 * 2), ("param_idx", ctypes.c_int32),
                ("data_idx", ctypes.c_int32), ("conj", ctypes.c_int32), ("angle", ctypes.c_double),
                ("block", ctypes.c_double * 8)]


EXPORTS = ("dq_ctx_create", "dq_ctx_destroy", "dq_last_error", "dq_ctx_set_path", "dq_ctx_set_option",
           "dq_state_norm", "dq_selftest_wait_expiry", "dq_selftest_bounds", "dq_plan_set_tile", "dq_batch_autotune", "dq_jit_source",
           "dq_jit_compile_check",
           "dq_ctx_set_workspace",
           "dq_workspace_bytes", "dq_batch_workspace_bytes", "dq_ctx_check", "dq_ctx_launch_count", "dq_ctx_set_graphs", "dq_ctx_set_tracing",
           "dq_ctx_trace_count", "dq_ctx_trace_get", "dq_state_init", "dq_apply_circuit",
           "dq_expect", "dq_adjoint_grad", "dq_forward_grad", "dq_forward_host", "dq_batch_forward_grad",
           "dq_plan_autotune",
           "dq_forward_grad_noalloc", "dq_apply_dense", "dq_sample_workspace_bytes", "dq_sample",
           "dq_hessian", "dq_density_workspace_bytes", "dq_density_forward",
           "dq_density_grad", "dq_plan_tuned", "dq_lower_circuit", "dq_tile_schedule", "dq_row_program",
           "dq_shift_rules")

_lib = None


def load_library(path: str = LIB_PATH):
    """Load libdq.so and declare the C signatures."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"libdq.so not found at {path}: build it with paper_2512_18995_gb300.build.build() "
                          "(there is no CPU fallback)")
    lib = ctypes.CDLL(path)
    P, I, D = ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_double)
    C = ctypes.POINTER(dq_circuit)
    O = ctypes.POINTER(dq_observables)
    sig = {
        "dq_ctx_create": ([ctypes.POINTER(P), I], I),
        "dq_ctx_destroy": ([P], I),
        "dq_last_error": ([P], ctypes.c_char_p),
        "dq_ctx_set_path": ([P, I], I),
        "dq_ctx_set_option": ([P, I, ctypes.c_int64], I),
        "dq_state_norm": ([P, I, P, I, I, P, P], I),
        "dq_jit_source": ([C, I, I, I, I, I, ctypes.c_char_p, ctypes.c_size_t, ctypes.POINTER(ctypes.c_size_t)], I),
        "dq_jit_compile_check": ([C, I, I, I, I, I, I, ctypes.c_char_p, ctypes.c_size_t], I),
        "dq_batch_autotune": ([P, I, C, P, ctypes.POINTER(ctypes.c_int64), O, I, P, P,
                               ctypes.POINTER(ctypes.c_int), P], I),
        "dq_selftest_wait_expiry": ([P, P], I),
        "dq_selftest_bounds": ([P, P], I),
        "dq_plan_set_tile": ([P, C, I, I, I, I, I], I),
        "dq_ctx_set_workspace": ([P, P, ctypes.c_size_t], I),
        "dq_workspace_bytes": ([P, C, O, I, I, ctypes.POINTER(ctypes.c_size_t)], I),
        "dq_batch_workspace_bytes": ([P, I, C, I, ctypes.POINTER(ctypes.c_size_t)], I),
        "dq_ctx_check": ([P, P], I),
        "dq_ctx_launch_count": ([P], ctypes.c_int64),
        "dq_ctx_set_graphs": ([P, I], I),
        "dq_ctx_set_tracing": ([P, I], I),
        "dq_ctx_trace_count": ([P], I),
        "dq_ctx_trace_get": ([P, I, ctypes.c_char_p, ctypes.c_size_t, ctypes.POINTER(ctypes.c_int64),
                              ctypes.POINTER(ctypes.c_double)], I),
        "dq_state_init": ([P, I, I, I, P, P], I),
        "dq_apply_circuit": ([P, C, P, I, P, P, I, I, P], I),
        "dq_expect": ([P, I, O, P, I, I, P, P], I),
        "dq_adjoint_grad": ([P, C, P, I, P, O, P, P, I, I, I, P, P, P], I),
        "dq_forward_grad": ([P, C, P, I, P, O, P, I, I, P, P, P, P, P], I),
        "dq_forward_host": ([P, C, P, O, I, I, P, P], I),
        "dq_batch_forward_grad": ([P, I, C, P, ctypes.POINTER(ctypes.c_int64), O, I, P, P, P], I),
        "dq_plan_autotune": ([P, C, I, I, P, P], I),
        "dq_forward_grad_noalloc": ([C, P, I, P, O, P, I, I, P, P, P, P, ctypes.c_char_p, ctypes.c_size_t], I),
        "dq_apply_dense": ([P, I, I, P, P, I, I, P], I),
        "dq_sample_workspace_bytes": ([P, I, I, ctypes.POINTER(ctypes.c_size_t)], I),
        "dq_hessian": ([P, C, P, P, O, P, I, I, ctypes.c_size_t, P, P, P], I),
        "dq_density_forward": ([P, C, P, P, O, I, I, P, P, P], I),
        "dq_density_workspace_bytes": ([P, C, I, I, ctypes.POINTER(ctypes.c_size_t)], I),
        "dq_density_grad": ([P, C, P, P, O, P, I, I, ctypes.c_size_t, P, P, P], I),
        "dq_plan_tuned": ([P, C, I, ctypes.POINTER(I), ctypes.POINTER(I), ctypes.POINTER(I)], I),
        "dq_sample": ([P, I, P, I, I, ctypes.c_int64, P, ctypes.c_uint64, ctypes.c_uint64, P, P], I),
        "dq_lower_circuit": ([C, I, ctypes.POINTER(dq_lowered_op), I, ctypes.POINTER(I)], I),
        "dq_tile_schedule": ([C, I, I, I, I, I, I, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32),
                              ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(I)], I),
        "dq_row_program": ([C, I, I, I, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32),
                            ctypes.POINTER(I), ctypes.POINTER(I)], I),
        "dq_shift_rules": ([C, I, I, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32), D, D,
                            ctypes.POINTER(I), ctypes.POINTER(I)], I),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    _lib = lib
    return lib


def _ptr(t: Optional[torch.Tensor]):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def dtype_code(dt: torch.dtype) -> int:
    if dt == torch.complex64:
        return DQ_C64
    if dt == torch.complex128:
        return DQ_C128
    raise TypeError(f"state dtype must be complex64 or complex128, got {dt}")


# ---------------------------------------------------------------------------
# tensor checks: the library receives bare device pointers and cannot see a
# buffer's device, type or size, so the binding checks them before a call
# ---------------------------------------------------------------------------
def _bad(msg: str):
    raise DQError(1, msg)


def _on_device(t, what: str, device: Optional[int]):
    if not isinstance(t, torch.Tensor) or t.device.type != "cuda":
        _bad(f"{what} must be a CUDA tensor")
    if device is not None and t.device.index != device:
        _bad(f"{what} is on cuda:{t.device.index}, the context on cuda:{device}")


def _f64_in(t: Optional[torch.Tensor], count: int, what: str, device: Optional[int]):
    """An FP64 input of which the call reads `count` values, converted to
    float64 and made contiguous (no-ops, same pointer, for tensors that
    already are); host tensors and short ones are rejected."""
    if t is None:
        return None
    _on_device(t, what, device)
    if t.dtype != torch.float64:
        t = t.to(torch.float64)
    t = t.contiguous()
    if t.numel() < count:
        _bad(f"{what} holds {t.numel()} values; the call reads {count}")
    return t


def _out(t: Optional[torch.Tensor], count: int, dtype: torch.dtype, what: str, device: Optional[int]):
    """A caller-supplied output buffer: `dtype`, contiguous, >= count values."""
    if t is None:
        return None
    _on_device(t, what, device)
    if t.dtype != dtype or not t.is_contiguous() or t.numel() < count:
        _bad(f"{what} must be a contiguous {dtype} tensor of at least {count} values")
    return t


def _state_rows(t: torch.Tensor, nqubits: int, what: str, device: Optional[int]) -> int:
    """Rows of a state batch tensor (contiguous complex rows of 2^nqubits)."""
    _on_device(t, what, device)
    dtype_code(t.dtype)
    if not t.is_contiguous():
        _bad(f"{what} must be contiguous")
    if 1 <= nqubits <= 34 and t.numel() % (1 << nqubits):
        _bad(f"{what} holds {t.numel()} amplitudes, not rows of 2^{nqubits}")
    return t.numel() >> nqubits if 0 <= nqubits < 63 else 0


def _angles(circuit, params, data, batch: int, params_per_row: bool, device: Optional[int]):
    """params and data of a call, checked against what the circuit reads."""
    params = _f64_in(params, circuit.nparams * (batch if params_per_row else 1), "params", device)
    data = _f64_in(data, batch * circuit.nfeatures, "data", device)
    return params, data


# ---------------------------------------------------------------------------
# circuit and observable descriptions
# ---------------------------------------------------------------------------
class Circuit:
    """A gate list in the C layout.  ``gates`` are objects with ``kind``,
    ``wires``, ``param``, ``data``, ``angle`` (e.g. ``workloads.Gate``) or
    tuples in that order."""

    def __init__(self, nqubits: int, gates: Sequence, nparams: Optional[int] = None,
                 nfeatures: Optional[int] = None):
        gl = list(gates)
        arr = (dq_gate * max(1, len(gl)))()
        maxp = maxd = -1
        for i, g in enumerate(gl):
            kind, wires, param, data, angle = (g.kind, g.wires, g.param, g.data, g.angle) \
                if hasattr(g, "kind") else tuple(g)
            arr[i].kind = KIND[kind] if isinstance(kind, str) else int(kind)
            for j in range(3):
                arr[i].wires[j] = int(wires[j]) if len(wires) > j else -1
            arr[i].param_idx = int(param)
            arr[i].data_idx = int(data)
            arr[i].angle = float(angle)
            span = ANGLE_SPAN.get(kind, 1) if isinstance(kind, str) else (3 if int(kind) == KIND["u3"] else 1)
            if int(param) >= 0:
                maxp = max(maxp, int(param) + span - 1)
            if int(data) >= 0:
                maxd = max(maxd, int(data) + span - 1)
        self.nqubits = int(nqubits)
        self.ngates = len(gl)
        self.nparams = int(nparams) if nparams is not None else maxp + 1
        self.nfeatures = int(nfeatures) if nfeatures is not None else maxd + 1
        self._arr = arr
        self.c = dq_circuit(self.nqubits, self.ngates, ctypes.cast(arr, ctypes.POINTER(dq_gate)),
                            self.nparams, self.nfeatures)

    def ref(self):
        return ctypes.byref(self.c)


class Observables:
    """``observables``: list of observables, each a list of
    ``(coeff, xmask, zmask)`` with bit q of a mask referring to wire q."""

    def __init__(self, observables: Sequence[Sequence[Tuple[float, int, int]]]):
        obs = [list(o) for o in observables]
        terms = [t for o in obs for t in o]
        self._terms = (dq_pauli_term * max(1, len(terms)))()
        for i, (c, x, z) in enumerate(terms):
            self._terms[i].coeff = float(c)
            self._terms[i].xmask = int(x)
            self._terms[i].zmask = int(z)
        offs = [0]
        for o in obs:
            offs.append(offs[-1] + len(o))
        self._offs = (ctypes.c_int32 * len(offs))(*offs)
        self.nobs = len(obs)
        self.c = dq_observables(self.nobs, ctypes.cast(self._offs, ctypes.POINTER(ctypes.c_int32)),
                                ctypes.cast(self._terms, ctypes.POINTER(dq_pauli_term)))

    def ref(self):
        return ctypes.byref(self.c)


# ---------------------------------------------------------------------------
# host-side plan inspection (no context, no GPU)
# ---------------------------------------------------------------------------
def _inspect_check(st: int, what: str):
    if st != DQ_OK:
        raise DQError(st, f"{what}: the circuit or arguments were rejected")


def lower_circuit(circuit: Circuit, density: bool = False) -> List[dict]:
    """The kernel-level ops the library runs for ``circuit`` (dq_lower_circuit):
    dicts with ``kind`` (name; "block"/"cblock" for fixed 2x2 blocks),
    ``wires``, ``param``, ``data``, ``angle``, ``conj`` and ``block`` (2x2
    complex, fixed blocks only)."""
    lib = load_library()
    cnt = ctypes.c_int(0)
    _inspect_check(lib.dq_lower_circuit(circuit.ref(), int(bool(density)), None, 0, ctypes.byref(cnt)),
                   "dq_lower_circuit")
    arr = (dq_lowered_op * max(1, cnt.value))()
    _inspect_check(lib.dq_lower_circuit(circuit.ref(), int(bool(density)), arr, cnt.value, ctypes.byref(cnt)),
                   "dq_lower_circuit")
    out = []
    for o in arr[:cnt.value]:
        w = tuple(int(x) for x in o.wires if x >= 0)
        b = None
        if o.kind in (LOWERED_BLOCK, LOWERED_CBLOCK):
            v = list(o.block)
            b = [[complex(v[0], v[1]), complex(v[2], v[3])], [complex(v[4], v[5]), complex(v[6], v[7])]]
        out.append({"kind": KIND_NAME[o.kind], "wires": w, "param": o.param_idx, "data": o.data_idx,
                    "angle": o.angle, "conj": bool(o.conj), "block": b})
    return out


# entry flags of dq_tile_schedule / dq_row_program
FLAG_PARITY_TRIPLE, FLAG_SWAP_CNOT = 1, 2


def tile_schedule(circuit: Circuit, k: int, low: int, M: int, dtype: int = DQ_C64,
                  adjoint: bool = False) -> List[Tuple[int, List[int], List[int]]]:
    """The fused path's tile passes for ``circuit`` (dq_tile_schedule): a list
    of (tile amplitude-bit mask, lowered-op index of every entry in execution
    order, entry flags FLAG_PARITY_TRIPLE / FLAG_SWAP_CNOT), or
    DQError(DQ_ERR_UNSUPPORTED) if no schedule exists for (k, low, M)."""
    lib = load_library()
    cnt = ctypes.c_int(0)
    _inspect_check(lib.dq_lower_circuit(circuit.ref(), 0, None, 0, ctypes.byref(cnt)), "dq_lower_circuit")
    cap = max(1, 3 * cnt.value)
    order = (ctypes.c_int32 * cap)()
    start = (ctypes.c_int32 * (cap + 1))()
    bits = (ctypes.c_uint64 * cap)()
    flags = (ctypes.c_int32 * cap)()
    npass = ctypes.c_int(0)
    _inspect_check(lib.dq_tile_schedule(circuit.ref(), int(dtype), int(k), int(low), int(M), int(bool(adjoint)),
                                        cap, order, start, bits, flags, ctypes.byref(npass)), "dq_tile_schedule")
    return [(int(bits[p]), [int(x) for x in order[start[p]:start[p + 1]]],
             [int(x) for x in flags[start[p]:start[p + 1]]]) for p in range(npass.value)]


JIT_FORWARD, JIT_REVERSE, JIT_ROWS = 0, 1, 2


def jit_source(circuit: Circuit, k: int, low: int, M: int, dtype: int = DQ_C64, adjoint: bool = False,
               kind: Optional[int] = None) -> str:
    """A run-time specialised program (dq_jit_source): the forward (or, with
    adjoint, reverse-sweep) passes of a tile schedule, one op runner and
    kernel per pass; or, with kind=JIT_ROWS, the whole-row kernel of the row
    program for M register bits (k and low ignored)."""
    lib = load_library()
    n = ctypes.c_size_t(0)
    a = int(bool(adjoint)) if kind is None else int(kind)
    _inspect_check(lib.dq_jit_source(circuit.ref(), int(dtype), int(k), int(low), int(M), a, None, 0,
                                     ctypes.byref(n)), "dq_jit_source")
    buf = ctypes.create_string_buffer(n.value + 1)
    _inspect_check(lib.dq_jit_source(circuit.ref(), int(dtype), int(k), int(low), int(M), a, buf, n.value + 1,
                                     ctypes.byref(n)), "dq_jit_source")
    return buf.value.decode()


def jit_compile_check(circuit: Circuit, k: int, low: int, M: int, dtype: int = DQ_C64, cc: int = 103,
                      adjoint: bool = False, kind: Optional[int] = None):
    """dq_jit_compile_check: (status, compiler log) of compiling the
    specialised program (as jit_source selects it) with NVRTC for compute
    capability cc (no device)."""
    lib = load_library()
    log = ctypes.create_string_buffer(4096)
    a = int(bool(adjoint)) if kind is None else int(kind)
    st = lib.dq_jit_compile_check(circuit.ref(), int(dtype), int(k), int(low), int(M), a, int(cc), log, 4096)
    return int(st), log.value.decode(errors="replace")


def row_program(circuit: Circuit, M: int = 0, dtype: int = DQ_C64) -> Tuple[int, List[int], List[int]]:
    """The whole-row kernel's program for ``circuit`` (dq_row_program):
    (register bits used, lowered-op index of every entry in execution order,
    entry flags as in tile_schedule)."""
    lib = load_library()
    cnt = ctypes.c_int(0)
    _inspect_check(lib.dq_lower_circuit(circuit.ref(), 0, None, 0, ctypes.byref(cnt)), "dq_lower_circuit")
    cap = max(1, 3 * cnt.value)
    order = (ctypes.c_int32 * cap)()
    flags = (ctypes.c_int32 * cap)()
    m = ctypes.c_int(0)
    _inspect_check(lib.dq_row_program(circuit.ref(), int(dtype), int(M), cap, order, flags, ctypes.byref(cnt),
                                      ctypes.byref(m)), "dq_row_program")
    return m.value, [int(x) for x in order[:cnt.value]], [int(x) for x in flags[:cnt.value]]


def shift_rules(circuit: Circuit):
    """The shift rules of dq_hessian / dq_density_grad (dq_shift_rules):
    (occurrence -> parameter, row offsets per occurrence (+1 entry), shifts,
    weights) as Python lists."""
    lib = load_library()
    nv, nj = ctypes.c_int(0), ctypes.c_int(0)
    _inspect_check(lib.dq_shift_rules(circuit.ref(), 0, 0, None, None, None, None, ctypes.byref(nv),
                                      ctypes.byref(nj)), "dq_shift_rules")
    occ = (ctypes.c_int32 * max(1, nv.value))()
    row0 = (ctypes.c_int32 * (nv.value + 1))()
    sh = (ctypes.c_double * max(1, nj.value))()
    wt = (ctypes.c_double * max(1, nj.value))()
    _inspect_check(lib.dq_shift_rules(circuit.ref(), nv.value, nj.value, occ, row0, sh, wt, ctypes.byref(nv),
                                      ctypes.byref(nj)), "dq_shift_rules")
    return (list(occ[:nv.value]), list(row0[:nv.value + 1]), list(sh[:nj.value]), list(wt[:nj.value]))


# ---------------------------------------------------------------------------
# context
# ---------------------------------------------------------------------------
class Context:
    """One libdq context on one CUDA device.  The workspace is a torch uint8
    tensor attached to the context and grown on demand."""

    def __init__(self, device: int = 0, path: int = PATH_AUTO):
        self.lib = load_library()
        self.device = int(device)
        h = ctypes.c_void_p()
        st = self.lib.dq_ctx_create(ctypes.byref(h), self.device)
        if st != DQ_OK:
            raise DQError(st, f"dq_ctx_create(device={device}) failed")
        self.h = h
        self._ws = None
        self._batch_arrays = None
        self.set_path(path)

    def close(self):
        if getattr(self, "h", None):
            self.lib.dq_ctx_destroy(self.h)
            self.h = None
            self._ws = None
            self._batch_arrays = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st: int, what: str):
        if st != DQ_OK:
            msg = self.lib.dq_last_error(self.h)
            raise DQError(st, f"{what}: {msg.decode() if msg else ''}")

    def set_path(self, path: int):
        self._check(self.lib.dq_ctx_set_path(self.h, int(path)), "dq_ctx_set_path")
        self.path = int(path)

    def set_option(self, option: int, value: int):
        """dq_ctx_set_option (OPT_MULTIPASS, OPT_WAIT_LIMIT_US, OPT_DENSE_BLOCKS, OPT_JIT, OPT_ROWS_PER_CTA)."""
        self._check(self.lib.dq_ctx_set_option(self.h, int(option), int(value)), "dq_ctx_set_option")

    def selftest_wait_expiry(self):
        """dq_selftest_wait_expiry: one bounded wait runs out on purpose; the
        next check() raises DQError(DQ_ERR_TIMEOUT)."""
        self._check(self.lib.dq_selftest_wait_expiry(self.h, _stream()), "dq_selftest_wait_expiry")

    def selftest_bounds(self):
        """dq_selftest_bounds (bounds-checking build only): one index check
        fails without touching memory; the next check() raises DQError
        (DQ_ERR_CUDA) naming it.  DQ_ERR_UNSUPPORTED in the normal build."""
        self._check(self.lib.dq_selftest_bounds(self.h, _stream()), "dq_selftest_bounds")

    def state_norm(self, state: torch.Tensor, nqubits: int, out: Optional[torch.Tensor] = None) -> torch.Tensor:
        """<psi|psi> of every row (FP64 accumulation), shape (batch,)."""
        batch = _state_rows(state, nqubits, "state", self.device)
        out = _out(out, batch, torch.float64, "out", self.device)
        if out is None:
            out = torch.empty(batch, dtype=torch.float64, device=f"cuda:{self.device}")
        self._check(self.lib.dq_state_norm(self.h, int(nqubits), _ptr(state), int(batch), dtype_code(state.dtype),
                                           _ptr(out), _stream()), "dq_state_norm")
        return out

    @property
    def launch_count(self) -> int:
        return int(self.lib.dq_ctx_launch_count(self.h))

    def check(self):
        self._check(self.lib.dq_ctx_check(self.h, _stream()), "dq_ctx_check")

    def set_graphs(self, on: bool):
        """CUDA-graph replay of repeated identical calls (see dq_ctx_set_graphs)."""
        self._check(self.lib.dq_ctx_set_graphs(self.h, int(bool(on))), "dq_ctx_set_graphs")

    def set_tracing(self, on: bool):
        self._check(self.lib.dq_ctx_set_tracing(self.h, int(bool(on))), "dq_ctx_set_tracing")

    def trace(self):
        """{kernel name: (launches, total device ms)} since tracing was turned on."""
        n = self.lib.dq_ctx_trace_count(self.h)
        if n < 0:
            raise DQError(4, "dq_ctx_trace_count failed")
        out = {}
        buf = ctypes.create_string_buffer(128)
        for i in range(n):
            cnt = ctypes.c_int64(0)
            ms = ctypes.c_double(0.0)
            self._check(self.lib.dq_ctx_trace_get(self.h, i, buf, 128, ctypes.byref(cnt), ctypes.byref(ms)),
                        "dq_ctx_trace_get")
            out[buf.value.decode()] = (int(cnt.value), float(ms.value))
        return out

    def release_workspace(self):
        """Detach and free the workspace tensor (the next call allocates again)."""
        torch.cuda.synchronize(self.device)
        self._check(self.lib.dq_ctx_set_workspace(self.h, None, 0), "dq_ctx_set_workspace")
        self._ws = None

    def ensure_workspace(self, circuit: Optional[Circuit], obs: Optional[Observables], batch: int, dtype: int,
                         need_bytes: Optional[int] = None):
        if need_bytes is None:
            if circuit is None:
                circuit = Circuit(1, [])
            need = ctypes.c_size_t(0)
            self._check(self.lib.dq_workspace_bytes(self.h, circuit.ref(), obs.ref() if obs else None, int(batch),
                                                    int(dtype), ctypes.byref(need)), "dq_workspace_bytes")
        else:
            need = ctypes.c_size_t(int(need_bytes))
        if self._ws is None or self._ws.numel() < need.value:
            self._ws = None
            self._check(self.lib.dq_ctx_set_workspace(self.h, None, 0), "dq_ctx_set_workspace")
            size = max(int(need.value), 1 << 20)
            self._ws = torch.empty(size, dtype=torch.uint8, device=f"cuda:{self.device}")
            self._check(self.lib.dq_ctx_set_workspace(self.h, _ptr(self._ws), size), "dq_ctx_set_workspace")

    # ---- hot path --------------------------------------------------------
    def state_init(self, state: torch.Tensor, nqubits: int):
        batch = _state_rows(state, nqubits, "state", self.device)
        self._check(self.lib.dq_state_init(self.h, int(nqubits), int(batch), dtype_code(state.dtype), _ptr(state),
                                           _stream()), "dq_state_init")

    def apply_circuit(self, circuit: Circuit, params: Optional[torch.Tensor], state: torch.Tensor,
                      data: Optional[torch.Tensor] = None, params_per_row: bool = False):
        batch = _state_rows(state, circuit.nqubits, "state", self.device)
        dt = dtype_code(state.dtype)
        params, data = _angles(circuit, params, data, batch, params_per_row, self.device)
        self.ensure_workspace(circuit, None, batch, dt)
        self._check(self.lib.dq_apply_circuit(self.h, circuit.ref(), _ptr(params), int(params_per_row), _ptr(data),
                                              _ptr(state), int(batch), dt, _stream()), "dq_apply_circuit")

    def apply_dense(self, nqubits: int, unitary: torch.Tensor, state: torch.Tensor):
        """Dense 2^nw x 2^nw unitary (complex128, on the device) on the nw
        lowest-order qubits of every row of a complex64 state, in place, on
        the tensor cores."""
        nw = int(unitary.shape[-1]).bit_length() - 1
        if unitary.dtype != torch.complex128 or tuple(unitary.shape) != (1 << nw, 1 << nw):
            raise ValueError("unitary must be a complex128 tensor of shape (2^nw, 2^nw)")
        _on_device(unitary, "unitary", self.device)
        u = unitary.contiguous()
        batch = _state_rows(state, nqubits, "state", self.device)
        self.ensure_workspace(None, None, batch, dtype_code(state.dtype), need_bytes=1 << 20)
        self._check(self.lib.dq_apply_dense(self.h, int(nqubits), nw, _ptr(u), _ptr(state), int(batch),
                                            dtype_code(state.dtype), _stream()), "dq_apply_dense")

    def density_forward(self, circuit: Circuit, params: Optional[torch.Tensor], obs: Optional[Observables],
                        batch: int = 1, dtype: torch.dtype = torch.complex64, data: Optional[torch.Tensor] = None,
                        want_rho: bool = False, rho: Optional[torch.Tensor] = None):
        """Mixed-state evolution from |0><0| with the circuit's gates and
        noise channels: (expectations (batch, nobs) FP64 or None, rho
        (batch, 2^n, 2^n) or None)."""
        n = circuit.nqubits
        dev = torch.device(f"cuda:{self.device}")
        params, data = _angles(circuit, params, data, batch, False, self.device)
        if rho is not None:
            rho = _out(rho, batch << (2 * n) if 1 <= n <= 17 else 0, dtype, "rho", self.device)
        if want_rho and rho is None:
            rho = torch.empty((batch, 1 << n, 1 << n), dtype=dtype, device=dev)
        expect = torch.empty((batch, obs.nobs), dtype=torch.float64, device=dev) if obs is not None else None
        need = ctypes.c_size_t(0)
        self._check(self.lib.dq_density_workspace_bytes(self.h, circuit.ref(), int(batch), dtype_code(dtype),
                                                        ctypes.byref(need)), "dq_density_workspace_bytes")
        self.ensure_workspace(None, None, int(batch), dtype_code(dtype), need_bytes=need.value)
        self._check(self.lib.dq_density_forward(self.h, circuit.ref(), _ptr(params), _ptr(data),
                                                obs.ref() if obs is not None else None, int(batch),
                                                dtype_code(dtype), _ptr(expect), _ptr(rho), _stream()),
                    "dq_density_forward")
        return expect, rho

    def density_grad(self, circuit: Circuit, params: torch.Tensor, obs: Observables,
                     data: Optional[torch.Tensor] = None, row_weights: Optional[torch.Tensor] = None,
                     dtype: torch.dtype = torch.complex64, max_bytes: int = 0):
        """(expectations (batch, nobs), gradient (nparams,)) of a density
        circuit's weighted expectation sum, by exact shift rules."""
        batch = int(data.shape[0]) if data is not None else 1
        dev = torch.device(f"cuda:{self.device}")
        params, data = _angles(circuit, params, data, batch, False, self.device)
        row_weights = _f64_in(row_weights, batch * obs.nobs, "row_weights", self.device)
        expect = torch.empty((batch, obs.nobs), dtype=torch.float64, device=dev)
        grad = torch.empty((circuit.nparams,), dtype=torch.float64, device=dev)
        if self._ws is not None:   # scratch is sized inside the call
            self.release_workspace()
        self._check(self.lib.dq_density_grad(self.h, circuit.ref(), _ptr(params), _ptr(data),
                                             obs.ref(), _ptr(row_weights), batch, dtype_code(dtype),
                                             ctypes.c_size_t(int(max_bytes)), _ptr(expect), _ptr(grad), _stream()),
                    "dq_density_grad")
        return expect, grad

    def hessian(self, circuit: Circuit, params: torch.Tensor, obs: Observables, data: Optional[torch.Tensor] = None,
                row_weights: Optional[torch.Tensor] = None, dtype: torch.dtype = torch.complex64,
                want_grad: bool = True, max_bytes: int = 0):
        """(hess (nparams, nparams), grad (nparams,) or None) of the weighted
        sum of expectations over the data rows (batch = data rows, or 1).
        ``max_bytes`` bounds the shifted rows' state memory per chunk (0: a
        quarter of the free device memory)."""
        batch = int(data.shape[0]) if data is not None else 1
        dev = torch.device(f"cuda:{self.device}")
        P = circuit.nparams
        params, data = _angles(circuit, params, data, batch, False, self.device)
        row_weights = _f64_in(row_weights, batch * obs.nobs, "row_weights", self.device)
        # the shifted rows' scratch is sized inside the call: let the context
        # grow its own workspace instead of an attached tensor
        if self._ws is not None:
            self.release_workspace()
        hess = torch.empty((P, P), dtype=torch.float64, device=dev)
        grad = torch.empty((P,), dtype=torch.float64, device=dev) if want_grad else None
        self._check(self.lib.dq_hessian(self.h, circuit.ref(), _ptr(params), _ptr(data),
                                        obs.ref(), _ptr(row_weights), batch, dtype_code(dtype),
                                        ctypes.c_size_t(int(max_bytes)), _ptr(hess),
                                        _ptr(grad), _stream()), "dq_hessian")
        return hess, grad

    def sample(self, nqubits: int, state: torch.Tensor, shots: int, uniforms: Optional[torch.Tensor] = None,
               seed: int = 0, wires: Optional[Sequence[int]] = None,
               out: Optional[torch.Tensor] = None) -> torch.Tensor:
        """Outcomes (batch, shots) int64 drawn from |psi|^2 of every row:
        basis indices, or the packed bits of ``wires`` (first listed wire =
        most significant; the wires are taken in increasing order).
        ``uniforms`` (FP64 (batch, shots) on the device, in [0, 1)) or, when
        None, the splitmix64 stream of ``seed`` drives the draws."""
        batch = _state_rows(state, nqubits, "state", self.device)
        mask = 0
        if wires is not None:
            for q in wires:
                mask |= 1 << int(q)
        if out is None:
            out = torch.empty((batch, int(shots)), dtype=torch.int64, device=state.device)
        else:
            out = _out(out, batch * int(shots), torch.int64, "out", self.device)
        need = ctypes.c_size_t(0)
        self._check(self.lib.dq_sample_workspace_bytes(self.h, int(nqubits), int(batch), ctypes.byref(need)),
                    "dq_sample_workspace_bytes")
        self.ensure_workspace(None, None, batch, dtype_code(state.dtype), need_bytes=need.value)
        u = None
        if uniforms is not None:
            if uniforms.numel() != batch * int(shots):
                raise ValueError("uniforms must hold batch * shots values")
            u = _f64_in(uniforms, batch * int(shots), "uniforms", self.device)
        self._check(self.lib.dq_sample(self.h, int(nqubits), _ptr(state), int(batch), dtype_code(state.dtype),
                                       int(shots), _ptr(u), ctypes.c_uint64(int(seed) & (2 ** 64 - 1)),
                                       ctypes.c_uint64(mask), _ptr(out), _stream()), "dq_sample")
        return out

    def expect(self, nqubits: int, obs: Observables, state: torch.Tensor,
               out: Optional[torch.Tensor] = None) -> torch.Tensor:
        batch = _state_rows(state, nqubits, "state", self.device)
        dt = dtype_code(state.dtype)
        if out is None:
            out = torch.empty((batch, obs.nobs), dtype=torch.float64, device=state.device)
        else:
            out = _out(out, batch * obs.nobs, torch.float64, "out", self.device)
        self.ensure_workspace(Circuit(nqubits, []), obs, batch, dt)
        self._check(self.lib.dq_expect(self.h, int(nqubits), obs.ref(), _ptr(state), int(batch), dt, _ptr(out),
                                       _stream()), "dq_expect")
        return out

    def adjoint_grad(self, circuit: Circuit, params: Optional[torch.Tensor], obs: Observables,
                     state: torch.Tensor, data: Optional[torch.Tensor] = None,
                     row_weights: Optional[torch.Tensor] = None, params_per_row: bool = False,
                     clobber: bool = False, grad_params: Optional[torch.Tensor] = None,
                     grad_data: Optional[torch.Tensor] = None):
        batch = _state_rows(state, circuit.nqubits, "state", self.device)
        dt = dtype_code(state.dtype)
        dev = state.device
        params, data = _angles(circuit, params, data, batch, params_per_row, self.device)
        row_weights = _f64_in(row_weights, batch * obs.nobs, "row_weights", self.device)
        grad_params = _out(grad_params, circuit.nparams * (batch if params_per_row else 1), torch.float64,
                           "grad_params", self.device)
        grad_data = _out(grad_data, batch * circuit.nfeatures, torch.float64, "grad_data", self.device)
        if grad_params is None and circuit.nparams > 0:
            shape = (batch, circuit.nparams) if params_per_row else (circuit.nparams,)
            grad_params = torch.empty(shape, dtype=torch.float64, device=dev)
        if grad_data is None and circuit.nfeatures > 0 and data is not None:
            grad_data = torch.empty((batch, circuit.nfeatures), dtype=torch.float64, device=dev)
        self.ensure_workspace(circuit, obs, batch, dt)
        self._check(self.lib.dq_adjoint_grad(self.h, circuit.ref(), _ptr(params), int(params_per_row), _ptr(data),
                                             obs.ref(), _ptr(row_weights), _ptr(state), int(batch), dt,
                                             ADJ_CLOBBER_STATE if clobber else 0, _ptr(grad_params),
                                             _ptr(grad_data), _stream()), "dq_adjoint_grad")
        return grad_params, grad_data

    def forward_grad(self, circuit: Circuit, params: Optional[torch.Tensor], obs: Optional[Observables],
                     batch: int, dtype: torch.dtype = torch.complex64, data: Optional[torch.Tensor] = None,
                     row_weights: Optional[torch.Tensor] = None, params_per_row: bool = False,
                     want_expect: bool = True, want_grad: bool = True, state_out: Optional[torch.Tensor] = None,
                     expect_out: Optional[torch.Tensor] = None, grad_params: Optional[torch.Tensor] = None,
                     grad_data: Optional[torch.Tensor] = None, want_data_grad: bool = True):
        dt = dtype_code(dtype)
        dev = torch.device(f"cuda:{self.device}")
        params, data = _angles(circuit, params, data, batch, params_per_row, self.device)
        nobs = obs.nobs if obs is not None else 0
        row_weights = _f64_in(row_weights, batch * nobs, "row_weights", self.device)
        expect_out = _out(expect_out, batch * nobs, torch.float64, "expect_out", self.device)
        grad_params = _out(grad_params, circuit.nparams * (batch if params_per_row else 1), torch.float64,
                           "grad_params", self.device)
        grad_data = _out(grad_data, batch * circuit.nfeatures, torch.float64, "grad_data", self.device)
        if state_out is not None:
            n = circuit.nqubits
            state_out = _out(state_out, batch << n if 1 <= n <= 34 else 0, dtype, "state_out", self.device)
        if want_expect and expect_out is None and obs is not None:
            expect_out = torch.empty((batch, obs.nobs), dtype=torch.float64, device=dev)
        if want_grad:
            if grad_params is None and circuit.nparams > 0:
                shape = (batch, circuit.nparams) if params_per_row else (circuit.nparams,)
                grad_params = torch.empty(shape, dtype=torch.float64, device=dev)
            if grad_data is None and circuit.nfeatures > 0 and data is not None and want_data_grad:
                grad_data = torch.empty((batch, circuit.nfeatures), dtype=torch.float64, device=dev)
        else:
            grad_params = grad_data = None
        self.ensure_workspace(circuit, obs, batch, dt)
        self._check(self.lib.dq_forward_grad(self.h, circuit.ref(), _ptr(params), int(params_per_row), _ptr(data),
                                             obs.ref() if obs is not None else None, _ptr(row_weights), int(batch),
                                             dt, _ptr(expect_out), _ptr(grad_params), _ptr(grad_data),
                                             _ptr(state_out), _stream()), "dq_forward_grad")
        return expect_out, grad_params, grad_data, state_out

    def forward_host(self, circuit: Circuit, params: Optional[torch.Tensor], obs: Observables, batch: int,
                     dtype: torch.dtype = torch.complex64, expect_out: Optional[torch.Tensor] = None):
        """dq_forward_host: the forward path with host buffers.  params and
        expect_out are CPU float64 tensors (pinned ones let the copies join
        the call's CUDA graph); returns expect_out, filled when the call
        returns."""
        def host(t, count, what):
            if not isinstance(t, torch.Tensor) or t.device.type != "cpu" or t.dtype != torch.float64 \
                    or not t.is_contiguous() or t.numel() < count:
                _bad(f"{what} must be a contiguous CPU float64 tensor of at least {count} values")
            return t
        if params is not None:
            params = host(params, circuit.nparams, "params")
        if expect_out is None:
            expect_out = torch.empty((batch, obs.nobs), dtype=torch.float64).pin_memory()
        expect_out = host(expect_out, batch * obs.nobs, "expect_out")
        dt = dtype_code(dtype)
        self.ensure_workspace(circuit, obs, batch, dt)
        self._check(self.lib.dq_forward_host(self.h, circuit.ref(), _ptr(params), obs.ref(), int(batch), dt,
                                             _ptr(expect_out), _stream()), "dq_forward_host")
        return expect_out

    def batch_autotune(self, circuits: Sequence[Circuit], params: torch.Tensor, obs: Observables,
                       dtype: torch.dtype = torch.complex64):
        """dq_batch_autotune: tune the uneven-batch launch for this batch;
        returns (qubits in shared memory, threads per circuit, CTAs per SM,
        MiB of scratch in flight for the larger circuits, 0: every CTA)."""
        choice = (ctypes.c_int * 4)()
        self.batch_forward_grad(circuits, params, obs, dtype, _tune_choice=choice)
        return tuple(int(x) for x in choice)

    def batch_forward_grad(self, circuits: Sequence[Circuit], params: torch.Tensor, obs: Observables,
                           dtype: torch.dtype = torch.complex64, want_grad: bool = True,
                           expect_out: Optional[torch.Tensor] = None, grad_params: Optional[torch.Tensor] = None,
                           _tune_choice=None):
        nc = len(circuits)
        # the C arrays of the batch, reused while the call passes the same
        # Circuit objects in the same order (held here, so their ids stay theirs)
        cached = self._batch_arrays
        if cached is not None and len(cached[0]) == nc and all(a is b for a, b in zip(cached[0], circuits)):
            arr, offs = cached[1], cached[2]
        else:
            arr = (dq_circuit * max(1, nc))()
            offs = (ctypes.c_int64 * (nc + 1))()
            for i, c in enumerate(circuits):
                arr[i] = c.c
                offs[i + 1] = offs[i] + c.nparams
            self._batch_arrays = (tuple(circuits), arr, offs)
        dev = torch.device(f"cuda:{self.device}")
        params = _f64_in(params, int(offs[nc]), "params", self.device)
        expect_out = _out(expect_out, nc * obs.nobs, torch.float64, "expect_out", self.device)
        grad_params = _out(grad_params, int(offs[nc]), torch.float64, "grad_params", self.device)
        if expect_out is None:
            expect_out = torch.empty((nc, obs.nobs), dtype=torch.float64, device=dev)
        if want_grad and grad_params is None:
            grad_params = torch.empty(max(1, int(offs[nc])), dtype=torch.float64, device=dev)
        if not want_grad:
            grad_params = None
        self._keep = (arr, offs)
        need = ctypes.c_size_t(0)
        self._check(self.lib.dq_batch_workspace_bytes(self.h, nc, ctypes.cast(arr, ctypes.POINTER(dq_circuit)),
                                                      dtype_code(dtype), ctypes.byref(need)),
                    "dq_batch_workspace_bytes")
        self.ensure_workspace(None, None, 0, dtype_code(dtype), need_bytes=need.value)
        if _tune_choice is not None:
            self._check(self.lib.dq_batch_autotune(self.h, nc, ctypes.cast(arr, ctypes.POINTER(dq_circuit)),
                                                   _ptr(params), offs, obs.ref(), dtype_code(dtype),
                                                   _ptr(expect_out), _ptr(grad_params), _tune_choice, _stream()),
                        "dq_batch_autotune")
        else:
            self._check(self.lib.dq_batch_forward_grad(self.h, nc, ctypes.cast(arr, ctypes.POINTER(dq_circuit)),
                                                       _ptr(params), offs, obs.ref(), dtype_code(dtype),
                                                       _ptr(expect_out), _ptr(grad_params), _stream()),
                        "dq_batch_forward_grad")
        return expect_out, grad_params

    def plan_tuned(self, circuit: Circuit, dtype: torch.dtype = torch.complex64):
        """(k, low, M) chosen by plan_autotune for this circuit, or zeros."""
        k, low, m = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_int(0)
        self._check(self.lib.dq_plan_tuned(self.h, circuit.ref(), dtype_code(dtype), ctypes.byref(k),
                                           ctypes.byref(low), ctypes.byref(m)), "dq_plan_tuned")
        return k.value, low.value, m.value

    def plan_set_tile(self, circuit: Circuit, k: int, low: int, M: int, jit: bool = True,
                      dtype: torch.dtype = torch.complex64):
        """dq_plan_set_tile: pin the forward tile shape (and the specialised
        passes) for this circuit structure without tuning."""
        self._check(self.lib.dq_plan_set_tile(self.h, circuit.ref(), dtype_code(dtype), int(k), int(low), int(M),
                                              int(bool(jit))), "dq_plan_set_tile")

    def plan_autotune(self, circuit: Circuit, state: torch.Tensor):
        batch = _state_rows(state, circuit.nqubits, "state", self.device)
        dt = dtype_code(state.dtype)
        self.ensure_workspace(circuit, None, batch, dt)
        self._check(self.lib.dq_plan_autotune(self.h, circuit.ref(), int(batch), dt, _ptr(state), _stream()),
                    "dq_plan_autotune")


def forward_grad_noalloc(circuit: Circuit, params: Optional[torch.Tensor], obs: Observables, batch: int,
                         dtype: torch.dtype = torch.complex64, data: Optional[torch.Tensor] = None,
                         row_weights: Optional[torch.Tensor] = None, params_per_row: bool = False,
                         expect_out: Optional[torch.Tensor] = None, grad_params: Optional[torch.Tensor] = None,
                         grad_data: Optional[torch.Tensor] = None):
    """Call dq_forward_grad_noalloc: the whole on-chip hot path without any
    device allocation inside the library (scratch is a static device array).
    Output tensors are supplied by the caller (allocated here if None)."""
    lib = load_library()
    dev = torch.device("cuda", torch.cuda.current_device())
    params, data = _angles(circuit, params, data, batch, params_per_row, dev.index)
    row_weights = _f64_in(row_weights, batch * obs.nobs, "row_weights", dev.index)
    expect_out = _out(expect_out, batch * obs.nobs, torch.float64, "expect_out", dev.index)
    grad_params = _out(grad_params, circuit.nparams * (batch if params_per_row else 1), torch.float64,
                       "grad_params", dev.index)
    grad_data = _out(grad_data, batch * circuit.nfeatures, torch.float64, "grad_data", dev.index)
    if expect_out is None:
        expect_out = torch.empty((batch, obs.nobs), dtype=torch.float64, device=dev)
    if grad_params is None and circuit.nparams > 0:
        shape = (batch, circuit.nparams) if params_per_row else (circuit.nparams,)
        grad_params = torch.empty(shape, dtype=torch.float64, device=dev)
    if grad_data is None and circuit.nfeatures > 0 and data is not None:
        grad_data = torch.empty((batch, circuit.nfeatures), dtype=torch.float64, device=dev)
    err = ctypes.create_string_buffer(256)
    st = lib.dq_forward_grad_noalloc(circuit.ref(), _ptr(params), int(params_per_row), _ptr(data), obs.ref(),
                                     _ptr(row_weights), int(batch), dtype_code(dtype), _ptr(expect_out),
                                     _ptr(grad_params), _ptr(grad_data), _stream(), err, 256)
    if st != DQ_OK:
        raise DQError(st, f"dq_forward_grad_noalloc: {err.value.decode()}")
    return expect_out, grad_params, grad_data
