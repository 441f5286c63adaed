"""CPU-only checks of the C ABI library and the input generators (no GPU
compute: loading, exported symbols, struct layouts, host-side validation
reachable without a device)."""
import ctypes
import os
import re
import subprocess
import tempfile

import numpy as np
import pytest

import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "dq.h")


@pytest.fixture(scope="module")
def libdq():
    from paper_2512_18995_gb300 import build
    build.build()
    from paper_2512_18995_gb300 import _lib
    return _lib.load_library()


def declared_symbols():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^DQ_API\s+[\w\s\*]+?\b(dq_\w+)\s*\(", text, flags=re.M)))


def test_header_declares_the_boundary():
    names = declared_symbols()
    for required in ("dq_state_init", "dq_apply_circuit", "dq_expect", "dq_adjoint_grad"):
        assert required in names
    assert len(names) >= 15


def test_library_exports_every_declared_symbol(libdq):
    out = subprocess.run(["nm", "-D", "--defined-only", libdq._name], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (dq_\w+)", out))
    missing = [s for s in declared_symbols() if s not in exported]
    assert not missing, missing
    for s in declared_symbols():
        assert hasattr(libdq, s)


def test_binding_exports_list_matches_header():
    from paper_2512_18995_gb300 import _lib
    assert sorted(_lib.EXPORTS) == declared_symbols()


def test_struct_layouts_match_header():
    """Compile a probe against dq.h and compare sizes/offsets with ctypes."""
    from paper_2512_18995_gb300 import _lib
    src = r'''
#include <stdio.h>
#include <stddef.h>
#include "dq.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu\n", sizeof(dq_gate), offsetof(dq_gate, angle), offsetof(dq_gate, param_idx),
         sizeof(dq_circuit), offsetof(dq_circuit, gates), offsetof(dq_circuit, nfeatures));
  printf("%zu %zu %zu %zu\n", sizeof(dq_pauli_term), sizeof(dq_observables),
         offsetof(dq_observables, term_offsets), offsetof(dq_observables, terms));
  printf("%d %d %d %d\n", (int)DQ_CRZ, (int)DQ_SWAP, (int)DQ_NUM_GATE_KINDS, (int)DQ_ERR_TIMEOUT);
  printf("%zu %zu %zu %zu %d %d\n", sizeof(dq_lowered_op), offsetof(dq_lowered_op, conj),
         offsetof(dq_lowered_op, angle), offsetof(dq_lowered_op, block), DQ_LOWERED_BLOCK, DQ_LOWERED_CBLOCK);
  return 0;
}
'''
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "probe.c")
        exe = os.path.join(d, "probe")
        open(c, "w").write(src)
        subprocess.check_call(["gcc", "-std=c11", "-I", os.path.dirname(HEADER), c, "-o", exe])
        lines = subprocess.check_output([exe], text=True).split("\n")
    a = list(map(int, lines[0].split()))
    assert a == [ctypes.sizeof(_lib.dq_gate), _lib.dq_gate.angle.offset, _lib.dq_gate.param_idx.offset,
                 ctypes.sizeof(_lib.dq_circuit), _lib.dq_circuit.gates.offset, _lib.dq_circuit.nfeatures.offset]
    b = list(map(int, lines[1].split()))
    assert b == [ctypes.sizeof(_lib.dq_pauli_term), ctypes.sizeof(_lib.dq_observables),
                 _lib.dq_observables.term_offsets.offset, _lib.dq_observables.terms.offset]
    k = list(map(int, lines[2].split()))
    assert k == [_lib.KIND["crz"], _lib.KIND["swap"], len(_lib.KIND), 5]
    lo = list(map(int, lines[3].split()))
    assert lo == [ctypes.sizeof(_lib.dq_lowered_op), _lib.dq_lowered_op.conj.offset, _lib.dq_lowered_op.angle.offset,
                  _lib.dq_lowered_op.block.offset, _lib.LOWERED_BLOCK, _lib.LOWERED_CBLOCK]


def test_context_creation_fails_cleanly_without_device(libdq):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    st = libdq.dq_ctx_create(ctypes.byref(h), 0)
    assert st != 0 and not h.value
    assert libdq.dq_ctx_launch_count(None) == 0


def test_null_context_is_rejected(libdq):
    from paper_2512_18995_gb300 import _lib
    c = _lib.Circuit(2, [W.Gate("h", (0,))])
    st = libdq.dq_apply_circuit(None, c.ref(), None, 0, None, None, 1, 0, None)
    assert st == 1   # DQ_ERR_INVALID_ARG
    assert libdq.dq_forward_host(None, c.ref(), None, None, 1, 0, None, None) == 1



def test_noalloc_entry_point_checks_arguments_before_the_device(libdq):
    """dq_forward_grad_noalloc validates every host argument before it
    touches the device, so these rejections need no GPU."""
    from paper_2512_18995_gb300 import _lib
    err = ctypes.create_string_buffer(128)
    c = _lib.Circuit(3, [W.Gate("ry", (0,), param=0), W.Gate("rx", (1,), data=0)], nparams=1, nfeatures=1)
    obs = _lib.Observables([W.obs_z(0)])
    fake = ctypes.c_void_p(0x1000)     # never dereferenced: the calls fail first

    def call(circ=c, params=fake, data=fake, o=obs, batch=2, dtype=0):
        return libdq.dq_forward_grad_noalloc(circ.ref() if circ is not None else None, params, 0, data,
                                             o.ref() if o is not None else None, None, batch, dtype,
                                             fake, None, None, None, err, 128)

    assert call(circ=None) == 1 and b"circuit" in err.value
    assert call(dtype=7) == 1 and b"dtype" in err.value
    assert call(batch=-1) == 1
    assert call(params=None) == 1 and b"params" in err.value
    assert call(data=None) == 1 and b"data" in err.value
    assert call(o=None) == 1 and b"observables" in err.value
    bad = _lib.Observables([W.obs_z(0)])
    bad.c.terms = ctypes.POINTER(_lib.dq_pauli_term)()        # NULL terms behind one term offset
    assert call(o=bad) == 1 and b"terms is NULL" in err.value
    wide = _lib.Observables([W.obs_z(5)])                     # a wire beyond the circuit
    assert call(o=wide) == 1 and b"wire" in err.value
    assert call(circ=_lib.Circuit(3, [W.Gate("h", (3,))])) == 1

# ---------------------------------------------------------------------------
# input generators
# ---------------------------------------------------------------------------
def test_splitmix64_reference_value():
    # First output of splitmix64 seeded with 0 (the generator's published
    # reference stream).
    assert W.SplitMix64(0).next_u64() == 0xE220A8397B1DCDAF


def test_uniform_ranges_and_determinism():
    a = W.uniform_array(7, 1000, -np.pi, np.pi)
    b = W.uniform_array(7, 1000, -np.pi, np.pi)
    assert np.array_equal(a, b)
    assert a.min() >= -np.pi and a.max() < np.pi
    assert abs(a.mean()) < 0.3


def test_config_shapes():
    c1, c2, c3, c5 = W.config_c1(), W.config_c2(), W.config_c3(), W.config_c5()
    assert (c1.n, len(c1.gates), c1.nparams) == (10, 120, 80)
    assert (c2.n, len(c2.gates), c2.nparams) == (20, 480, 320)
    assert (c3.n, len(c3.gates), c3.nparams, c3.data.shape) == (12, 228, 144, (4096, 12))
    assert (c5.n, len(c5.gates), c5.nparams) == (30, 1380, 600)
    assert np.all((c1.params >= 0) & (c1.params < 2 * np.pi))
    assert np.all((c3.data >= -np.pi) & (c3.data < np.pi))
    qft = W.qft_gates(30)
    assert sum(g.kind == "h" for g in qft) == 30
    assert sum(g.kind == "cp" for g in qft) == 435
    assert sum(g.kind == "swap" for g in qft) == 15


def test_uneven_batch_generator():
    circs = W.config_c4(1024)
    ns = np.array([c[0] for c in circs])
    ds = np.array([len(c[1]) for c in circs])
    assert ns.min() == 8 and ns.max() == 16
    assert ds.min() >= 10 and ds.max() <= 40
    kinds = {g.kind for c in circs for g in c[1]}
    assert kinds == {"h", "rx", "ry", "rz", "cnot", "cz"}
    for n, gates, angles in circs[:50]:
        for g in gates:
            assert all(0 <= w < n for w in g.wires)
            if len(g.wires) == 2:
                assert g.wires[0] != g.wires[1]
        assert len(angles) == sum(g.param >= 0 for g in gates)


# ---------------------------------------------------------------------------
# tensor checks of the binding (the library sees bare device pointers)
# ---------------------------------------------------------------------------
def test_binding_rejects_host_tensors():
    import torch
    from paper_2512_18995_gb300 import _lib
    for call in (lambda: _lib._f64_in(torch.zeros(4, dtype=torch.float64), 4, "params", None),
                 lambda: _lib._out(torch.zeros(4, dtype=torch.float64), 4, torch.float64, "out", None),
                 lambda: _lib._state_rows(torch.zeros((1, 8), dtype=torch.complex64), 3, "state", None)):
        with pytest.raises(_lib.DQError) as e:
            call()
        assert e.value.status == 1 and "CUDA tensor" in str(e.value)


def test_binding_tensor_checks(monkeypatch):
    """Conversion, size, type and layout checks (device check bypassed so
    that host tensors stand in for device ones)."""
    import torch
    from paper_2512_18995_gb300 import _lib
    monkeypatch.setattr(_lib, "_on_device", lambda t, what, device: None)
    t = torch.arange(6, dtype=torch.float64)
    assert _lib._f64_in(t, 6, "params", None) is t                 # already right: same tensor
    f = _lib._f64_in(torch.arange(6, dtype=torch.float32)[::2], 3, "params", None)
    assert f.dtype == torch.float64 and f.is_contiguous() and f.tolist() == [0.0, 2.0, 4.0]
    with pytest.raises(_lib.DQError):
        _lib._f64_in(t, 7, "params", None)
    assert _lib._f64_in(None, 5, "params", None) is None
    assert _lib._out(t, 6, torch.float64, "out", None) is t
    for bad in (t.float(), t[::2], t[:5]):
        with pytest.raises(_lib.DQError):
            _lib._out(bad, 6, torch.float64, "out", None)
    st = torch.zeros((3, 16), dtype=torch.complex64)
    assert _lib._state_rows(st, 4, "state", None) == 3
    with pytest.raises(_lib.DQError):
        _lib._state_rows(torch.zeros(24, dtype=torch.complex64), 4, "state", None)
    with pytest.raises(_lib.DQError):
        _lib._state_rows(torch.zeros((16, 3), dtype=torch.complex64).t(), 4, "state", None)
    with pytest.raises(TypeError):
        _lib._state_rows(torch.zeros((1, 16), dtype=torch.float32), 4, "state", None)
    c = _lib.Circuit(2, [W.Gate("rx", (0,), param=1), W.Gate("ry", (1,), data=0)])
    p, d = _lib._angles(c, torch.zeros(4), torch.zeros((2, 1)), 2, True, None)
    assert p.dtype == d.dtype == torch.float64
    with pytest.raises(_lib.DQError):
        _lib._angles(c, torch.zeros(3), None, 2, True, None)      # per-row: 2 rows x 2 params
    with pytest.raises(_lib.DQError):
        _lib._angles(c, torch.zeros(2), torch.zeros(1), 2, False, None)   # 2 rows x 1 feature


def test_missing_library_fails_loudly(tmp_path, monkeypatch):
    """No CPU fallback: without libdq.so the binding refuses to load."""
    from paper_2512_18995_gb300 import _lib
    monkeypatch.setattr(_lib, "_lib", None)
    with pytest.raises(ImportError, match="no CPU fallback"):
        _lib.load_library(str(tmp_path / "libdq.so"))


def test_product_never_touches_the_oracle():
    """The library and its binding share nothing with the oracle: no import,
    include, path or symbol of it anywhere in the package."""
    pkg = os.path.join(ROOT, "paper_2512_18995_gb300")
    hits = []
    for d, _, files in os.walk(pkg):
        if "_build" in d or "__pycache__" in d:
            continue
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".c", ".cpp")):
                text = open(os.path.join(d, f), encoding="utf-8").read()
                if re.search(r"\boracle\b", text):
                    hits.append(os.path.relpath(os.path.join(d, f), ROOT))
    assert not hits, hits


def test_oracle_shares_nothing_with_the_library():
    """The oracle includes only the C standard library and OpenMP and imports
    neither the package nor its headers."""
    src = open(os.path.join(ROOT, "oracle", "oracle.c"), encoding="utf-8").read()
    includes = set(re.findall(r"#include\s*[<\"]([^>\"]+)[>\"]", src))
    assert includes <= {"complex.h", "math.h", "stdint.h", "stdlib.h", "string.h", "omp.h"}, includes
    py = open(os.path.join(ROOT, "oracle", "__init__.py"), encoding="utf-8").read()
    assert "paper_2512_18995_gb300" not in py and "dq.h" not in py and "libdq" not in py


def test_bounds_checking_build_is_separate():
    """The bounds-checking build goes to its own library and object folder
    and differs from the normal build only by the check macro; the binding
    selects it only when DQ_DEBUG_BOUNDS is 1 (compiled and run on the GPU
    by the failure tests)."""
    import subprocess
    import sys
    from paper_2512_18995_gb300 import build as b
    assert b.LIB_DEBUG != b.LIB and b.BUILD_DEBUG != b.BUILD
    assert b.DEBUG_FLAGS == ["-DDQ_DEBUG_BOUNDS"]
    code = "from paper_2512_18995_gb300 import _lib; print(_lib.LIB_PATH)"
    for val, name in (("1", "libdq_debug.so"), ("0", "libdq.so")):
        env = dict(os.environ, DQ_DEBUG_BOUNDS=val)
        out = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True, text=True)
        assert out.stdout.strip().endswith(name), out.stdout + out.stderr
