"""GB300-native batched state-vector simulation of parameterised qubit
circuits: evolution, Pauli-sum expectations and adjoint gradients (the
qubit-circuit hot path of DeepQuantum, arXiv 2512.18995), implemented as
hand-written CUDA for sm_103a behind the C ABI in ``include/dq.h``.

Typical use::

    import torch, paper_2512_18995_gb300 as dq
    ctx = dq.Context()
    circ = dq.Circuit(n, gates)                  # gates: workloads.Gate tuples
    obs = dq.Observables([[(1.0, 0, 1)]])        # <Z_0>
    e = dq.expectation(circ, params, obs, context=ctx)   # differentiable
    e.sum().backward()                                   # adjoint method
"""
from ._lib import (ADJ_CLOBBER_STATE, DQ_C64, DQ_C128, OPT_DENSE_BLOCKS, OPT_JIT, OPT_MULTIPASS, OPT_ROWS_PER_CTA, OPT_WAIT_LIMIT_US, PATH_AUTO, PATH_FUSED, PATH_PLAIN, Circuit,
                   Context,
                   DQError, Observables, load_library, lower_circuit, row_program, shift_rules, tile_schedule)
from .autograd import (DensityExpectationFunction, ExpectationFunction, density_expectation, expectation,
                       measure)

__all__ = ["Circuit", "Context", "DQError", "Observables", "expectation", "ExpectationFunction",
           "density_expectation", "DensityExpectationFunction", "measure",
           "load_library", "lower_circuit", "tile_schedule", "row_program", "shift_rules", "PATH_AUTO", "PATH_PLAIN", "PATH_FUSED", "OPT_MULTIPASS", "OPT_WAIT_LIMIT_US", "OPT_DENSE_BLOCKS", "OPT_JIT", "OPT_ROWS_PER_CTA", "DQ_C64", "DQ_C128", "ADJ_CLOBBER_STATE"]
