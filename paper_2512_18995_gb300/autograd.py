"""torch.autograd.Function over the library: forward = state preparation,
evolution and Pauli-sum expectations; backward = the adjoint method with the
upstream gradient as per-row observable weights (the custom autograd function
with adjoint differentiation described in Sec. "Distributed Simulations").

Checkpointing: when the final states of the batch fit the memory budget they
are kept from the forward pass and the backward pass only runs the reverse
sweep; otherwise nothing but the inputs is kept and the backward pass
recomputes the forward states (dq_forward_grad) before sweeping back.  Small
states take the fused on-chip path, which always recomputes (it is cheaper
than storing).  The kept states are consumed by the first backward pass (the
sweep runs on them in place); a further backward through the same graph
recomputes.
"""
from __future__ import annotations

from typing import Optional

import torch

from ._lib import Circuit, Context, Observables

_default_ctx = {}


def default_context(device: int = None) -> Context:
    dev = torch.cuda.current_device() if device is None else device
    if dev not in _default_ctx:
        _default_ctx[dev] = Context(dev)
    return _default_ctx[dev]


def _small(n: int, dtype: torch.dtype) -> bool:
    # both vectors of one row fit in one CTA's shared memory
    amp = 8 if dtype == torch.complex64 else 16
    return (2 * amp << n) <= 200 * 1024


class ExpectationFunction(torch.autograd.Function):
    @staticmethod
    def forward(fctx, params, data, circuit: Circuit, obs: Observables, context: Context, dtype, params_per_row,
                memory_budget):
        if data is not None:
            batch = data.shape[0]
        elif params_per_row:
            batch = params.shape[0]
        else:
            batch = 1
        state_bytes = (batch << circuit.nqubits) * (8 if dtype == torch.complex64 else 16)
        keep = (not _small(circuit.nqubits, dtype)) and state_bytes <= memory_budget
        state = None
        if keep:
            state = torch.empty((batch, 1 << circuit.nqubits), dtype=dtype, device=f"cuda:{context.device}")
        exp, _, _, _ = context.forward_grad(circuit, params, obs, batch, dtype, data=data,
                                            params_per_row=params_per_row, want_grad=False, state_out=state)
        fctx.circuit, fctx.obs, fctx.context, fctx.dtype = circuit, obs, context, dtype
        fctx.ppr, fctx.batch = params_per_row, batch
        fctx.save_for_backward(params, data, state)
        return exp

    @staticmethod
    def backward(fctx, grad_out):
        params, data, state = fctx.saved_tensors
        w = grad_out.detach().to(torch.float64).contiguous()
        ctx = fctx.context
        if state is not None and not getattr(fctx, "state_swept", False):
            # The reverse sweep un-applies the circuit on the kept states in
            # place (no copy).  The library writes through a raw pointer, so
            # torch does not see the change: remember it, and let a second
            # backward through the same graph (retain_graph=True) recompute.
            fctx.state_swept = True
            gp, gd = ctx.adjoint_grad(fctx.circuit, params, fctx.obs, state, data=data, row_weights=w,
                                      params_per_row=fctx.ppr, clobber=True)
        else:
            _, gp, gd, _ = ctx.forward_grad(fctx.circuit, params, fctx.obs, fctx.batch, fctx.dtype, data=data,
                                            row_weights=w, params_per_row=fctx.ppr, want_expect=False,
                                            want_grad=True)
        gpo = gp if (params is not None and fctx.needs_input_grad[0]) else None
        gdo = gd if (data is not None and fctx.needs_input_grad[1]) else None
        if gpo is not None:
            gpo = gpo.to(params.dtype).reshape(params.shape)
        if gdo is not None:
            gdo = gdo.to(data.dtype).reshape(data.shape)
        return gpo, gdo, None, None, None, None, None, None


def expectation(circuit: Circuit, params: Optional[torch.Tensor], obs: Observables,
                data: Optional[torch.Tensor] = None, dtype: torch.dtype = torch.complex64,
                context: Optional[Context] = None, params_per_row: bool = False,
                memory_budget: Optional[int] = None) -> torch.Tensor:
    """Differentiable expectations, shape (batch, nobs), FP64.

    ``params`` (FP64 CUDA tensor, (nparams,) or (batch, nparams)) and ``data``
    (FP64 CUDA tensor (batch, nfeatures)) may require grad; backward runs the
    adjoint method on the GPU."""
    context = context or default_context()
    if memory_budget is None:
        free, _ = torch.cuda.mem_get_info(context.device)
        memory_budget = free // 4
    if params is not None and params.dtype != torch.float64:
        params = params.to(torch.float64)
    if data is not None and data.dtype != torch.float64:
        data = data.to(torch.float64)
    return ExpectationFunction.apply(params, data, circuit, obs, context, dtype, params_per_row, memory_budget)


class DensityExpectationFunction(torch.autograd.Function):
    """Expectations Re Tr(O rho) of a noisy (density-matrix) circuit; backward
    runs the exact shift rules of dq_density_grad with the upstream gradient
    as per-row observable weights (shared parameters only)."""

    @staticmethod
    def forward(fctx, params, data, circuit: Circuit, obs: Observables, context: Context, dtype):
        batch = data.shape[0] if data is not None else 1
        exp, _ = context.density_forward(circuit, params, obs, batch, dtype, data=data)
        fctx.circuit, fctx.obs, fctx.context, fctx.dtype = circuit, obs, context, dtype
        fctx.save_for_backward(params, data)
        return exp

    @staticmethod
    def backward(fctx, grad_out):
        params, data = fctx.saved_tensors
        grad_params = None
        if fctx.needs_input_grad[0]:
            _, grad_params = fctx.context.density_grad(fctx.circuit, params, fctx.obs, data=data,
                                                       row_weights=grad_out.contiguous().to(torch.float64),
                                                       dtype=fctx.dtype)
        return grad_params, None, None, None, None, None


def density_expectation(circuit: Circuit, params: torch.Tensor, obs: Observables,
                        data: Optional[torch.Tensor] = None, dtype: torch.dtype = torch.complex64,
                        context: Optional[Context] = None) -> torch.Tensor:
    """Differentiable (with respect to ``params``) expectations (batch, nobs)
    of a circuit with noise channels, simulated as density matrices."""
    context = context or default_context()
    if params.dtype != torch.float64:
        params = params.to(torch.float64)
    if data is not None and data.dtype != torch.float64:
        data = data.to(torch.float64)
    return DensityExpectationFunction.apply(params, data, circuit, obs, context, dtype)


def measure(state: torch.Tensor, nqubits: int, shots: int, wires=None, seed: int = 0,
            context: Optional[Context] = None):
    """Shot counts of a batch of states (the API overview's measure(shots,
    wires)): a list (one per row) of {bitstring: count}, bitstrings over
    ``wires`` (all wires by default) in increasing wire order, the lowest wire
    leftmost (as in the full basis bitstring)."""
    context = context or default_context()
    ws = list(range(nqubits)) if wires is None else sorted(int(w) for w in wires)
    out = context.sample(nqubits, state, shots, seed=seed, wires=None if wires is None else ws)
    width = len(ws)
    counts = []
    for row in out.cpu().tolist():
        d = {}
        for v in row:
            key = format(v, f"0{width}b")
            d[key] = d.get(key, 0) + 1
        counts.append(dict(sorted(d.items())))
    return counts
