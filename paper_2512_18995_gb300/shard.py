"""Sharding of batched work across ranks (one process per GPU).

The paper's distributed class splits one state across devices; this module
covers the other kind of parallelism its batched circuits have (Sec.
"Distributed Simulations": expectation values are gathered on one rank and
gradients come from a custom autograd function): independent batch rows of
one circuit (encoded-input batches) and independent circuits of an uneven
batch.  Every rank runs the fused forward + adjoint path on its share; the
only exchange is

* one all-reduce (sum) of the FP64 gradient of the shared parameters, which
  the loss sums over all rows, and
* all-gathers of the per-row (per-circuit) results: expectations, gradients
  with respect to encoded data, per-circuit parameter gradients.

Partitions are contiguous and deterministic, so every rank computes every
other rank's share without communication.  The collectives move host-visible
FP64 vectors only (through torch.distributed: NCCL for CUDA tensors, gloo for
CPU ones); nothing here touches another rank's device memory.

The compute step is passed in (`compute`), so the same partition, merge and
reduce code runs with the GPU library on each rank's device or, in tests,
with any other implementation on CPU tensors.
"""
from __future__ import annotations

from typing import Callable, List, Optional, Sequence, Tuple

import torch


def row_blocks(nrows: int, world: int) -> List[Tuple[int, int]]:
    """Contiguous [start, stop) row ranges, sizes differing by at most one."""
    if world < 1:
        raise ValueError("world must be >= 1")
    base, extra = divmod(max(0, nrows), world)
    out, start = [], 0
    for r in range(world):
        stop = start + base + (1 if r < extra else 0)
        out.append((start, stop))
        start = stop
    return out


def circuit_blocks(costs: Sequence[float], world: int) -> List[Tuple[int, int]]:
    """Contiguous [start, stop) circuit ranges of nearly equal total cost:
    rank r takes the circuits whose cost prefix midpoint falls in the r-th
    equal share of the total (every circuit to exactly one rank)."""
    if world < 1:
        raise ValueError("world must be >= 1")
    total = float(sum(costs))
    bounds = [0] * (world + 1)
    acc = 0.0
    r = 0
    for i, c in enumerate(costs):
        mid = acc + 0.5 * float(c)
        while r + 1 < world and total > 0 and mid >= total * (r + 1) / world:
            r += 1
            bounds[r] = i
        acc += float(c)
    for q in range(r + 1, world + 1):
        bounds[q] = len(costs)
    bounds[world] = len(costs)
    return [(bounds[q], bounds[q + 1]) for q in range(world)]


def circuit_cost(nqubits: int, ngates: int) -> float:
    """Work estimate of one circuit's forward + adjoint: gates x amplitudes."""
    return float(max(1, ngates)) * float(1 << nqubits)


def _gather_rows(local: torch.Tensor, blocks: List[Tuple[int, int]], rank: int, group) -> torch.Tensor:
    """All-gather of row blocks of unequal sizes: pad to the largest block,
    gather, cut each rank's rows back out, concatenate in rank order."""
    import torch.distributed as dist
    world = len(blocks)
    width = local.shape[1:] if local.dim() > 1 else ()
    most = max(b - a for a, b in blocks)
    pad = torch.zeros((most, *width), dtype=local.dtype, device=local.device)
    pad[: local.shape[0]] = local
    parts = [torch.empty_like(pad) for _ in range(world)]
    dist.all_gather(parts, pad, group=group)
    return torch.cat([parts[r][: blocks[r][1] - blocks[r][0]] for r in range(world)], dim=0)


def sharded_rows(compute: Callable[[int, int], Tuple[torch.Tensor, Optional[torch.Tensor], Optional[torch.Tensor]]],
                 nrows: int, nparams: int, nfeat: int, device: torch.device, group=None, params_per_row: bool = False):
    """Rows of one circuit split across the ranks of `group`.

    compute(start, stop) runs rows [start, stop) and returns (expectations
    (rows, nobs), gradient of the shared parameters summed over those rows
    (nparams,) -- or per-row (rows, nparams) when params_per_row -- and the
    data gradient (rows, nfeat) or None), all FP64 on `device`.  Returns the
    same three for the whole batch on every rank: expectations and per-row
    gradients gathered in row order, shared gradients summed over ranks."""
    import torch.distributed as dist
    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    blocks = row_blocks(nrows, world)
    a, b = blocks[rank]
    e, gp, gd = compute(a, b)
    e = _gather_rows(e.to(device=device, dtype=torch.float64).contiguous(), blocks, rank, group)
    if gp is not None:
        gp = gp.to(device=device, dtype=torch.float64).contiguous()
        if params_per_row:
            gp = _gather_rows(gp.reshape(b - a, nparams), blocks, rank, group)
        else:
            gp = gp.reshape(nparams).clone()
            dist.all_reduce(gp, op=dist.ReduceOp.SUM, group=group)
    if gd is not None:
        gd = _gather_rows(gd.to(device=device, dtype=torch.float64).reshape(b - a, nfeat).contiguous(), blocks,
                          rank, group)
    return e, gp, gd


def sharded_circuits(compute: Callable[[int, int], Tuple[torch.Tensor, Optional[torch.Tensor]]],
                     costs: Sequence[float], param_offsets: Sequence[int], nobs: int, device: torch.device,
                     group=None):
    """Circuits of an uneven batch split across ranks by cost.

    compute(start, stop) runs circuits [start, stop) and returns
    (expectations (stop - start, nobs), their parameter gradients
    concatenated (param_offsets[stop] - param_offsets[start],)).  Returns the
    whole batch's expectations and concatenated gradients on every rank."""
    import torch.distributed as dist
    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    blocks = circuit_blocks(costs, world)
    a, b = blocks[rank]
    e, gp = compute(a, b)
    e = e.to(device=device, dtype=torch.float64).reshape(b - a, nobs).contiguous()
    e = _gather_rows(e, blocks, rank, group)
    if gp is not None:
        pblocks = [(int(param_offsets[s]), int(param_offsets[t])) for s, t in blocks]
        gp = gp.to(device=device, dtype=torch.float64).reshape(-1).contiguous()
        gp = _gather_rows(gp, pblocks, rank, group)
    return e, gp


def forward_grad_sharded(ctx, circuit, params: Optional[torch.Tensor], obs, batch: int,
                         dtype=torch.complex64, data: Optional[torch.Tensor] = None,
                         row_weights: Optional[torch.Tensor] = None, params_per_row: bool = False, group=None):
    """dq_forward_grad over a batch whose rows are split across the ranks of
    `group` (each rank passes the full inputs; it runs only its rows)."""
    dev = torch.device(f"cuda:{ctx.device}")

    def compute(a, b):
        rows = b - a
        if rows == 0:
            gp = torch.zeros((0, circuit.nparams) if params_per_row else circuit.nparams, dtype=torch.float64,
                             device=dev)
            gd = torch.zeros((0, circuit.nfeatures), dtype=torch.float64, device=dev) if data is not None else None
            return torch.zeros((0, obs.nobs), dtype=torch.float64, device=dev), gp, gd
        p = params[a:b] if (params_per_row and params is not None) else params
        x = data[a:b] if data is not None else None
        w = row_weights[a:b] if row_weights is not None else None
        e, gp, gd, _ = ctx.forward_grad(circuit, p, obs, rows, dtype, data=x, row_weights=w,
                                        params_per_row=params_per_row)
        return e, gp, gd

    return sharded_rows(compute, batch, circuit.nparams, circuit.nfeatures, dev, group, params_per_row)


def batch_forward_grad_sharded(ctx, circuits, params: torch.Tensor, obs, dtype=torch.complex64, group=None):
    """dq_batch_forward_grad with the circuits split across the ranks of
    `group` by cost (each rank passes the full inputs)."""
    dev = torch.device(f"cuda:{ctx.device}")
    offs = [0]
    for c in circuits:
        offs.append(offs[-1] + c.nparams)
    costs = [circuit_cost(c.nqubits, c.ngates) for c in circuits]

    def compute(a, b):
        if b == a:
            return (torch.zeros((0, obs.nobs), dtype=torch.float64, device=dev),
                    torch.zeros(0, dtype=torch.float64, device=dev))
        e, gp = ctx.batch_forward_grad(list(circuits[a:b]), params[offs[a]:offs[b]], obs, dtype)
        return e, gp[: offs[b] - offs[a]]

    return sharded_circuits(compute, costs, offs, obs.nobs, dev, group)
