"""Row and circuit sharding across ranks (Sec. "Distributed Simulations":
results gathered from all ranks, gradients of the shared parameters summed)
on CPU: gloo ranks feed the same partition, gather and all-reduce code that
the GPU path uses with host arrays that the FP64 oracle computes for each
rank's share, and the merged results must equal the oracle's single-rank
answer for the whole batch (to FP64 summation-order rounding)."""
import os
import socket
import sys

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import workloads as W
from paper_2512_18995_gb300 import shard

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


# ---------------------------------------------------------------------------
# partitions
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("nrows,world", [(0, 2), (1, 3), (7, 2), (4096, 8), (10, 10), (5, 8)])
def test_row_blocks_cover_every_row_once(nrows, world):
    b = shard.row_blocks(nrows, world)
    assert len(b) == world and b[0][0] == 0 and b[-1][1] == nrows
    assert all(b[i][1] == b[i + 1][0] for i in range(world - 1))
    sizes = [y - x for x, y in b]
    assert min(sizes) >= 0 and max(sizes) - min(sizes) <= 1


@pytest.mark.parametrize("world", [1, 2, 3, 8])
def test_circuit_blocks_balance_cost(world):
    rng = np.random.default_rng(world)
    costs = [float(rng.integers(10, 40)) * 2.0 ** int(rng.integers(8, 17)) for _ in range(1024)]
    b = shard.circuit_blocks(costs, world)
    assert len(b) == world and b[0][0] == 0 and b[-1][1] == len(costs)
    assert all(b[i][1] == b[i + 1][0] and b[i][0] <= b[i][1] for i in range(world - 1))
    share = [sum(costs[x:y]) for x, y in b]
    # each share within one largest circuit of the ideal
    assert max(abs(s - sum(costs) / world) for s in share) <= max(costs)


def test_circuit_blocks_degenerate():
    assert shard.circuit_blocks([], 3) == [(0, 0)] * 3
    assert shard.circuit_blocks([5.0], 2) in ([(0, 1), (1, 1)], [(0, 0), (0, 1)])
    assert shard.circuit_blocks([1.0, 1.0, 1.0, 1.0], 2) == [(0, 2), (2, 4)]


# ---------------------------------------------------------------------------
# gloo ranks
# ---------------------------------------------------------------------------
def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rows_workload():
    n, batch, layers = 8, 37, 2
    gates = W.encode_layer(n) + W.hea_layers(n, layers)
    rng = np.random.default_rng(11)
    params = rng.uniform(0, 2 * np.pi, 2 * n * layers)
    data = rng.uniform(-np.pi, np.pi, (batch, n))
    obs = [W.obs_z(0), W.obs_tfim_open(n, 0.5)]
    w = rng.normal(size=(batch, 2))
    return n, batch, gates, params, data, obs, w


def _circuits_workload():
    return [W.random_circuit(5000 + c, nmin=3, nmax=8) for c in range(41)]


def _rank_main(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import oracle
    oracle.build()
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    cpu = torch.device("cpu")
    try:
        # rows of one circuit: shared parameters (all-reduced) and per-row ones (gathered)
        n, batch, gates, params, data, obs, w = _rows_workload()
        res = {}
        for ppr in (False, True):
            p = np.tile(params, (batch, 1)) + 0.01 * np.arange(batch)[:, None] if ppr else params

            def compute(a, b, p=p, ppr=ppr):
                if b == a:
                    gp = torch.zeros((0, p.shape[-1]) if ppr else p.shape[-1], dtype=torch.float64)
                    return torch.zeros((0, 2), dtype=torch.float64), gp, torch.zeros((0, n), dtype=torch.float64)
                e, gp, gd = oracle.adjoint(n, gates, obs, p[a:b] if ppr else p, data[a:b], batch=b - a,
                                           params_per_row=ppr, row_weights=w[a:b])
                return torch.from_numpy(e), torch.from_numpy(gp), torch.from_numpy(gd)

            e, gp, gd = shard.sharded_rows(compute, batch, params.size, n, cpu, None, ppr)
            res[ppr] = (e.numpy(), gp.numpy(), gd.numpy())
        # circuits of an uneven batch
        circs = _circuits_workload()
        cobs = [W.obs_zz01_x0()]
        offs = np.cumsum([0] + [len(a) for _, _, a in circs])
        costs = [shard.circuit_cost(nq, len(g)) for nq, g, _ in circs]

        def ccompute(a, b):
            es, gs = [], []
            for nq, g, ang in circs[a:b]:
                e, gp, _ = oracle.adjoint(nq, g, cobs, ang)
                es.append(e[0])
                gs.append(gp)
            e = torch.from_numpy(np.array(es).reshape(b - a, 1))
            g = torch.from_numpy(np.concatenate(gs)) if gs else torch.zeros(0, dtype=torch.float64)
            return e, g

        ce, cg = shard.sharded_circuits(ccompute, costs, offs, 1, cpu, None)
        res["circuits"] = (ce.numpy(), cg.numpy(), shard.circuit_blocks(costs, world))
        out[rank] = res
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_sharded_results_equal_the_single_rank_oracle(world, oracle_mod):
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        mp.start_processes(_rank_main, args=(world, port, out), nprocs=world, join=True, start_method="spawn")
        res = dict(out)
    assert sorted(res) == list(range(world))
    n, batch, gates, params, data, obs, w = _rows_workload()
    for ppr in (False, True):
        p = np.tile(params, (batch, 1)) + 0.01 * np.arange(batch)[:, None] if ppr else params
        e_ref, gp_ref, gd_ref = oracle_mod.adjoint(n, gates, obs, p, data, batch=batch, params_per_row=ppr,
                                                   row_weights=w)
        for r in range(world):
            e, gp, gd = res[r][ppr]
            # gathered blocks are the oracle's own numbers, in row order
            assert np.array_equal(e, e_ref) and np.array_equal(gd, gd_ref)
            if ppr:
                assert np.array_equal(gp, gp_ref)
            else:
                # the all-reduce sums the ranks' partial sums: summation order only
                assert np.max(np.abs(gp - gp_ref)) <= 1e-12 * np.max(np.abs(gp_ref))
                assert np.array_equal(gp, res[0][ppr][1])          # every rank holds the same sum
    circs = _circuits_workload()
    cobs = [W.obs_zz01_x0()]
    e_ref = []
    g_ref = []
    for nq, g, ang in circs:
        e, gp, _ = oracle_mod.adjoint(nq, g, cobs, ang)
        e_ref.append(e[0, 0])
        g_ref.append(gp)
    for r in range(world):
        ce, cg, blocks = res[r]["circuits"]
        assert np.array_equal(ce.reshape(-1), np.array(e_ref))
        assert np.array_equal(cg, np.concatenate(g_ref))
        assert sum(b - a for a, b in blocks) == len(circs)
