"""Slice sharding across ranks: the block partition and the one exchange
that sums the partial (mantissa, exponent) results, run as world-size-2
(and 3) gloo process groups on the host.  Each rank's partial comes from
the FP64 oracle over its own slice block; the combined value must equal
the oracle's sum over all slices."""
import math
import os
import socket

import numpy as np
import pytest

from paper_2002_01935_gb300 import inputs, planner, shard


@pytest.mark.parametrize("world", [1, 2, 3, 5, 8])
@pytest.mark.parametrize("d", [0, 1, 2, 7, 16, 1000])
def test_slice_range_partitions(world, d):
    seen = []
    prev_end = 0
    for r in range(world):
        b, c = shard.slice_range(r, world, d)
        assert b == prev_end and c >= 0
        prev_end = b + c
        seen.extend(range(b, b + c))
    assert seen == list(range(d))
    counts = [shard.slice_range(r, world, d)[1] for r in range(world)]
    assert max(counts) - min(counts) <= 1


def test_slice_range_rejects_bad_arguments():
    for args in [(0, 0, 4), (2, 2, 4), (-1, 2, 4), (0, 2, -1)]:
        with pytest.raises(ValueError):
            shard.slice_range(*args)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, case, q):
    import torch
    import torch.distributed as dist
    from oracle import tree

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        net, pairs, sliced, d = case()
        b, c = shard.slice_range(rank, world, d)
        if c:
            m, e = tree.contract_net(net, pairs, sliced, slice_begin=b, slice_count=c)
            m = np.asarray(m)
        else:  # no slices on this rank: an exact zero
            m, e = np.zeros([net.dims[l] for l in net.open], dtype=np.complex128), 0
        mt = torch.from_numpy(np.ascontiguousarray(m, dtype=np.complex128))
        out, ex = shard.combine(mt, int(e))
        q.put((rank, out.numpy(), ex))
    finally:
        dist.destroy_process_group()


def _ising_case():
    net = inputs.random_ising(24, seed=3)
    pairs = planner.greedy_tree(net.labels, net.dims, net.open)
    sliced = [l for l in sorted(net.dims) if l not in net.open][:3]
    return net, pairs, sliced, 8


def _open_case():
    circ = inputs.random_circuit(2, 3, 4, seed=1)
    net = inputs.circuit_network(circ, open_qubits=[0, 3])
    pairs = planner.greedy_tree(net.labels, net.dims, net.open)
    sliced = [l for l in sorted(net.dims) if l not in net.open][:2]
    return net, pairs, sliced, 4


def _run(world, case):
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, case, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    return sorted(res, key=lambda t: t[0])


@pytest.mark.parametrize("world", [2, 3])
def test_combine_sums_slices_across_ranks(world):
    from oracle import tree
    for case in (_ising_case, _open_case):
        net, pairs, sliced, d = case()
        assert d == math.prod(net.dims[l] for l in sliced)
        mo, eo = tree.contract_net(net, pairs, sliced)
        ref = np.asarray(mo, dtype=np.complex128) * 2.0 ** eo
        res = _run(world, case)
        for rank, m, e in res:
            got = m * 2.0 ** e
            np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-12 * np.max(np.abs(ref)))
        # every rank ends with the same result
        assert all(np.array_equal(res[0][1], r[1]) and res[0][2] == r[2] for r in res)


def _slice_env_grads(net, pairs_fn, sliced, begin, count):
    """Leaf gradients (conj of the environments, adjoint 1) of the slices
    [begin, begin + count) of a closed network, from the oracle: each slice
    fixes the sliced labels (last listed fastest) and contributes its
    environments at those index values."""
    from oracle import gradient
    dims = net.dims
    grads = [np.zeros(np.shape(t), dtype=np.complex128) for t in net.tensors]
    radix = [dims[l] for l in sliced]
    for s in range(begin, begin + count):
        val, rem = {}, s
        for l, d in zip(reversed(sliced), reversed(radix)):
            val[l] = rem % d
            rem //= d
        ts, ls, idx = [], [], []
        for t, lab in zip(net.tensors, net.labels):
            sel = tuple(val[l] if l in val else slice(None) for l in lab)
            ts.append(np.asarray(t)[sel])
            ls.append([l for l in lab if l not in val])
            idx.append(sel)
        for v in range(net.n_tensors):
            env = gradient.environment(ts, ls, dims, v, pairs_fn)
            grads[v][idx[v]] += np.conj(env)
    return grads


def _grad_worker(rank, world, port, q):
    import torch
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        net = inputs.random_network(6, 9, 812, n_open=0, complex_=True)
        sliced = sorted(net.dims)[:3]
        d = math.prod(net.dims[l] for l in sliced)
        b, c = shard.slice_range(rank, world, d)
        part = _slice_env_grads(net, planner.greedy_tree, sliced, b, c)
        ts = [torch.from_numpy(g.copy()) for g in part]
        shard.combine_grads(ts + [None])
        q.put((rank, [t.numpy() for t in ts]))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_combine_grads_sums_slice_blocks(world):
    """Per-rank gradients over blocks of slices, summed by combine_grads,
    equal the gradient of the whole (unsliced) network."""
    from oracle import gradient
    import torch.multiprocessing as mp
    net = inputs.random_network(6, 9, 812, n_open=0, complex_=True)
    full = [np.conj(gradient.environment(net.tensors, net.labels, net.dims, v, planner.greedy_tree))
            for v in range(net.n_tensors)]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_grad_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=180) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, gs in res:
        for g, ref in zip(gs, full):
            np.testing.assert_allclose(g, ref, rtol=1e-11, atol=1e-12 * np.max(np.abs(ref)))


def test_combine_grads_rejects_strided_buffers():
    import torch
    with pytest.raises(ValueError):
        shard.combine_grads([torch.zeros(4, 4)[:, 1]])


def _leaving_worker(rank, world, port, q):
    """The last rank leaves between steps (nothing in flight); the others'
    next exchange must end with an error instead of waiting forever."""
    import datetime
    import torch
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=10))
    if rank == world - 1:
        os._exit(0)
    try:
        shard.combine(torch.zeros(2, dtype=torch.complex128), 0)
        q.put((rank, "completed"))
    except Exception as e:  # the backend reports the lost peer
        q.put((rank, type(e).__name__))


@pytest.mark.parametrize("world", [2, 3])
def test_exchange_fails_cleanly_when_a_rank_leaves(world):
    import time
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_leaving_worker, args=(r, world, port, q)) for r in range(world)]
    t0 = time.monotonic()
    for p in procs:
        p.start()
    try:
        res = sorted(q.get(timeout=120) for _ in range(world - 1))
    finally:
        for p in procs:
            p.join(timeout=30)
            if p.is_alive():
                p.kill()
                p.join()
    assert [r for r, _ in res] == list(range(world - 1))
    assert all(outcome != "completed" for _, outcome in res), res
    assert time.monotonic() - t0 < 120
