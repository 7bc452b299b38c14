"""Checkpoint and resume of a sliced contraction, on the host: the blocks'
partials come from the FP64 oracle over each slice block, the folded result
must equal the oracle's sum over all slices, and an interrupted run resumed
from its checkpoint must contract only the missing blocks and give the same
result bit for bit."""
import numpy as np
import pytest

from oracle import tree
from paper_2002_01935_gb300 import checkpoint, inputs, planner


def _case(open_out: bool):
    if open_out:
        circ = inputs.random_circuit(2, 3, 5, seed=2)
        net = inputs.circuit_network(circ, open_qubits=[1, 4])
    else:
        net = inputs.random_ising(20, seed=7)
    pairs = planner.greedy_tree(net.labels, net.dims, net.open)
    sliced = [l for l in sorted(net.dims) if l not in net.open][:3]
    d = int(np.prod([net.dims[l] for l in sliced]))
    return net, pairs, sliced, d


def _oracle_block(net, pairs, sliced, calls=None, fail_after=None):
    def contract_block(b, c):
        if calls is not None:
            if fail_after is not None and len(calls) == fail_after:
                raise RuntimeError("interrupted")
            calls.append((b, c))
        m, e = tree.contract_net(net, pairs, sliced, slice_begin=b, slice_count=c)
        return np.asarray(m), int(e)
    return contract_block


def test_blocks_cover_the_range():
    assert checkpoint.blocks(8, 3) == [(0, 3), (3, 3), (6, 2)]
    assert checkpoint.blocks(1, 5) == [(0, 1)]
    for bad in ((0, 1), (4, 0)):
        with pytest.raises(ValueError):
            checkpoint.blocks(*bad)


def test_fold_aligns_exponents():
    m, e = checkpoint.fold([(np.array(0.75), 10), (np.array(0.5), 12), (np.array(0.0), 500)])
    assert m * 2.0 ** e == 0.75 * 2 ** 10 + 0.5 * 2 ** 12
    m, e = checkpoint.fold([(np.array([1.0 + 1j]), -2000), (np.array([0.5j]), -1990)])
    assert e == -1990 and np.allclose(m, [2.0 ** -10 * (1 + 1j) + 0.5j], rtol=1e-15)
    m, e = checkpoint.fold([(np.zeros(3), 7)])
    assert e == 0 and not np.any(m)


@pytest.mark.parametrize("open_out", [False, True])
def test_blocks_sum_to_the_full_contraction(tmp_path, open_out):
    net, pairs, sliced, d = _case(open_out)
    m, e = checkpoint.run(_oracle_block(net, pairs, sliced), d, 3, str(tmp_path / "ck"), "case")
    rm, re = tree.contract_net(net, pairs, sliced)
    got, ref = np.asarray(m) * 2.0 ** e, np.asarray(rm) * 2.0 ** re
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))


@pytest.mark.parametrize("open_out", [False, True])
def test_interrupted_run_resumes_missing_blocks_only(tmp_path, open_out):
    net, pairs, sliced, d = _case(open_out)
    ref = checkpoint.run(_oracle_block(net, pairs, sliced), d, 3, str(tmp_path / "ref"), "case")
    path = str(tmp_path / "ck")
    first = []
    with pytest.raises(RuntimeError):
        checkpoint.run(_oracle_block(net, pairs, sliced, first, fail_after=2), d, 3, path, "case")
    assert first == [(0, 3), (3, 3)]
    again = []
    got = checkpoint.run(_oracle_block(net, pairs, sliced, again), d, 3, path, "case")
    assert again == checkpoint.blocks(d, 3)[2:]
    assert got[1] == ref[1] and np.array_equal(got[0], ref[0])
    # a finished checkpoint contracts nothing more
    none = []
    got2 = checkpoint.run(_oracle_block(net, pairs, sliced, none), d, 3, path, "case")
    assert none == [] and np.array_equal(got2[0], ref[0])


def test_checkpoint_of_another_problem_is_refused(tmp_path):
    net, pairs, sliced, d = _case(False)
    path = str(tmp_path / "ck")
    checkpoint.run(_oracle_block(net, pairs, sliced), d, 4, path, "ising-20")
    for key, block in (("other", 4), ("ising-20", 2)):
        with pytest.raises(ValueError):
            checkpoint.run(_oracle_block(net, pairs, sliced), d, block, path, key)


def test_each_block_is_its_own_file(tmp_path):
    """Recording a block writes that block only: the directory holds the
    metadata and one file per finished block."""
    import os
    net, pairs, sliced, d = _case(False)
    path = str(tmp_path / "ck")
    checkpoint.run(_oracle_block(net, pairs, sliced), d, 3, path, "case")
    names = set(os.listdir(path))
    assert names == {"meta.json"} | {f"block_{i}.npz" for i in range(len(checkpoint.blocks(d, 3)))}


def test_damaged_or_foreign_block_files_are_recomputed(tmp_path):
    """A truncated block file, one whose index lies outside the slice range,
    and one whose mantissa has another shape are treated as missing blocks:
    the resumed run contracts those blocks again and gives the same result."""
    import os
    net, pairs, sliced, d = _case(False)
    ref = checkpoint.run(_oracle_block(net, pairs, sliced), d, 3, str(tmp_path / "ref"), "case")
    path = str(tmp_path / "ck")
    checkpoint.run(_oracle_block(net, pairs, sliced), d, 3, path, "case")
    n = len(checkpoint.blocks(d, 3))
    with open(os.path.join(path, "block_1.npz"), "r+b") as f:
        f.truncate(20)
    np.savez(os.path.join(path, "block_2.npz"), index=np.array(n + 5), mantissa=np.array(1.0),
             exp2=np.array(0))
    np.savez(os.path.join(path, "block_0.npz"), index=np.array(0), mantissa=np.ones(3), exp2=np.array(0))
    again = []
    got = checkpoint.run(_oracle_block(net, pairs, sliced, again), d, 3, path, "case")
    assert sorted(again) == [checkpoint.blocks(d, 3)[i] for i in (0, 1, 2)]
    assert got[1] == ref[1] and np.array_equal(got[0], ref[0])
