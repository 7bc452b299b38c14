"""tn_contract_grad_ex: device adjoints, device exponents, accumulation,
and the reuse of the captured reverse-sweep graph across calls whose leaf
and gradient pointers change.  Every result is checked against either the
FP64 oracle (environments of the leaves) or the host-adjoint call, which the
oracle tests pin."""
import numpy as np
import pytest

from oracle import gradient
from paper_2002_01935_gb300 import inputs, planner

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as _t
    if not _t.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2002_01935_gb300 import build
    build.build()
    return _t


def _tree(l, d, o):
    return planner.greedy_tree(l, d, o)


def _setup(torch, seed=11, n_open=1, complex_=True, sliced_n=0):
    from paper_2002_01935_gb300 import binding
    net = inputs.random_network(7, 12, 900 + seed, n_open=n_open, complex_=complex_)
    pairs = planner.greedy_tree(net.labels, net.dims, net.open)
    dt = torch.complex64 if complex_ else torch.float32
    ts = [torch.from_numpy(np.array(t, order="C")).to(dt).cuda() for t in net.tensors]
    tnw = binding.TensorNetwork(net.labels, net.dims, net.open, ts, complex_=complex_)
    summed = [l for l in sorted(net.dims) if l not in net.open]
    return net, pairs, summed[:sliced_n], ts, tnw


def _adjoint(net, seed):
    rng = np.random.default_rng(seed)
    shape = tuple(net.dims[l] for l in net.open)
    a = rng.standard_normal(shape)
    if net.is_complex:
        a = a + 1j * rng.standard_normal(shape)
    return a


def _oracle(net, adj):
    ts, ls = list(net.tensors), [list(x) for x in net.labels]
    ts.append(np.conj(np.asarray(adj)))
    ls.append(list(net.open))
    return [np.conj(gradient.environment(ts, ls, net.dims, v, _tree)) for v in range(net.n_tensors)]


@pytest.mark.parametrize("sliced_n", [0, 2])
def test_device_adjoint_matches_host_adjoint(torch, sliced_n):
    net, pairs, sliced, ts, tnw = _setup(torch, sliced_n=sliced_n)
    adj = _adjoint(net, 1)
    g_host = [g.cpu().numpy() for g in tnw.grad(pairs, sliced, "fp32", adj)]
    adj_dev = torch.from_numpy(np.ascontiguousarray(adj)).cuda()
    g_dev = tnw.grad(pairs, sliced, "fp32", adj_dev)
    torch.cuda.synchronize()
    for a, b in zip(g_host, g_dev):
        assert np.array_equal(a, b.cpu().numpy())
    ref = _oracle(net, adj)
    for v in range(net.n_tensors):
        assert np.linalg.norm(g_host[v] - ref[v]) <= 1e-5 * (np.linalg.norm(ref[v]) + 1e-30), v
    tnw.close()


def test_device_exponent_scales_exactly(torch):
    net, pairs, sliced, ts, tnw = _setup(torch, seed=12)
    adj = _adjoint(net, 2)
    adj_dev = torch.from_numpy(np.ascontiguousarray(adj)).cuda()
    base = [g.cpu().numpy() for g in tnw.grad(pairs, sliced, "fp32", adj_dev)]
    for k in (-7, 5):
        e = torch.tensor(k, dtype=torch.int64, device="cuda")
        got = tnw.grad(pairs, sliced, "fp32", adj_dev, adj_exp2=e)
        torch.cuda.synchronize()
        for a, b in zip(base, got):
            assert np.array_equal(np.ldexp(a.real, k) + 1j * np.ldexp(a.imag, k), b.cpu().numpy())
    tnw.close()


def test_accumulate_adds_into_buffers(torch):
    net, pairs, sliced, ts, tnw = _setup(torch, seed=13, sliced_n=1)
    adj1, adj2 = _adjoint(net, 3), _adjoint(net, 4)
    g1 = [g.cpu().numpy() for g in tnw.grad(pairs, sliced, "fp32", adj1)]
    g2 = [g.cpu().numpy() for g in tnw.grad(pairs, sliced, "fp32", adj2)]
    acc = [torch.full_like(t, 0.25 + 0.5j) for t in ts]
    acc[1] = None  # skipped leaf
    tnw.grad(pairs, sliced, "fp32", adj1, grads=acc, accumulate=True)
    tnw.grad(pairs, sliced, "fp32", adj2, grads=acc, accumulate=True)
    torch.cuda.synchronize()
    for v, a in enumerate(acc):
        if a is None:
            continue
        want = (np.complex64(0.25 + 0.5j) + g1[v]) + g2[v]  # float32 adds, in call order
        assert np.array_equal(a.cpu().numpy(), want.astype(np.complex64)), v
    tnw.close()


def test_graph_reuse_with_new_pointers(torch):
    """Second and later calls replay the captured sweep: new leaf tensors
    (other addresses, other values) and new gradient buffers must give the
    oracle's gradients for the new values."""
    net, pairs, sliced, ts, tnw = _setup(torch, seed=14, sliced_n=1)
    adj = _adjoint(net, 5)
    tnw.grad(pairs, sliced, "fp32", adj)  # captures
    rng = np.random.default_rng(6)
    for rep in range(3):
        new = [t * np.float32(1.0 + 0.1 * rng.standard_normal()) for t in net.tensors]
        net2 = net.with_tensors(new)
        ts2 = [torch.from_numpy(np.array(t, order="C")).to(torch.complex64).cuda() for t in new]
        tnw.set_tensors(ts2)
        got = [g.cpu().numpy() for g in tnw.grad(pairs, sliced, "fp32", adj)]
        ref = _oracle(net2, adj)
        for v in range(net.n_tensors):
            assert np.linalg.norm(got[v] - ref[v]) <= 1e-5 * (np.linalg.norm(ref[v]) + 1e-30), (rep, v)
    tnw.close()


def test_bad_arguments_are_refused(torch):
    from paper_2002_01935_gb300 import binding
    net, pairs, sliced, ts, tnw = _setup(torch, seed=15)
    adj = _adjoint(net, 7)
    e = torch.tensor(1, dtype=torch.int64, device="cuda")
    with pytest.raises(TypeError):  # device exponent with a host adjoint
        tnw.grad(pairs, sliced, "fp32", adj, adj_exp2=e)
    gp = [torch.empty_like(t).data_ptr() for t in ts]
    adj_np = np.ascontiguousarray(adj)
    with pytest.raises(binding.TNError):  # same, at the C-ABI
        binding.tn_contract_grad_ex(tnw.h, pairs, sliced, 0, adj_np.ctypes.data, binding.TN_MEM_HOST, 0,
                                    e.data_ptr(), gp, 0, 0)
    with pytest.raises(binding.TNError):  # unknown flag
        binding.tn_contract_grad_ex(tnw.h, pairs, sliced, 0, adj_np.ctypes.data, binding.TN_MEM_HOST, 0,
                                    0, gp, 2, 0)
    tnw.close()


def test_refused_under_stream_capture(torch):
    from paper_2002_01935_gb300 import binding
    net, pairs, sliced, ts, tnw = _setup(torch, seed=16)
    adj_dev = torch.from_numpy(np.ascontiguousarray(_adjoint(net, 8))).cuda()
    tnw.grad(pairs, sliced, "fp32", adj_dev)
    torch.cuda.synchronize()
    grads = [torch.empty_like(t) for t in ts]
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with pytest.raises(binding.TNError):
        with torch.cuda.graph(g, stream=s):
            tnw.grad(pairs, sliced, "fp32", adj_dev, grads=grads, stream=s)
    tnw.close()


def test_accumulated_step_matches_autograd(torch):
    """A loop over bitstrings at the C-ABI level (device adjoint 2 / (B
    conj(A)) formed from each forward result, accumulation over the
    bitstrings, one torch backward to the fSim parameters) against the
    autograd Function."""
    from paper_2002_01935_gb300 import autograd, binding
    R, C, T = 3, 3, 6
    circ = inputs.random_circuit(R, C, T, seed=2)
    bits = inputs.random_bitstrings(R * C, 6, seed=3)
    fs = circ.fsim_gates()
    nets = [inputs.circuit_network(circ, b) for b in bits]
    net0 = nets[0]
    n = net0.n_tensors
    first_out = n - R * C
    pairs = planner.greedy_tree(net0.labels, net0.dims, net0.open)
    leaf_of = [net0.meta["gate_leaf"][g] for g in fs]
    base = [torch.from_numpy(np.array(t, order="C")).to(torch.complex64).cuda() for t in net0.tensors]
    outs = [torch.stack([torch.from_numpy(np.array(nt.tensors[v], order="C")).to(torch.complex64)
                         for v in range(first_out, n)]).cuda() for nt in nets]

    def params():
        th = torch.tensor([circ.gates[g].params[0] for g in fs], dtype=torch.float64, device="cuda",
                          requires_grad=True)
        ph = torch.tensor([circ.gates[g].params[1] for g in fs], dtype=torch.float64, device="cuda",
                          requires_grad=True)
        return th, ph

    def fsim_batch(th, ph):
        c, s = torch.cos(th).to(torch.complex128), torch.sin(th).to(torch.complex128)
        g = torch.zeros((th.shape[0], 4, 4), dtype=torch.complex128, device="cuda")
        g[:, 0, 0] = 1
        g[:, 1, 1] = c
        g[:, 2, 2] = c
        g[:, 1, 2] = -1j * s
        g[:, 2, 1] = -1j * s
        g[:, 3, 3] = torch.exp(-1j * ph.to(torch.complex128))
        return g.to(torch.complex64).reshape(-1, 2, 2, 2, 2)

    # autograd Function
    th, ph = params()
    G = fsim_batch(th, ph)
    tnw = binding.TensorNetwork(net0.labels, net0.dims, net0.open, None, complex_=True)
    loss = 0.0
    for x in range(len(bits)):
        lv = list(base)
        for i, v in enumerate(leaf_of):
            lv[v] = G[i]
        lv = lv[:first_out] + [outs[x][q] for q in range(R * C)]
        loss = loss + torch.log(torch.abs(autograd.contract(tnw, pairs, [], "fp32", *lv)) ** 2) / len(bits)
    loss.backward()
    ref_th, ref_ph = th.grad.cpu().numpy(), ph.grad.cpu().numpy()
    tnw.close()

    # accumulation through tn_contract_grad_ex
    th, ph = params()
    tnw = binding.TensorNetwork(net0.labels, net0.dims, net0.open, None, complex_=True)
    dG = torch.zeros((len(fs), 2, 2, 2, 2), dtype=torch.complex64, device="cuda")
    gbuf = [None] * n
    for i, v in enumerate(leaf_of):
        gbuf[v] = dG[i]
    out_buf = torch.empty_like(outs[0])
    with torch.no_grad():
        Gd = fsim_batch(th.detach(), ph.detach())
        lv = list(base)
        for i, v in enumerate(leaf_of):
            lv[v] = Gd[i]
        tnw.set_tensors(lv[:first_out] + [out_buf[q] for q in range(R * C)])
        for x in range(len(bits)):
            out_buf.copy_(outs[x])
            m, e = tnw.contract(pairs, [], "fp32")
            adj = 2.0 / (len(bits) * torch.conj(m))
            tnw.grad(pairs, [], "fp32", adj, adj_exp2=torch.neg(e), grads=gbuf, accumulate=True)
    torch.autograd.backward(fsim_batch(th, ph), dG)
    got_th, got_ph = th.grad.cpu().numpy(), ph.grad.cpu().numpy()
    tnw.close()
    scale = max(np.max(np.abs(ref_th)), np.max(np.abs(ref_ph)))
    assert np.max(np.abs(got_th - ref_th)) <= 1e-5 * scale
    assert np.max(np.abs(got_ph - ref_ph)) <= 1e-5 * scale


def test_contract_batch_matches_per_network_function(torch):
    """contract_batch (instances forward, per-network sweeps with summed
    shared-leaf gradients) against autograd.contract called per network:
    values, fSim-leaf gradients and output-leaf gradients."""
    from paper_2002_01935_gb300 import autograd, binding
    R, C, T = 3, 3, 6
    circ = inputs.random_circuit(R, C, T, seed=7)
    bits = inputs.random_bitstrings(R * C, 5, seed=8)
    nets = [inputs.circuit_network(circ, b) for b in bits]
    net0 = nets[0]
    n = net0.n_tensors
    first_out = n - R * C
    pairs = planner.greedy_tree(net0.labels, net0.dims, net0.open)

    def leaves_of(req):
        base = [torch.from_numpy(np.array(t, order="C")).to(torch.complex64).cuda() for t in net0.tensors]
        for v in (0, 5, first_out - 1):
            base[v].requires_grad_(req)
        outs = torch.stack([torch.stack([torch.from_numpy(np.array(nt.tensors[v], order="C")).to(torch.complex64)
                                         for v in range(first_out, n)]) for nt in nets]).cuda()
        outs.requires_grad_(req)
        return base, outs

    base, outs = leaves_of(True)
    tnw = binding.TensorNetwork(net0.labels, net0.dims, net0.open, None, complex_=True)
    vals = []
    for x in range(len(bits)):
        lv = base[:first_out] + [outs[x, q] for q in range(R * C)]
        vals.append(autograd.contract(tnw, pairs, [], "fp32", *lv))
    ref_v = torch.stack(vals)
    loss = torch.sum(torch.log(torch.abs(ref_v) ** 2))
    loss.backward()
    ref = [base[v].grad.cpu().numpy() for v in (0, 5, first_out - 1)] + [outs.grad.cpu().numpy()]
    tnw.close()

    base, outs = leaves_of(True)
    tnw = binding.TensorNetwork(net0.labels, net0.dims, net0.open, None, complex_=True)
    batch = {first_out + q: outs[:, q] for q in range(R * C)}
    got_v = autograd.contract_batch(tnw, pairs, "fp32", base[:first_out] + [None] * (R * C), batch)
    loss = torch.sum(torch.log(torch.abs(got_v) ** 2))
    loss.backward()
    got = [base[v].grad.cpu().numpy() for v in (0, 5, first_out - 1)] + [outs.grad.cpu().numpy()]
    tnw.close()
    rv, gv = ref_v.detach().cpu().numpy(), got_v.detach().cpu().numpy()
    assert np.max(np.abs(gv - rv)) <= 1e-5 * np.max(np.abs(rv))
    for a, b in zip(got, ref):
        assert np.linalg.norm(a - b) <= 1e-5 * np.linalg.norm(b)


@pytest.mark.parametrize("sliced_n,mode", [(0, "fp32"), (1, "fp32"), (0, "tf32_split")])
def test_grad_instances_match_single_sweeps(torch, sliced_n, mode):
    """n copies in one sweep (two leaves varying per copy, the rest shared)
    against one tn_contract_grad call per copy: shared leaves get the sum
    over the copies, varying leaves each copy's gradient."""
    net, pairs, sliced, ts, tnw = _setup(torch, seed=21, sliced_n=sliced_n)
    B = 5
    rng = np.random.default_rng(9)
    var = [1, 4]
    stacks = {v: torch.stack([ts[v] * np.float32(1.0 + 0.2 * rng.standard_normal()) for _ in range(B)])
              for v in var}
    adjs = np.stack([_adjoint(net, 30 + i) for i in range(B)])
    singles = []
    for i in range(B):
        lv = list(ts)
        for v in var:
            lv[v] = stacks[v][i].contiguous()
        tnw.set_tensors(lv)
        singles.append([g.cpu().numpy() for g in tnw.grad(pairs, sliced, mode, adjs[i])])
    lv = list(ts)
    strides = [0] * len(ts)
    for v in var:
        lv[v] = stacks[v]
        strides[v] = ts[v].numel()
    tnw.set_tensors(lv)
    adj_dev = torch.from_numpy(np.ascontiguousarray(adjs)).cuda()
    got = [g.cpu().numpy() for g in tnw.grad_instances(pairs, sliced, mode, B, strides, adj_dev)]
    for v in range(len(ts)):
        if v in var:
            ref = np.stack([singles[i][v] for i in range(B)])
        else:
            ref = sum(singles[i][v].astype(np.complex128) for i in range(B))
        assert got[v].shape == ref.shape, v
        assert np.linalg.norm(got[v] - ref) <= 1e-5 * (np.linalg.norm(ref) + 1e-30), v
    # accumulation into the same buffers doubles them
    acc = [torch.from_numpy(g.copy()).cuda() for g in got]
    tnw.grad_instances(pairs, sliced, mode, B, strides, adj_dev, grads=acc, accumulate=True)
    for v in range(len(ts)):
        assert np.array_equal(acc[v].cpu().numpy(), (got[v] + got[v]).astype(got[v].dtype)), v
    tnw.close()


def test_grad_instances_refuses_overlapping_copies(torch):
    from paper_2002_01935_gb300 import binding
    net, pairs, sliced, ts, tnw = _setup(torch, seed=22)
    strides = [0] * len(ts)
    v = int(np.argmax([t.numel() for t in ts]))
    assert ts[v].numel() >= 2
    strides[v] = ts[v].numel() // 2  # copies would overlap
    adj = np.stack([_adjoint(net, 1), _adjoint(net, 2)])
    with pytest.raises(binding.TNError):
        tnw.grad_instances(pairs, sliced, "fp32", 2, strides, adj)
    tnw.close()


def _stacked_setup(torch, seed, B):
    net, pairs, sliced, ts, tnw = _setup(torch, seed=seed, n_open=0)
    rng = np.random.default_rng(seed)
    var = [0, 3]
    lv = list(ts)
    strides = [0] * len(ts)
    for v in var:
        lv[v] = torch.stack([ts[v] * np.float32(1.0 + 0.2 * rng.standard_normal()) for _ in range(B)])
        strides[v] = ts[v].numel()
    tnw.set_tensors(lv)
    adjs = torch.from_numpy(rng.standard_normal((B, 2)).view(np.complex128).reshape(B)).cuda()
    return net, pairs, tnw, lv, strides, adjs


def test_kept_forward_matches_recompute(torch):
    """grad_instances after contract_instances_keep (sweep only) against the
    full call (forward recomputed): identical gradients; the kept values
    against tn_contract_instances."""
    B = 4
    net, pairs, tnw, lv, strides, adjs = _stacked_setup(torch, 23, B)
    for mode in ("fp32", "tf32_split"):
        full = [g.cpu().numpy() for g in tnw.grad_instances(pairs, [], mode, B, strides, adjs)]
        m, e, token = tnw.contract_instances_keep(pairs, mode, B, strides)
        kept = [g.cpu().numpy() for g in tnw.grad_instances(pairs, [], mode, B, strides, adjs, kept_forward=token)]
        for a, b in zip(full, kept):
            assert np.array_equal(a, b)
        m2, e2 = tnw.contract_instances(pairs, mode, B, strides)
        v1 = (m[:, 0] + 1j * m[:, 1]).cpu().numpy() * np.exp2(e.cpu().numpy().astype(float))
        v2 = (m2[:, 0] + 1j * m2[:, 1]).cpu().numpy() * np.exp2(e2.cpu().numpy().astype(float))
        assert np.max(np.abs(v1 - v2)) <= 1e-5 * np.max(np.abs(v2))
    tnw.close()


def test_kept_forward_refused_when_stale(torch):
    """After another gradient call the kept forward is gone: the C-ABI
    refuses the flag, and the binding falls back to the full call."""
    from paper_2002_01935_gb300 import binding
    B = 3
    net, pairs, tnw, lv, strides, adjs = _stacked_setup(torch, 24, B)
    ref = [g.cpu().numpy() for g in tnw.grad_instances(pairs, [], "fp32", B, strides, adjs)]
    m, e, token = tnw.contract_instances_keep(pairs, "fp32", B, strides)
    tnw.grad_instances(pairs, [], "fp32", B, strides, adjs * 2)  # rewrites the sweep's workspace
    gp = [torch.empty_like(t).data_ptr() for t in lv]
    with pytest.raises(binding.TNError):
        binding.tn_contract_grad_instances(tnw.h, pairs, [], 0, B, strides, adjs.data_ptr(), binding.TN_MEM_DEVICE,
                                           0, 0, gp, binding.TN_GRAD_KEPT_FORWARD,
                                           torch.cuda.current_stream().cuda_stream)
    got = [g.cpu().numpy() for g in tnw.grad_instances(pairs, [], "fp32", B, strides, adjs, kept_forward=token)]
    for a, b in zip(got, ref):
        assert np.array_equal(a, b)
    tnw.close()


@pytest.mark.parametrize("parts", [2, 3])
def test_slice_ranges_sum_to_the_full_gradient(torch, parts):
    """Gradients over disjoint slice ranges (as ranks sharing the slices
    compute them) add up to the gradient over all slices."""
    from paper_2002_01935_gb300 import shard
    net, pairs, sliced, ts, tnw = _setup(torch, seed=31, sliced_n=3)
    d = int(np.prod([net.dims[l] for l in sliced]))
    adj = _adjoint(net, 9)
    full = [g.cpu().numpy() for g in tnw.grad(pairs, sliced, "fp32", adj)]
    acc = [np.zeros_like(g) for g in full]
    for r in range(parts):
        b, cnt = shard.slice_range(r, parts, d)
        part = tnw.grad(pairs, sliced, "fp32", adj, slice_begin=b, slice_count=cnt)
        for a, g in zip(acc, part):
            a += g.cpu().numpy()
    for a, f in zip(acc, full):
        assert np.linalg.norm(a - f) <= 1e-6 * (np.linalg.norm(f) + 1e-30)
    from paper_2002_01935_gb300 import binding
    with pytest.raises(binding.TNError):
        tnw.grad(pairs, sliced, "fp32", adj, slice_begin=d - 1, slice_count=2)
    tnw.close()


def test_keep_forward_refuses_open_outputs(torch):
    """The keeping forward serves scalar networks (one value per copy)."""
    from paper_2002_01935_gb300 import binding
    net, pairs, sliced, ts, tnw = _setup(torch, seed=41, n_open=1)
    lv = list(ts)
    strides = [0] * len(ts)
    lv[0] = torch.stack([ts[0], ts[0]])
    strides[0] = ts[0].numel()
    tnw.set_tensors(lv)
    with pytest.raises(binding.TNError):
        tnw.contract_instances_keep(pairs, "fp32", 2, strides)
    tnw.close()


def test_single_tensor_network_gradient(torch):
    """A network of one tensor: its value is the sum of its entries over the
    summed labels, the gradient of a leaf is conj(adjoint) broadcast."""
    from paper_2002_01935_gb300 import binding
    rng = np.random.default_rng(3)
    t = (rng.standard_normal((2, 2, 2)) + 1j * rng.standard_normal((2, 2, 2))).astype(np.complex64)
    labels, dims = [[1, 2, 3]], {1: 2, 2: 2, 3: 2}
    tt = torch.from_numpy(t).cuda()
    tnw = binding.TensorNetwork(labels, dims, [2], [tt], complex_=True)
    adj = np.array([0.5 - 1.0j, 2.0 + 0.25j])
    g = tnw.grad([], [], "fp32", adj)[0].cpu().numpy()
    # value[o] = sum over a, c of T[a, o, c]: d value[o] / d T[a, o, c] = 1, so
    # the gradient (conj(derivative) * adjoint) is adj[o] along every a, c
    ref = np.broadcast_to(adj[None, :, None], (2, 2, 2))
    assert np.allclose(g, ref, rtol=1e-6, atol=1e-6)
    tnw.close()


@pytest.mark.parametrize("parts", [2])
def test_grad_instances_slice_ranges(torch, parts):
    """Copies and slice ranges together: the ranges add up to the full sweep."""
    from paper_2002_01935_gb300 import shard
    net, pairs, sliced, ts, tnw = _setup(torch, seed=42, n_open=0, sliced_n=2)
    B = 3
    lv = list(ts)
    strides = [0] * len(ts)
    lv[2] = torch.stack([ts[2] * np.float32(1.0 + 0.1 * i) for i in range(B)])
    strides[2] = ts[2].numel()
    tnw.set_tensors(lv)
    adjs = torch.from_numpy(np.array([1.0 + 0.5j, -0.5 + 0.25j, 0.75 - 1.0j])).cuda()
    d = int(np.prod([net.dims[l] for l in sliced]))
    full = [g.cpu().numpy() for g in tnw.grad_instances(pairs, sliced, "fp32", B, strides, adjs)]
    acc = [np.zeros_like(g) for g in full]
    for r in range(parts):
        b, cnt = shard.slice_range(r, parts, d)
        part = tnw.grad_instances(pairs, sliced, "fp32", B, strides, adjs, slice_begin=b, slice_count=cnt)
        for a, g in zip(acc, part):
            a += g.cpu().numpy()
    for a, f in zip(acc, full):
        assert np.linalg.norm(a - f) <= 1e-6 * (np.linalg.norm(f) + 1e-30)
    tnw.close()
