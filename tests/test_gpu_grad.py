"""Reverse-mode gradients (tn_contract_grad) against the FP64 oracle.

Leaf gradients follow torch's convention, conj(d value / d T_v) * adjoint,
summed over slices and open labels.  The oracle's derivative of a
multilinear network is the contraction of the network without T_v (its
environment); open outputs are closed with conj(adjoint) first.
Tolerance: 1e-5 of the cancellation-free scale for FP32 arithmetic.
"""
import math

import numpy as np
import pytest

from oracle import gradient, statevector, tree
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


def tree_fn(l, d, o):
    return planner.greedy_tree(l, d, o)


def oracle_leaf_grads(net, adj):
    """conj(d s / d T_v) for s = sum_o value[o] conj(adj[o])."""
    ts, ls = list(net.tensors), [list(x) for x in net.labels]
    if net.open:
        ts.append(np.conj(np.asarray(adj)))
        ls.append(list(net.open))
    else:
        ts.append(np.array(np.conj(adj)))
        ls.append([])
    out = []
    for v in range(net.n_tensors):
        env = gradient.environment(ts, ls, net.dims, v, tree_fn)
        out.append(np.conj(env))
    return out


def gpu_grads(torch, net, pairs, sliced, adj, mode="fp32"):
    from paper_2002_01935_gb300 import binding
    cplx = net.is_complex
    dt = torch.complex64 if cplx else torch.float32
    ts = [torch.from_numpy(np.array(t, order="C")).to(dt).contiguous().cuda() for t in net.tensors]
    tnw = binding.TensorNetwork(net.labels, net.dims, net.open, ts, complex_=cplx)
    try:
        gs = tnw.grad(pairs, sliced, mode, adj)
        torch.cuda.synchronize()
        return [g.cpu().numpy() for g in gs]
    finally:
        tnw.close()


@pytest.mark.parametrize("seed", range(10))
def test_leaf_grads_random_networks(torch, seed):
    net = inputs.random_network(6 + seed % 3, 10 + seed % 4, 700 + seed, n_open=seed % 3,
                                complex_=seed % 2 == 0)
    pairs = planner.greedy_tree(net.labels, net.dims, net.open)
    rng = np.random.default_rng(seed)
    shape = tuple(net.dims[l] for l in net.open)
    adj = rng.standard_normal(shape)
    if net.is_complex:
        adj = adj + 1j * rng.standard_normal(shape)
    sliced = []
    if seed >= 5:
        summed = [l for l in sorted(net.dims) if l not in net.open]
        sliced = summed[:2]
    got = gpu_grads(torch, net, pairs, sliced, adj)
    ref = oracle_leaf_grads(net, adj)
    absnet = net.with_tensors([np.abs(t) for t in net.tensors])
    scale = oracle_leaf_grads(absnet, np.abs(adj))
    for v in range(net.n_tensors):
        assert got[v].shape == ref[v].shape
        assert np.all(np.abs(got[v] - ref[v]) <= 1e-5 * np.abs(scale[v]) + 1e-30), v


@pytest.mark.parametrize("mode", ["fp32", "tf32_split"])
def test_circuit_leaf_grads_against_environments(torch, mode):
    circ = inputs.random_circuit(3, 3, 6, seed=4)
    bs = inputs.random_bitstrings(9, 1, seed=5)[0]
    net = inputs.circuit_network(circ, bs)
    pairs = planner.greedy_tree(net.labels, net.dims, net.open)
    c = complex(tree.value(net.tensors, net.labels, net.dims, net.open, pairs))
    adj = np.array(1.0 / np.conj(c))  # d ln|c|^2 / d conj(c)
    got = gpu_grads(torch, net, pairs, [], adj, mode)
    stored = net.as_stored()  # the leaf values the GPU reads
    for v in [0, 10, 20, net.meta["gate_leaf"][circ.fsim_gates()[0]], net.n_tensors - 1]:
        env = gradient.environment(stored.tensors, stored.labels, stored.dims, v, tree_fn)
        ref = np.conj(env) * adj
        assert np.linalg.norm(got[v] - ref) <= 1e-5 * np.linalg.norm(ref), v


def fsim_torch(torch, theta, phi):
    c, s = torch.cos(theta), torch.sin(theta)
    z = torch.zeros((), dtype=torch.complex128, device=theta.device)
    one = torch.ones((), dtype=torch.complex128, device=theta.device)
    ms = -1j * s.to(torch.complex128)
    cc = c.to(torch.complex128)
    ph = torch.exp(-1j * phi.to(torch.complex128))
    rows = [torch.stack([one, z, z, z]), torch.stack([z, cc, ms, z]),
            torch.stack([z, ms, cc, z]), torch.stack([z, z, z, ph])]
    return torch.stack(rows)


def test_cfg3_fsim_parameter_gradients(torch):
    """5x4 grid, 12 cycles, 64 seeded bitstrings, L = mean ln|c_x|^2, the
    (theta, phi) of every fSim as torch parameters; gradients through the
    autograd Function (GPU reverse sweep) against central differences of
    the FP64 state vector (h = 1e-3) on a sample of parameters."""
    from paper_2002_01935_gb300 import autograd, binding
    R, C, T = 5, 4, 12
    circ = inputs.random_circuit(R, C, T, seed=0)
    bits = inputs.random_bitstrings(R * C, 64, seed=1000)
    fs = circ.fsim_gates()
    assert len(fs) == 93
    theta = torch.tensor([circ.gates[g].params[0] for g in fs], dtype=torch.float64, device="cuda",
                         requires_grad=True)
    phi = torch.tensor([circ.gates[g].params[1] for g in fs], dtype=torch.float64, device="cuda",
                       requires_grad=True)
    net0 = inputs.circuit_network(circ, bits[0])
    pairs = planner.greedy_tree(net0.labels, net0.dims, net0.open)
    tnw = binding.TensorNetwork(net0.labels, net0.dims, net0.open, None, complex_=True)
    leaf_of = {g: net0.meta["gate_leaf"][g] for g in fs}
    loss = 0.0
    for x in bits:
        net = inputs.circuit_network(circ, x)
        leaves = [torch.from_numpy(np.array(t, order="C")).to(torch.complex64).cuda()
                  for t in net.tensors]
        for i, g in enumerate(fs):
            leaves[leaf_of[g]] = fsim_torch(torch, theta[i], phi[i]).to(torch.complex64).reshape(2, 2, 2, 2)
        c = autograd.contract(tnw, pairs, [], "fp32", *leaves)
        loss = loss + torch.log(torch.abs(c) ** 2) / len(bits)
    loss.backward()
    g_theta, g_phi = theta.grad.cpu().numpy(), phi.grad.cpu().numpy()
    tnw.close()

    def loss_sv(th, ph):
        gates = [inputs.Gate(g.name, g.qubits, g.matrix, g.params) for g in circ.gates]
        for i, gi in enumerate(fs):
            gates[gi] = inputs.Gate("fsim", gates[gi].qubits, inputs.fsim(th[i], ph[i]), (th[i], ph[i]))
        psi = statevector.final_state(R * C, gates)
        return float(np.mean([math.log(abs(psi[tuple(x)]) ** 2) for x in bits]))

    th0 = np.array([circ.gates[g].params[0] for g in fs])
    ph0 = np.array([circ.gates[g].params[1] for g in fs])
    h = 1e-3
    scale = max(np.max(np.abs(g_theta)), np.max(np.abs(g_phi)))
    for i in (0, 31, 92):
        for which, gvec in ((0, g_theta), (1, g_phi)):
            p_plus = [th0.copy(), ph0.copy()]
            p_minus = [th0.copy(), ph0.copy()]
            p_plus[which][i] += h
            p_minus[which][i] -= h
            fd = (loss_sv(*p_plus) - loss_sv(*p_minus)) / (2 * h)
            assert abs(gvec[i] - fd) <= 2e-3 * scale, (i, which, gvec[i], fd)


def _fsim_stack(torch, theta, phi):
    n = theta.shape[0]
    c, s = torch.cos(theta).to(torch.complex128), torch.sin(theta).to(torch.complex128)
    g = torch.zeros((n, 4, 4), dtype=torch.complex128, device=theta.device)
    g[:, 0, 0] = 1
    g[:, 1, 1] = c
    g[:, 2, 2] = c
    g[:, 1, 2] = -1j * s
    g[:, 2, 1] = -1j * s
    g[:, 3, 3] = torch.exp(-1j * phi.to(torch.complex128))
    return g.to(torch.complex64).reshape(n, 2, 2, 2, 2)


@pytest.mark.parametrize("mode", ["fp32", "tf32_split", "fp16_split"])
def test_cfg3_all_fsim_gradients_against_adjoint_state(torch, mode):
    """All 186 fSim parameters of the 5x4, 12-cycle circuit, L = mean over
    64 seeded bitstrings of ln|c_x|^2, through the batched autograd Function
    (one forward for the 64 copies, one reverse sweep): the gradient vector
    against the state-vector adjoint gradient of the same L (gates as the
    GPU reads them, complex64; their derivatives exact), norm-relative."""
    from paper_2002_01935_gb300 import autograd, binding
    R, C, T = 5, 4, 12
    circ = inputs.random_circuit(R, C, T, seed=0)
    bits = inputs.random_bitstrings(R * C, 64, seed=1000)
    fs = circ.fsim_gates()
    nets = [inputs.circuit_network(circ, b) for b in bits]
    net0 = nets[0]
    pairs = planner.greedy_tree(net0.labels, net0.dims, net0.open)
    n = net0.n_tensors
    first_out = n - R * C
    base = [torch.from_numpy(np.array(t, order="C")).to(torch.complex64).cuda() for t in net0.tensors]
    outs = torch.stack([torch.stack([torch.from_numpy(np.array(nt.tensors[v], order="C")).to(torch.complex64)
                                     for v in range(first_out, n)]) for nt in nets]).cuda()
    batch = {first_out + q: outs[:, q].contiguous() for q in range(R * C)}
    leaf_of = [net0.meta["gate_leaf"][g] for g in fs]
    theta = torch.tensor([circ.gates[g].params[0] for g in fs], dtype=torch.float64, device="cuda",
                         requires_grad=True)
    phi = torch.tensor([circ.gates[g].params[1] for g in fs], dtype=torch.float64, device="cuda",
                       requires_grad=True)
    tnw = binding.TensorNetwork(net0.labels, net0.dims, net0.open, base, complex_=True)
    try:
        G = _fsim_stack(torch, theta, phi)
        leaves = list(base)
        for i, v in enumerate(leaf_of):
            leaves[v] = G[i]
        vals = autograd.contract_batch(tnw, pairs, mode, leaves[:first_out] + [None] * (R * C), batch)
        loss = torch.mean(torch.log(torch.abs(vals) ** 2))
        loss.backward()
        got = np.concatenate([theta.grad.cpu().numpy(), phi.grad.cpu().numpy()])
        got_loss = float(loss.detach().cpu())
    finally:
        tnw.close()
    gates = [inputs.Gate(g.name, g.qubits, np.asarray(g.matrix).astype(np.complex64).astype(np.complex128),
                         g.params) for g in circ.gates]
    dg = {g: list(statevector.fsim_derivatives(*circ.gates[g].params)) for g in fs}
    L, grads = statevector.mean_log_prob_grad(R * C, gates, bits, dg)
    ref = np.concatenate([[grads[g][0] for g in fs], [grads[g][1] for g in fs]])
    assert abs(got_loss - L) <= 1e-5 * abs(L)
    err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    assert err <= 1e-5, err
