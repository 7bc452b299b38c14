"""Seeded synthetic tensor networks: random quantum circuits and Ising models.

This module only *builds* inputs (tensor entries, index labels, open labels).
It holds none of the contraction arithmetic, so both the GPU executor and the
CPU oracle can consume what it produces without sharing any method code.

Workloads follow the paper's benchmark families:

* random-circuit transition amplitudes c_x = <x| U_d ... U_1 |0^N> (Sec. 4.6,
  Eq. trans-amp), on a rows x cols square grid with single-qubit gates drawn
  from {sqrt(X), sqrt(Y), sqrt(W)} and fSim entangling gates (Sec. 4.6.2);
  the circuit network holds rank-1 input/output states, rank-2 single-qubit
  gates and rank-4 two-qubit gates (Sec. 4.6.1);
* classical Ising partition functions on random 3-regular graphs (the graph
  family of Sec. 4.1), one COPY tensor per vertex and one Boltzmann matrix per
  edge, i.e. the "vertex" form of a spin-model network (Sec. 4.3).

Readings of points the paper leaves open (gate matrices, coupler patterns,
axis order, RNG) are fixed here and listed with the design notes:
sqrt(G) = (I - iG)/sqrt(2); fSim(theta, phi) in the |ab> basis with qubit a
most significant; pattern t mod 4 over {A,B,C,D}; gate tensors g[out, in] and
G[out_a, out_b, in_a, in_b]; spin index 0 -> s=+1, 1 -> s=-1; PCG64 seeds.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Dict, List, Optional, Sequence, Tuple

import numpy as np

__all__ = [
    "Network",
    "Circuit",
    "Gate",
    "gate_matrix",
    "fsim",
    "random_circuit",
    "random_bitstrings",
    "circuit_network",
    "random_regular_graph",
    "ising_network",
    "random_network",
]


# ---------------------------------------------------------------------------
# Network container
# ---------------------------------------------------------------------------

@dataclasses.dataclass
class Network:
    """A tensor network in the paper's Sec. 2 form.

    ``tensors[v]`` is T_v, an ndarray whose axes follow the ordered index
    tuple ``labels[v]`` (t_v).  ``dims[e]`` is w(e) for label e.  ``open``
    lists the labels left uncontracted, in the order of the output tensor.
    A label shared by more than two tensors is a hyperedge (Sec. 3.5).
    """

    tensors: List[np.ndarray]
    labels: List[List[int]]
    dims: Dict[int, int]
    open: List[int] = dataclasses.field(default_factory=list)
    meta: dict = dataclasses.field(default_factory=dict)

    @property
    def n_tensors(self) -> int:
        return len(self.tensors)

    @property
    def is_complex(self) -> bool:
        return any(np.iscomplexobj(t) for t in self.tensors)

    def label_ids(self) -> List[int]:
        return sorted(self.dims)

    def flat_labels(self) -> List[int]:
        return [l for ls in self.labels for l in ls]

    def ranks(self) -> List[int]:
        return [len(ls) for ls in self.labels]

    def validate(self) -> None:
        for v, (t, ls) in enumerate(zip(self.tensors, self.labels)):
            if t.ndim != len(ls):
                raise ValueError(f"tensor {v}: ndim {t.ndim} != rank {len(ls)}")
            if len(set(ls)) != len(ls):
                raise ValueError(f"tensor {v}: repeated label")
            for ax, l in enumerate(ls):
                if t.shape[ax] != self.dims[l]:
                    raise ValueError(f"tensor {v}: axis {ax} dim mismatch")

    def with_tensors(self, tensors: Sequence[np.ndarray]) -> "Network":
        return dataclasses.replace(self, tensors=list(tensors))

    def as_stored(self) -> "Network":
        """The same network with every entry rounded to the storage type of
        the GPU leaves (complex64, or float32 for a real network) and
        widened back to complex128 / float64: the exact values a device
        contraction reads, so that a reference computed on them compares
        arithmetic with arithmetic, without the rounding of the inputs."""
        cplx = self.is_complex
        narrow, wide = (np.complex64, np.complex128) if cplx else (np.float32, np.float64)
        return self.with_tensors([np.asarray(t).astype(narrow).astype(wide) for t in self.tensors])


# ---------------------------------------------------------------------------
# Random quantum circuits (Sec. 4.6)
# ---------------------------------------------------------------------------

_SQ2 = 1.0 / math.sqrt(2.0)
_PAULI = {
    "X": np.array([[0, 1], [1, 0]], dtype=np.complex128),
    "Y": np.array([[0, -1j], [1j, 0]], dtype=np.complex128),
}
_PAULI["W"] = (_PAULI["X"] + _PAULI["Y"]) * _SQ2
_ONE_QUBIT = ("sqrt_x", "sqrt_y", "sqrt_w")


def gate_matrix(name: str) -> np.ndarray:
    """sqrt(G) := (I - iG)/sqrt(2) for G in {X, Y, W}; W = (X+Y)/sqrt(2).

    Matrix convention g[out, in]."""
    g = _PAULI[name[-1].upper()]
    return (np.eye(2, dtype=np.complex128) - 1j * g) * _SQ2


def fsim(theta: float, phi: float) -> np.ndarray:
    """fSim(theta, phi) as a 4x4 matrix in the basis |00>,|01>,|10>,|11>
    (first qubit most significant)."""
    c, s = math.cos(theta), math.sin(theta)
    m = np.zeros((4, 4), dtype=np.complex128)
    m[0, 0] = 1.0
    m[1, 1] = c
    m[1, 2] = -1j * s
    m[2, 1] = -1j * s
    m[2, 2] = c
    m[3, 3] = complex(math.cos(phi), -math.sin(phi))
    return m


@dataclasses.dataclass
class Gate:
    name: str                       # "sqrt_x" | "sqrt_y" | "sqrt_w" | "fsim"
    qubits: Tuple[int, ...]
    matrix: np.ndarray              # 2x2 or 4x4, [out, in]
    params: Tuple[float, ...] = ()  # (theta, phi) for fsim


@dataclasses.dataclass
class Circuit:
    rows: int
    cols: int
    cycles: int
    seed: int
    gates: List[Gate]

    @property
    def n_qubits(self) -> int:
        return self.rows * self.cols

    def fsim_gates(self) -> List[int]:
        return [i for i, g in enumerate(self.gates) if g.name == "fsim"]


def coupler_pairs(rows: int, cols: int, pattern: str) -> List[Tuple[int, int]]:
    """Nearest-neighbour coupler pattern on a rows x cols grid, qubit r*cols+c.

    A: horizontal (r,c)-(r,c+1) with c even;  B: horizontal with c odd;
    C: vertical (r,c)-(r+1,c) with r even;    D: vertical with r odd.
    """
    out = []
    if pattern in "AB":
        par = 0 if pattern == "A" else 1
        for r in range(rows):
            for c in range(par, cols - 1, 2):
                out.append((r * cols + c, r * cols + c + 1))
    elif pattern in "CD":
        par = 0 if pattern == "C" else 1
        for r in range(par, rows - 1, 2):
            for c in range(cols):
                out.append((r * cols + c, (r + 1) * cols + c))
    else:
        raise ValueError(pattern)
    return out


def random_circuit(rows: int, cols: int, cycles: int, seed: int) -> Circuit:
    """Random circuit: each cycle puts a single-qubit gate on every qubit
    (uniform over the three, never the qubit's previous gate), then fSim with
    independent theta~U(0,pi/2), phi~U(0,pi) on pattern [A,B,C,D][t mod 4]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    n = rows * cols
    prev: List[Optional[str]] = [None] * n
    gates: List[Gate] = []
    for t in range(cycles):
        for q in range(n):
            choices = [g for g in _ONE_QUBIT if g != prev[q]]
            name = choices[int(rng.integers(len(choices)))]
            prev[q] = name
            gates.append(Gate(name, (q,), gate_matrix(name)))
        for a, b in coupler_pairs(rows, cols, "ABCD"[t % 4]):
            theta = float(rng.uniform(0.0, math.pi / 2))
            phi = float(rng.uniform(0.0, math.pi))
            gates.append(Gate("fsim", (a, b), fsim(theta, phi), (theta, phi)))
    return Circuit(rows, cols, cycles, seed, gates)


def random_bitstrings(n_qubits: int, count: int, seed: int) -> np.ndarray:
    """Seeded uniform random output bitstrings, shape (count, n_qubits)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.integers(0, 2, size=(count, n_qubits)).astype(np.int8)


def circuit_network(circuit: Circuit, bitstring: Optional[Sequence[int]] = None,
                    open_qubits: Sequence[int] = (),
                    gate_overrides: Optional[Dict[int, np.ndarray]] = None) -> Network:
    """Tensor network of <x| U |0^N> (Eq. trans-amp).

    Leaves, in order: N input states |0> (rank 1), then the gates in time
    order (rank 2: g[out,in]; rank 4: G[out_a,out_b,in_a,in_b]), then one
    output state <x_q| (rank 1) per qubit not in ``open_qubits``.  The final
    wire labels of ``open_qubits`` are left open, in that order.
    ``gate_overrides`` maps a gate index to a replacement matrix (used to
    perturb fSim parameters for finite differences).
    """
    n = circuit.n_qubits
    if bitstring is None:
        bitstring = [0] * n
    next_label = 0
    wire = [0] * n
    tensors: List[np.ndarray] = []
    labels: List[List[int]] = []
    for q in range(n):
        wire[q] = next_label
        next_label += 1
        tensors.append(np.array([1.0, 0.0], dtype=np.complex128))
        labels.append([wire[q]])
    gate_leaf: List[int] = []
    for gi, g in enumerate(circuit.gates):
        m = g.matrix if gate_overrides is None or gi not in gate_overrides else gate_overrides[gi]
        gate_leaf.append(len(tensors))
        if len(g.qubits) == 1:
            (q,) = g.qubits
            out = next_label
            next_label += 1
            tensors.append(np.array(m, dtype=np.complex128).reshape(2, 2))
            labels.append([out, wire[q]])
            wire[q] = out
        else:
            a, b = g.qubits
            oa, ob = next_label, next_label + 1
            next_label += 2
            tensors.append(np.array(m, dtype=np.complex128).reshape(2, 2, 2, 2))
            labels.append([oa, ob, wire[a], wire[b]])
            wire[a], wire[b] = oa, ob
    open_set = set(open_qubits)
    for q in range(n):
        if q in open_set:
            continue
        e = np.zeros(2, dtype=np.complex128)
        e[int(bitstring[q])] = 1.0
        tensors.append(e)
        labels.append([wire[q]])
    dims = {l: 2 for l in range(next_label)}
    net = Network(tensors, labels, dims, [wire[q] for q in open_qubits],
                  meta={"kind": "circuit", "gate_leaf": gate_leaf,
                        "n_qubits": n, "bitstring": list(map(int, bitstring))})
    net.validate()
    return net


# ---------------------------------------------------------------------------
# Ising partition functions on random regular graphs (Sec. 4.1, 4.3)
# ---------------------------------------------------------------------------

def random_regular_graph(n: int, degree: int, seed: int, max_tries: int = 10000
                         ) -> List[Tuple[int, int]]:
    """Uniform simple d-regular graph by the pairing (configuration) model
    with rejection of self-loops and multi-edges."""
    if (n * degree) % 2:
        raise ValueError("n*degree must be even")
    rng = np.random.Generator(np.random.PCG64(seed))
    stubs = np.repeat(np.arange(n), degree)
    for _ in range(max_tries):
        perm = rng.permutation(stubs)
        pairs = perm.reshape(-1, 2)
        if np.any(pairs[:, 0] == pairs[:, 1]):
            continue
        canon = {(int(min(a, b)), int(max(a, b))) for a, b in pairs}
        if len(canon) != len(pairs):
            continue
        return sorted(canon)
    raise RuntimeError("no simple regular graph found")


def ising_couplings(n_edges: int, seed: int) -> np.ndarray:
    """J_e = +1 or -1 with probability 1/2 each, independently."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return np.where(rng.integers(0, 2, size=n_edges) == 0, 1.0, -1.0)


def ising_network(n_vertices: int, edges: Sequence[Tuple[int, int]], J: Sequence[float],
                  beta: float) -> Network:
    """Vertex-form network of Z = sum_s exp(beta * sum_e J_e s_u s_v).

    Vertex v carries a COPY tensor delta over one label per incident edge;
    edge e=(u,v) carries M_e[a,b] = exp(beta J_e s(a) s(b)) with s(0)=+1,
    s(1)=-1.  Label of the (edge e, endpoint side k) stub is 2e+k.
    Leaves: the n_vertices COPY tensors first, then the edge matrices.
    """
    inc: List[List[int]] = [[] for _ in range(n_vertices)]
    for ei, (u, v) in enumerate(edges):
        inc[u].append(2 * ei)
        inc[v].append(2 * ei + 1)
    tensors: List[np.ndarray] = []
    labels: List[List[int]] = []
    for v in range(n_vertices):
        d = len(inc[v])
        t = np.zeros((2,) * d, dtype=np.float64)
        t[(0,) * d] = 1.0
        t[(1,) * d] = 1.0
        tensors.append(t)
        labels.append(list(inc[v]))
    spin = np.array([1.0, -1.0])
    for ei, (u, v) in enumerate(edges):
        m = np.exp(beta * float(J[ei]) * np.outer(spin, spin))
        tensors.append(m)
        labels.append([2 * ei, 2 * ei + 1])
    dims = {l: 2 for ls in labels for l in ls}
    net = Network(tensors, labels, dims, [],
                  meta={"kind": "ising", "edges": [tuple(e) for e in edges],
                        "J": [float(j) for j in J], "beta": beta, "n": n_vertices})
    net.validate()
    return net


def random_ising(n_vertices: int, seed: int, beta: float = 0.3, degree: int = 3) -> Network:
    edges = random_regular_graph(n_vertices, degree, seed)
    J = ising_couplings(len(edges), seed + 1_000_003)
    return ising_network(n_vertices, edges, J, beta)


def ising_hyper_network(n_vertices: int, edges: Sequence[Tuple[int, int]], J: Sequence[float],
                        beta: float) -> Network:
    """Hyperedge form of the same Z (Sec. 3.5: a COPY tensor is a hyperedge):
    the spin of vertex v is one label (id v) shared by the matrices of all
    its edges, M_e[s_u, s_v] = exp(beta J_e s(a) s(b)) over labels (u, v); a
    vertex without edges gets a vector of ones.  Leaves: the edge matrices
    in edge order, then those vectors."""
    spin = np.array([1.0, -1.0])
    tensors: List[np.ndarray] = []
    labels: List[List[int]] = []
    deg = [0] * n_vertices
    for ei, (u, v) in enumerate(edges):
        tensors.append(np.exp(beta * float(J[ei]) * np.outer(spin, spin)))
        labels.append([int(u), int(v)])
        deg[u] += 1
        deg[v] += 1
    for v in range(n_vertices):
        if deg[v] == 0:
            tensors.append(np.ones(2))
            labels.append([v])
    dims = {v: 2 for v in range(n_vertices)}
    net = Network(tensors, labels, dims, [],
                  meta={"kind": "ising_hyper", "edges": [tuple(e) for e in edges],
                        "J": [float(j) for j in J], "beta": beta, "n": n_vertices})
    net.validate()
    return net


def random_ising_hyper(n_vertices: int, seed: int, beta: float = 0.3, degree: int = 3) -> Network:
    """random_ising's graph and couplings (same seed) in the hyperedge form."""
    edges = random_regular_graph(n_vertices, degree, seed)
    J = ising_couplings(len(edges), seed + 1_000_003)
    return ising_hyper_network(n_vertices, edges, J, beta)


# ---------------------------------------------------------------------------
# Small random networks for brute-force checks
# ---------------------------------------------------------------------------

def random_network(n_tensors: int, n_labels: int, seed: int, *, max_rank: int = 4,
                   max_dim: int = 3, n_open: int = 0, hyper: bool = True,
                   complex_: bool = True, allow_dangling: bool = True) -> Network:
    """Random small network: random label dims in [1, max_dim], each label
    placed in 1..4 tensors (hyperedges when >2), some labels open.  Used to
    pin contraction semantics against the nested sum of products."""
    rng = np.random.Generator(np.random.PCG64(seed))
    dims = {l: int(rng.integers(1, max_dim + 1)) for l in range(n_labels)}
    labels: List[List[int]] = [[] for _ in range(n_tensors)]
    for l in range(n_labels):
        hi = 4 if hyper else 2
        lo = 1 if allow_dangling else 2
        k = int(rng.integers(lo, hi + 1))
        k = min(k, n_tensors)
        owners = rng.choice(n_tensors, size=k, replace=False)
        for v in owners:
            if len(labels[v]) < max_rank:
                labels[v].append(l)
    used = sorted({l for ls in labels for l in ls})
    dims = {l: dims[l] for l in used}
    for ls in labels:
        rng.shuffle(ls)
    open_labels = [int(x) for x in rng.choice(used, size=min(n_open, len(used)), replace=False)] if n_open else []
    tensors = []
    for ls in labels:
        shape = tuple(dims[l] for l in ls)
        t = rng.standard_normal(shape)
        if complex_:
            t = t + 1j * rng.standard_normal(shape)
        tensors.append(np.asarray(t))
    net = Network(tensors, labels, dims, open_labels, meta={"kind": "random", "seed": seed})
    net.validate()
    return net
