"""Host-side contraction planner: tree, slicing and cost model.

The paper's subject is the search for good contraction trees; here only a
plain deterministic planner is kept, whose output (a tree and a set of sliced
labels) is what the GPU executor runs.

* Tree encoding (Sec. 2): leaves are ids 0..n-1, internal node n+i has
  children ``pairs[i]``; every id is used once, the root is last.
* Node incidence (Sec. 2, Eq. incidence) generalised to open labels and
  hyperedges: a node keeps a label iff the label is open or occurs in a leaf
  outside the node's subtree.  For a plain graph with no open labels this is
  the symmetric difference s_l (+) s_r of the paper.
* Width W = max_v sum_{e in s_v} log2 w(e)   (Eq. edgecon; leaves included)
  Cost  C = sum_v 2^{vc(v)}, vc = sum_{e in s_l u s_r} log2 w(e)
  (Eq. vertexcon; summed over contraction vertices).  FLOPs = 8C complex,
  2C real (Sec. 2, text after Eq. vertexcon).
* Greedy tree (Sec. 3.4, Eq. greedy-cost-function, Eq. greedy-boltzmann-factor):
  cost(i,j) = size(k) - alpha (size(i)+size(j)); tau = 0 picks the minimum,
  ties broken by the smallest (min id, max id); only pairs sharing a label
  are candidates; when none remain the two smallest tensors are joined by an
  outer product.  tau > 0 samples pairs with weight exp(-cost/tau).
* Slicing (Sec. 4.7.1): greedily remove the summed label that minimises the
  total sliced cost C_s = d_sliced * C(sliced tree) until the sliced width
  reaches the target.
"""
from __future__ import annotations

import dataclasses
import heapq
import math
from typing import Dict, Iterable, List, Optional, Sequence, Set, Tuple

import numpy as np

__all__ = [
    "TreeInfo",
    "greedy_tree_sampled",
    "hyper_greedy",
    "slice_repeats",
    "node_labels",
    "tree_info",
    "greedy_tree",
    "left_deep_tree",
    "slice_greedy",
    "plan",
    "validate_tree",
    "structure_fingerprint",
    "save_tree",
    "load_tree",
]


def validate_tree(n_leaves: int, pairs: Sequence[Tuple[int, int]]) -> None:
    """SSA tree checks: n-1 pairs for n>=1 leaves, ids < own id, each id used once."""
    if n_leaves < 1:
        raise ValueError("empty network")
    if len(pairs) != n_leaves - 1:
        raise ValueError(f"tree has {len(pairs)} pairs, expected {n_leaves - 1}")
    used = [False] * (2 * n_leaves - 1)
    for i, (a, b) in enumerate(pairs):
        me = n_leaves + i
        for c in (a, b):
            if not (0 <= c < me):
                raise ValueError(f"node {me}: child {c} out of range")
            if used[c]:
                raise ValueError(f"id {c} used twice")
            used[c] = True
        if a == b:
            raise ValueError(f"node {me}: children equal")


def node_labels(leaf_labels: Sequence[Sequence[int]], pairs: Sequence[Tuple[int, int]],
                open_labels: Iterable[int] = (), removed: Iterable[int] = ()
                ) -> List[frozenset]:
    """Incidence set s_v of every tree vertex (leaves first), Eq. incidence
    generalised: keep a label iff it is open or still occurs outside the
    subtree.  Labels in ``removed`` (sliced) are dropped everywhere."""
    rm = set(removed)
    opn = set(open_labels)
    total: Dict[int, int] = {}
    sets: List[frozenset] = []
    sub: List[Dict[int, int]] = []
    for ls in leaf_labels:
        s = frozenset(l for l in ls if l not in rm)
        for l in s:
            total[l] = total.get(l, 0) + 1
        sets.append(s)
        sub.append({l: 1 for l in s})
    for a, b in pairs:
        sa, sb = sets[a], sets[b]
        ca, cb = sub[a], sub[b]
        cnt: Dict[int, int] = {}
        for l in sa | sb:
            c = ca.get(l, 0) + cb.get(l, 0)
            if l in opn or c < total[l]:
                cnt[l] = c
        sets.append(frozenset(cnt))
        sub.append(cnt)
    return sets


@dataclasses.dataclass
class TreeInfo:
    n_leaves: int
    sets: List[frozenset]           # s_v for all tree vertices
    vc: List[float]                 # vertex congestion of internal nodes (log2)
    W: float                        # contraction width (Eq. edgecon)
    C: float                        # contraction cost (Eq. vertexcon), per slice
    d_sliced: int
    sliced: Tuple[int, ...]

    @property
    def C_s(self) -> float:
        return self.d_sliced * self.C

    def flops(self, is_complex: bool) -> float:
        return (8.0 if is_complex else 2.0) * self.C_s

    def node_sizes(self) -> List[float]:
        return []


def _log2w(dims: Dict[int, int], labels: Iterable[int]) -> float:
    return float(sum(math.log2(dims[l]) for l in labels))


def tree_info(leaf_labels: Sequence[Sequence[int]], dims: Dict[int, int],
              pairs: Sequence[Tuple[int, int]], open_labels: Iterable[int] = (),
              sliced: Sequence[int] = ()) -> TreeInfo:
    n = len(leaf_labels)
    validate_tree(n, pairs)
    sets = node_labels(leaf_labels, pairs, open_labels, sliced)
    W = max(_log2w(dims, s) for s in sets)
    vc: List[float] = []
    C = 0.0
    for a, b in pairs:
        v = _log2w(dims, sets[a] | sets[b])
        vc.append(v)
        C += 2.0 ** v
    d = 1
    for l in sliced:
        d *= dims[l]
    return TreeInfo(n, sets, vc, W, C, d, tuple(sliced))


# ---------------------------------------------------------------------------
# Greedy tree (Sec. 3.4)
# ---------------------------------------------------------------------------

def greedy_tree(leaf_labels: Sequence[Sequence[int]], dims: Dict[int, int],
                open_labels: Iterable[int] = (), alpha: float = 1.0, tau: float = 0.0,
                seed: Optional[int] = None) -> List[Tuple[int, int]]:
    """Agglomerative tree by Eq. greedy-cost-function.

    tau == 0: deterministic minimum with (min id, max id) tie break.
    tau > 0: Boltzmann sampling (Eq. greedy-boltzmann-factor), seeded.
    """
    n = len(leaf_labels)
    if n == 1:
        return []
    opn = set(open_labels)
    sets: Dict[int, frozenset] = {}
    users: Dict[int, Set[int]] = {}
    size: Dict[int, int] = {}

    def tsize(s: Iterable[int]) -> int:
        p = 1
        for l in s:
            p *= dims[l]
        return p

    for v, ls in enumerate(leaf_labels):
        sets[v] = frozenset(ls)
        size[v] = tsize(ls)
        for l in ls:
            users.setdefault(l, set()).add(v)

    def out_set(i: int, j: int) -> frozenset:
        keep = []
        for l in sets[i] | sets[j]:
            if l in opn:
                keep.append(l)
                continue
            u = users[l]
            c = (i in u) + (j in u)
            if len(u) > c:
                keep.append(l)
        return frozenset(keep)

    def cost(i: int, j: int) -> float:
        return tsize(out_set(i, j)) - alpha * (size[i] + size[j])

    rng = np.random.Generator(np.random.PCG64(seed if seed is not None else 0))
    alive: Set[int] = set(range(n))
    heap: List[Tuple[float, int, int]] = []
    cand: Set[Tuple[int, int]] = set()

    def push(i: int, j: int) -> None:
        a, b = (i, j) if i < j else (j, i)
        if (a, b) in cand:
            return
        cand.add((a, b))
        heapq.heappush(heap, (cost(a, b), a, b))

    for l, u in users.items():
        us = sorted(u)
        for x in range(len(us)):
            for y in range(x + 1, len(us)):
                push(us[x], us[y])

    pairs: List[Tuple[int, int]] = []
    nxt = n
    while len(alive) > 1:
        choice: Optional[Tuple[int, int]] = None
        if tau > 0.0:
            live = [(c, a, b) for (c, a, b) in heap if a in alive and b in alive]
            heap = live
            heapq.heapify(heap)
            if live:
                cs = np.array([c for c, _, _ in live], dtype=np.float64)
                w = np.exp(-(cs - cs.min()) / tau)
                k = int(rng.choice(len(live), p=w / w.sum()))
                _, a, b = live[k]
                choice = (a, b)
                heap.remove(live[k])
                heapq.heapify(heap)
        else:
            while heap:
                c, a, b = heapq.heappop(heap)
                if a in alive and b in alive:
                    choice = (a, b)
                    break
        if choice is None:
            # disconnected components: outer product of the two smallest
            ordered = sorted(alive, key=lambda v: (size[v], v))
            a, b = sorted(ordered[:2])
            choice = (a, b)
        a, b = choice
        s = out_set(a, b)
        k = nxt
        nxt += 1
        pairs.append((a, b))
        for l in sets[a] | sets[b]:
            u = users[l]
            u.discard(a)
            u.discard(b)
            if l in s:
                u.add(k)
        alive.discard(a)
        alive.discard(b)
        sets[k] = s
        size[k] = tsize(s)
        alive.add(k)
        nbrs: Set[int] = set()
        for l in s:
            nbrs |= users[l]
        nbrs.discard(k)
        for m in sorted(nbrs):
            push(m, k)
    return pairs


def greedy_tree_sampled(leaf_labels: Sequence[Sequence[int]], dims: Dict[int, int],
                        open_labels: Iterable[int], alpha: float, tau: float,
                        seed: int) -> List[Tuple[int, int]]:
    """One Boltzmann-sampled greedy tree (Eq. greedy-boltzmann-factor), fast form.

    The cost of Eq. greedy-cost-function spans many orders of magnitude,
    so the temperature acts on sign(c) log2(1 + |c|); each candidate pair
    draws one Gumbel perturbation when it enters the queue (Gumbel-max
    sampling of exp(-cost/tau) among the queued candidates)."""
    n = len(leaf_labels)
    if n == 1:
        return []
    opn = set(open_labels)
    rng = np.random.Generator(np.random.PCG64(seed))
    sets: Dict[int, frozenset] = {}
    users: Dict[int, Set[int]] = {}
    lsz: Dict[int, float] = {}

    def lsize(s: Iterable[int]) -> float:
        return float(sum(math.log2(dims[l]) for l in s))

    for v, ls in enumerate(leaf_labels):
        sets[v] = frozenset(ls)
        lsz[v] = lsize(ls)
        for l in ls:
            users.setdefault(l, set()).add(v)

    def out_set(i: int, j: int) -> frozenset:
        keep = []
        for l in sets[i] | sets[j]:
            if l in opn:
                keep.append(l)
                continue
            u = users[l]
            if len(u) > (i in u) + (j in u):
                keep.append(l)
        return frozenset(keep)

    heap: List[Tuple[float, int, int]] = []
    cand: Set[Tuple[int, int]] = set()
    alive: Set[int] = set(range(n))

    def push(i: int, j: int) -> None:
        a, b = (i, j) if i < j else (j, i)
        if (a, b) in cand:
            return
        cand.add((a, b))
        c = 2.0 ** lsize(out_set(a, b)) - alpha * (2.0 ** lsz[a] + 2.0 ** lsz[b])
        lc = math.copysign(math.log2(1.0 + abs(c)), c)
        g = -math.log(-math.log(rng.random() + 1e-300) + 1e-300)
        heapq.heappush(heap, (lc - tau * g, a, b))

    for l, u in users.items():
        us = sorted(u)
        for x in range(len(us)):
            for y in range(x + 1, len(us)):
                push(us[x], us[y])
    pairs: List[Tuple[int, int]] = []
    nxt = n
    while len(alive) > 1:
        choice = None
        while heap:
            _, a, b = heapq.heappop(heap)
            if a in alive and b in alive:
                choice = (a, b)
                break
        if choice is None:
            ordered = sorted(alive, key=lambda v: (lsz[v], v))
            choice = tuple(sorted(ordered[:2]))
        a, b = choice
        s = out_set(a, b)
        k = nxt
        nxt += 1
        pairs.append((a, b))
        for l in sets[a] | sets[b]:
            u = users[l]
            u.discard(a)
            u.discard(b)
            if l in s:
                u.add(k)
        alive.discard(a)
        alive.discard(b)
        sets[k] = s
        lsz[k] = lsize(s)
        alive.add(k)
        nb: Set[int] = set()
        for l in s:
            nb |= users[l]
        nb.discard(k)
        for m in sorted(nb):
            push(m, k)
    return pairs


def hyper_greedy(leaf_labels: Sequence[Sequence[int]], dims: Dict[int, int],
                 open_labels: Iterable[int] = (), trials: int = 32, seed: int = 0,
                 target_width: Optional[float] = None, slicer_repeats: int = 0):
    """Hyper-Greedy (Sec. 3.4): repeated Boltzmann-sampled greedy trees with
    alpha ~ U(0, 2) and tau ~ logU(0.01, 3), keeping the lowest cost -- the
    sliced cost C_s at target_width when given (slicing inside the search,
    Sec. 4.7.1; with ``slicer_repeats`` > 0 each tree gets the best of that
    many randomised slicer runs besides the greedy one).  Returns (pairs,
    sliced, TreeInfo); seeded."""
    opn = list(open_labels)
    rng = np.random.Generator(np.random.PCG64(seed))
    best = None
    cands = [(1.0, 0.0, None)]
    for t in range(trials):
        cands.append((float(rng.uniform(0.0, 2.0)), float(10 ** rng.uniform(-2, math.log10(3))),
                      int(rng.integers(1 << 31))))
    for alpha, tau, sd in cands:
        if sd is None:
            pairs = greedy_tree(leaf_labels, dims, opn, alpha=1.0)
        else:
            pairs = greedy_tree_sampled(leaf_labels, dims, opn, alpha, tau, sd)
        sliced: List[int] = []
        if target_width is not None:
            info0 = tree_info(leaf_labels, dims, pairs, opn)
            if info0.W > target_width:
                try:
                    sliced = (slice_repeats(leaf_labels, dims, pairs, opn, target_width, slicer_repeats,
                                            seed=seed + 7919 * (sd or 0))
                              if slicer_repeats > 0 else
                              slice_greedy(leaf_labels, dims, pairs, opn, target_width))
                except RuntimeError:
                    continue  # too wide to slice down: not a candidate
        info = tree_info(leaf_labels, dims, pairs, opn, sliced)
        if best is None or info.C_s < best[2].C_s:
            best = (pairs, sliced, info)
    if best is None:
        raise RuntimeError("no sampled tree could be sliced to the target width")
    return best


def left_deep_tree(n_leaves: int, order: Optional[Sequence[int]] = None) -> List[Tuple[int, int]]:
    """((((t0 t1) t2) t3) ...) in the given leaf order."""
    order = list(range(n_leaves)) if order is None else list(order)
    pairs = []
    cur = order[0]
    for i, v in enumerate(order[1:]):
        pairs.append((cur, v))
        cur = n_leaves + i
    return pairs


# ---------------------------------------------------------------------------
# Slicing (Sec. 4.7.1)
# ---------------------------------------------------------------------------

def slice_greedy(leaf_labels: Sequence[Sequence[int]], dims: Dict[int, int],
                 pairs: Sequence[Tuple[int, int]], open_labels: Iterable[int],
                 target_width: float, max_sliced: int = 64, temperature: float = 0.0,
                 rng: Optional[np.random.Generator] = None) -> List[int]:
    """Greedy index slicing to a target sliced width W_s.

    Each step considers the summed labels of tensors wider than the target
    and removes the one minimising d_sliced * C(tree without it); ties go to
    the smallest label id.  Stops when W_s <= target_width.  With a
    temperature > 0 (and ``rng``) each step instead draws a label with
    weight exp(-(log2 score - log2 min score) / temperature): the "slight
    randomization" of the paper's slicer (Sec. 4.7.1), for repeats.
    """
    opn = set(open_labels)
    sliced: List[int] = []
    n = len(leaf_labels)
    while True:
        info = tree_info(leaf_labels, dims, pairs, opn, sliced)
        if info.W <= target_width + 1e-9:
            return sliced
        if len(sliced) >= max_sliced:
            raise RuntimeError("slicing did not reach the target width")
        big = [s for s in info.sets if _log2w(dims, s) > target_width + 1e-9]
        cands = sorted({l for s in big for l in s if l not in opn})
        if not cands:
            raise RuntimeError("only open labels exceed the target width")
        col = {l: i for i, l in enumerate(cands)}
        node_cost = np.array([2.0 ** v for v in info.vc])
        red = np.zeros(len(cands))
        for k, (a, b) in enumerate(pairs):
            u = info.sets[a] | info.sets[b]
            for l in u:
                i = col.get(l)
                if i is not None:
                    red[i] += node_cost[k] * (1.0 - 1.0 / dims[l])
        w = np.array([dims[l] for l in cands], dtype=np.float64)
        score = info.d_sliced * w * (info.C - red)
        if temperature > 0.0 and rng is not None and len(cands) > 1:
            ls = np.log2(np.maximum(score, 1e-300))
            wgt = np.exp(-(ls - ls.min()) / temperature)
            best = int(rng.choice(len(cands), p=wgt / wgt.sum()))
        else:
            best = int(np.flatnonzero(score <= score.min() * (1 + 1e-12))[0])
        sliced.append(cands[best])


def slice_repeats(leaf_labels: Sequence[Sequence[int]], dims: Dict[int, int],
                  pairs: Sequence[Tuple[int, int]], open_labels: Iterable[int],
                  target_width: float, repeats: int = 8, temperature: float = 0.5,
                  seed: int = 0) -> List[int]:
    """The greedy slicer, then ``repeats`` randomised runs of it (seeded),
    keeping the slicing with the lowest sliced cost C_s (Sec. 4.7.1: the
    search targets C_s; W_s <= target for every candidate)."""
    opn = list(open_labels)
    best = slice_greedy(leaf_labels, dims, pairs, opn, target_width)
    best_c = tree_info(leaf_labels, dims, pairs, opn, best).C_s
    rng = np.random.Generator(np.random.PCG64(seed))
    for _ in range(repeats):
        try:
            cand = slice_greedy(leaf_labels, dims, pairs, opn, target_width, temperature=temperature, rng=rng)
        except RuntimeError:
            continue
        c_s = tree_info(leaf_labels, dims, pairs, opn, cand).C_s
        if c_s < best_c:
            best, best_c = cand, c_s
    return best


def plan(net, target_width: Optional[float] = None, alpha: float = 1.0):
    """Greedy tree plus optional slicing for a ``inputs.Network``.

    Returns (pairs, sliced, TreeInfo)."""
    pairs = greedy_tree(net.labels, net.dims, net.open, alpha=alpha)
    sliced: List[int] = []
    if target_width is not None:
        sliced = slice_greedy(net.labels, net.dims, pairs, net.open, target_width)
    info = tree_info(net.labels, net.dims, pairs, net.open, sliced)
    return pairs, sliced, info


# --------------------------------------------------------------------------
# tree files: a tree found once serves every later contraction of networks
# with the same structure (other bitstrings, other runs)
# --------------------------------------------------------------------------

TREE_FORMAT = 1


def structure_fingerprint(leaf_labels: Sequence[Sequence[int]], dims: Dict[int, int],
                          open_labels: Iterable[int] = ()) -> str:
    """Digest of what a tree depends on: the leaves' label tuples, the
    label sizes and the open labels (not the tensor entries)."""
    import hashlib
    import json
    doc = {"labels": [[int(x) for x in ls] for ls in leaf_labels],
           "dims": sorted([int(k), int(v)] for k, v in dims.items()),
           "open": [int(x) for x in open_labels]}
    return hashlib.sha256(json.dumps(doc, separators=(",", ":")).encode()).hexdigest()


def save_tree(path: str, leaf_labels: Sequence[Sequence[int]], dims: Dict[int, int],
              open_labels: Iterable[int], pairs: Sequence[Tuple[int, int]],
              sliced: Sequence[int] = ()) -> None:
    """Write a tree and its sliced labels as JSON, with the network's
    structure fingerprint and the tree's W_s and C_s (for reading only)."""
    import json
    import os
    opn = list(open_labels)
    validate_tree(len(leaf_labels), pairs)
    info = tree_info(leaf_labels, dims, pairs, opn, sliced)
    doc = {"format": TREE_FORMAT, "n_leaves": len(leaf_labels),
           "fingerprint": structure_fingerprint(leaf_labels, dims, opn),
           "pairs": [[int(a), int(b)] for a, b in pairs], "sliced": [int(x) for x in sliced],
           "W_s": info.W, "C_s": info.C_s, "d_sliced": info.d_sliced}
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(doc, f)
    os.replace(tmp, path)


def load_tree(path: str, leaf_labels: Sequence[Sequence[int]], dims: Dict[int, int],
              open_labels: Iterable[int] = ()) -> Tuple[List[Tuple[int, int]], List[int]]:
    """(pairs, sliced) from a tree file written for a network of this
    structure; a file for another structure, another format or holding an
    invalid tree raises ValueError."""
    import json
    with open(path) as f:
        doc = json.load(f)
    if doc.get("format") != TREE_FORMAT:
        raise ValueError(f"{path}: unknown tree file format {doc.get('format')!r}")
    if doc.get("fingerprint") != structure_fingerprint(leaf_labels, dims, open_labels):
        raise ValueError(f"{path}: the tree was found for a network of another structure")
    pairs = [(int(a), int(b)) for a, b in doc["pairs"]]
    validate_tree(len(leaf_labels), pairs)
    sliced = [int(x) for x in doc["sliced"]]
    summed = set(dims) - set(int(x) for x in open_labels)
    if len(set(sliced)) != len(sliced) or not set(sliced) <= summed:
        raise ValueError(f"{path}: sliced labels must be distinct summed labels")
    return pairs, sliced
