"""Structure simplifications of a tensor network before path search
(Sec. 3.7), applied on the host: they change the network the GPU executes,
never its value.

Rules, each applied where it finds something to do, cycled in the order
antidiagonal-gauging, diagonal-reduction, column-reduction,
rank-simplification, split-simplification until none changes the
network:

- column-reduction: a tensor that vanishes unless index i_x takes one value
  c projects that label onto c in every tensor carrying it (the label
  leaves the network);
- diagonal-reduction: a tensor that vanishes unless i_x == i_y keeps only
  its diagonal, and label i_y becomes i_x everywhere (i_x turns into a
  hyperedge; tensors that then carry i_x twice keep their diagonal);
- antidiagonal-gauging: a tensor that vanishes unless i_x == d - 1 - i_y has
  the order of label i_y (or i_x) reversed in every tensor carrying it,
  which makes it diagonal for the rule above; a reversal is taken only if
  it makes more axis pairs diagonal than it makes antidiagonal among the
  label's tensors, so that the rule cannot undo itself;
- rank-simplification: pairs of tensors sharing a label are contracted
  (numpy, FP64 or complex128) when the result's rank is at most the larger
  of their two ranks -- for networks without hyperedges, absorbing every
  rank-1 and rank-2 tensor into a neighbour -- and its size at most the
  larger of their sizes, smallest result first;
- split-simplification: a tensor with an exact low-rank decomposition
  across a bipartition of its labels (SVD, singular values above rtol of
  the largest), whose two factors are both smaller than the tensor, is
  replaced by the factors joined by a new label.

Zero tests are relative: |entry| <= rtol * max |entry| of the tensor.  Open
labels are never projected, merged away or reversed, so the simplified
network has the same output axes.  ``frozen`` names leaves whose entries
may change between calls with the same simplified structure (e.g. the
output states of sampled bitstrings): the sparsity rules do not inspect
them, and rank- and split-simplification leave them alone, so that a tree
found for one bitstring serves all.
"""
from __future__ import annotations

from typing import Dict, Iterable, List, Optional, Sequence, Tuple

import numpy as np

from .inputs import Network


def _zero(t: np.ndarray, mask: np.ndarray, rtol: float) -> bool:
    m = float(np.max(np.abs(t))) if t.size else 0.0
    return bool(np.all(np.abs(t[mask]) <= rtol * m))


class _Net:
    def __init__(self, net: Network, frozen: Iterable[int]):
        self.t: List[Optional[np.ndarray]] = [np.asarray(x) for x in net.tensors]
        self.l: List[List[int]] = [list(x) for x in net.labels]
        self.dims: Dict[int, int] = dict(net.dims)
        self.open = list(net.open)
        self.frozen = set(frozen)

    def live(self) -> List[int]:
        return [v for v, t in enumerate(self.t) if t is not None]

    def carriers(self, label: int) -> List[int]:
        return [v for v in self.live() if label in self.l[v]]

    # --- column-reduction
    def column(self, rtol: float) -> bool:
        for v in self.live():
            if v in self.frozen:
                continue
            t, ls = self.t[v], self.l[v]
            for x, lab in enumerate(ls):
                if lab in self.open or self.dims[lab] == 1:
                    continue
                for c in range(self.dims[lab]):
                    mask = np.ones(t.shape, dtype=bool)
                    idx = [slice(None)] * t.ndim
                    idx[x] = c
                    mask[tuple(idx)] = False
                    if _zero(t, mask, rtol):
                        if any(w in self.frozen for w in self.carriers(lab)):
                            break
                        for w in self.carriers(lab):
                            ax = self.l[w].index(lab)
                            self.t[w] = np.take(self.t[w], c, axis=ax)
                            del self.l[w][ax]
                        del self.dims[lab]
                        return True
        return False

    # --- diagonal-reduction (and the diagonal of tensors that carry a label twice)
    def _dedupe(self, w: int) -> None:
        while True:
            ls = self.l[w]
            dup = next((l for l in ls if ls.count(l) > 1), None)
            if dup is None:
                return
            a = ls.index(dup)
            b = ls.index(dup, a + 1)
            self.t[w] = np.diagonal(self.t[w], axis1=a, axis2=b)  # diagonal axis goes last
            self.l[w] = [l for i, l in enumerate(ls) if i not in (a, b)] + [dup]

    def diagonal(self, rtol: float) -> bool:
        for v in self.live():
            if v in self.frozen:
                continue
            t, ls = self.t[v], self.l[v]
            for x in range(len(ls)):
                for y in range(x + 1, len(ls)):
                    lx, ly = ls[x], ls[y]
                    if self.dims[lx] != self.dims[ly] or self.dims[lx] == 1 or ly in self.open:
                        continue
                    ix = np.arange(self.dims[lx])
                    shape = [1] * t.ndim
                    shape[x] = shape[y] = self.dims[lx]
                    off = (ix[:, None] != ix[None, :])
                    mask = np.broadcast_to(off.reshape([self.dims[lx] if i in (x, y) else 1
                                                        for i in range(t.ndim)]), t.shape)
                    if not _zero(t, mask, rtol):
                        continue
                    if any(w in self.frozen for w in self.carriers(ly)):
                        continue
                    for w in self.carriers(ly):
                        self.l[w] = [lx if l == ly else l for l in self.l[w]]
                        self._dedupe(w)
                    del self.dims[ly]
                    return True
        return False

    # --- antidiagonal-gauging
    def _pair_kind(self, t: np.ndarray, x: int, y: int, rtol: float) -> Tuple[bool, bool]:
        """(diagonal, antidiagonal): whether t vanishes off the diagonal,
        and off the antidiagonal, of its axes x and y (equal sizes)."""
        d = t.shape[x]
        ix = np.arange(d)
        shape = [d if i in (x, y) else 1 for i in range(t.ndim)]
        res = []
        for keep in (ix[:, None] == ix[None, :], ix[:, None] == d - 1 - ix[None, :]):
            off = ~keep if x < y else ~keep.T
            res.append(_zero(t, np.broadcast_to(off.reshape(shape), t.shape), rtol))
        return res[0], res[1]

    def _flip_gain(self, label: int, rtol: float) -> int:
        """Reversing ``label`` everywhere turns every antidiagonal axis pair
        containing it diagonal and every diagonal one antidiagonal: the net
        number of antidiagonal-only pairs it removes."""
        gain = 0
        for w in self.carriers(label):
            t, ls = self.t[w], self.l[w]
            a = ls.index(label)
            for b, other in enumerate(ls):
                if b == a or self.dims[other] != self.dims[label]:
                    continue
                diag, anti = self._pair_kind(t, a, b, rtol)
                gain += int(anti and not diag) - int(diag and not anti)
        return gain

    def antidiagonal(self, rtol: float) -> bool:
        """Reverse one label that makes an antidiagonal axis pair diagonal.
        A reversal is taken only if it removes more antidiagonal pairs than
        it creates over all tensors carrying the label, so the number of
        antidiagonal pairs falls with every step and the rule terminates
        (a label shared by two tensors, antidiagonal in one and diagonal in
        the other, is left alone rather than flipped back and forth)."""
        for v in self.live():
            if v in self.frozen:
                continue
            t, ls = self.t[v], self.l[v]
            for x in range(len(ls)):
                for y in range(x + 1, len(ls)):
                    lx, ly = ls[x], ls[y]
                    d = self.dims[lx]
                    if d != self.dims[ly] or d == 1:
                        continue
                    diag, anti = self._pair_kind(t, x, y, rtol)
                    if not anti or diag:
                        continue  # not antidiagonal, or already diagonal (d = 1 or a zero tensor)
                    for flip in (ly, lx):
                        if flip in self.open or any(w in self.frozen for w in self.carriers(flip)):
                            continue
                        if self._flip_gain(flip, rtol) <= 0:
                            continue
                        for w in self.carriers(flip):
                            ax = self.l[w].index(flip)
                            self.t[w] = np.flip(self.t[w], axis=ax).copy()
                        return True
        return False

    # --- rank-simplification
    def rank(self) -> bool:
        best = None
        live = [v for v in self.live() if v not in self.frozen]
        count: Dict[int, int] = {}
        for v in self.live():
            for l in self.l[v]:
                count[l] = count.get(l, 0) + 1
        for i, a in enumerate(live):
            for b in live[i + 1:]:
                shared = set(self.l[a]) & set(self.l[b])
                if not shared:
                    continue
                out = [l for l in self.l[a] + [l for l in self.l[b] if l not in self.l[a]]
                       if l in self.open or count[l] > (l in self.l[a]) + (l in self.l[b])]
                if len(out) > max(len(self.l[a]), len(self.l[b])):
                    continue
                size = int(np.prod([self.dims[l] for l in out])) if out else 1
                # never larger than the larger input: this also keeps the
                # factors of a split from being merged back
                if size > max(self.t[a].size, self.t[b].size):
                    continue
                key = (size, len(out), a, b)
                if best is None or key < best[0]:
                    best = (key, a, b, out)
        if best is None:
            return False
        _, a, b, out = best
        sym = {}
        for l in set(self.l[a]) | set(self.l[b]) | set(out):
            sym[l] = len(sym)
        letters = "abcdefghijklmnopqrstuvwxyzABCDEFGHIJKLMNOPQRSTUVWXYZ"
        if len(sym) > len(letters):
            return False
        spec = ("".join(letters[sym[l]] for l in self.l[a]) + "," +
                "".join(letters[sym[l]] for l in self.l[b]) + "->" +
                "".join(letters[sym[l]] for l in out))
        self.t[a] = np.einsum(spec, self.t[a], self.t[b])
        self.l[a] = out
        self.t[b] = None
        for l in list(self.dims):
            if not any(l in self.l[v] for v in self.live()) and l not in self.open:
                del self.dims[l]
        return True

    # --- split-simplification
    def split(self, rtol: float) -> bool:
        """A tensor with an exact low-rank decomposition across a bipartition
        of its labels, t = l r with max(size(l), size(r)) < size(t), is
        replaced by l and r joined by a new label (SVD; singular values
        above rtol times the largest are kept)."""
        for v in self.live():
            if v in self.frozen:
                continue
            t, ls = self.t[v], self.l[v]
            k = len(ls)
            if k < 3 or k > 12:
                continue
            size = t.size
            for mask in range(1, 1 << (k - 1)):  # bipartitions (label 0 on the left... or not)
                left = [i for i in range(k) if (mask >> i) & 1]
                right = [i for i in range(k) if not (mask >> i) & 1]
                if not left or not right:
                    continue
                dl = int(np.prod([t.shape[i] for i in left]))
                dr = int(np.prod([t.shape[i] for i in right]))
                if min(dl, dr) < 2:
                    continue
                mat = np.transpose(t, left + right).reshape(dl, dr)
                u, s, vh = np.linalg.svd(mat, full_matrices=False)
                if s.size == 0 or not s[0] > 0:
                    continue
                r = int(np.sum(s > rtol * s[0]))
                if max(dl * r, dr * r) >= size:
                    continue
                new = max(self.dims) + 1 if self.dims else 0
                lt = (u[:, :r] * s[:r]).reshape([t.shape[i] for i in left] + [r])
                rt = vh[:r, :].reshape([r] + [t.shape[i] for i in right])
                self.t[v] = lt
                self.l[v] = [ls[i] for i in left] + [new]
                self.t.append(rt)
                self.l.append([new] + [ls[i] for i in right])
                self.dims[new] = r
                return True
        return False

    def result(self, meta: dict) -> Network:
        live = self.live()
        tensors = [self.t[v] for v in live]
        labels = [self.l[v] for v in live]
        if not tensors:
            tensors, labels = [np.array(1.0)], [[]]
        used = {l for ls in labels for l in ls} | set(self.open)
        dims = {l: d for l, d in self.dims.items() if l in used}
        return Network(tensors, labels, dims, list(self.open), meta=meta)


def simplify(net: Network, frozen: Sequence[int] = (), rtol: float = 1e-12,
             max_rounds: int = 10000, split: bool = True) -> Tuple[Network, Dict[str, int]]:
    """The simplified network (same value, same open labels) and counts of
    the operations applied.  ``frozen``: leaf indices left out (see module
    docstring); in the result they come first, in their original order, so
    that callers can keep addressing them."""
    w = _Net(net, frozen)
    done = {"antidiagonal": 0, "diagonal": 0, "column": 0, "rank": 0, "split": 0}
    for _ in range(max_rounds):
        changed = False
        for name in ("antidiagonal", "diagonal", "column", "rank") + (("split",) if split else ()):
            fn = getattr(w, name)
            while (fn(rtol) if name != "rank" else fn()):
                done[name] += 1
                changed = True
        if not changed:
            break
    order = [v for v in sorted(w.frozen) if w.t[v] is not None] + \
        [v for v in w.live() if v not in w.frozen]
    w.t = [w.t[v] for v in order]
    w.l = [w.l[v] for v in order]
    meta = dict(net.meta)
    meta["simplified"] = dict(done, leaves_before=net.n_tensors)
    return w.result(meta), done
