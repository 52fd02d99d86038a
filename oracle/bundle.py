"""Index bundling and the logical dimension heuristic -- oracle side.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

``classify`` follows the definition of Section 4: a label shared by A and C is
in the I bundle, by B and C in J, by A and B in P; every label must occur in
exactly two tensors with one extent.  d_I, d_J, d_P then satisfy
d_P = (d(A)+d(B)-d(C))/2 and its two companions.

``normalize`` applies the five steps of Section 7.3 in the paper's order:
  1. every dimension whose length is 1 is discarded;
  2. within a bundle, two dimensions merge into one when, in both tensors that
     carry the bundle, the second one's stride equals the first one's stride
     times its length;
  3. the I dims and the J dims are ordered by their stride in C, smallest first;
  4. when the first J dim then has unit stride in C, the roles of A and B are
     exchanged, and with them those of I and J;
  5. the P dims are ordered by their stride in A, smallest first.
Readings (the paper does not say): sorting uses |stride| and is stable in the
order the labels appear in C (I, J) or A (P); folding merges a pair (x, y)
whenever s_y(T) == s_x(T) * n_x in both tensors of the bundle, scanning pairs
in label order and repeating until no pair merges.  The steps move no data.
"""
from dataclasses import dataclass, field
from typing import Dict, List, Tuple


class LabelError(ValueError):
    pass


class ExtentError(ValueError):
    pass


@dataclass
class Dim:
    labels: Tuple[str, ...]
    n: int
    s: Dict[str, int]  # tensor name ('A', 'B', 'C') -> stride in elements


@dataclass
class Bundles:
    I: List[Dim] = field(default_factory=list)
    J: List[Dim] = field(default_factory=list)
    P: List[Dim] = field(default_factory=list)
    swapped: bool = False

    @property
    def m(self):
        return _prod(d.n for d in self.I)

    @property
    def n(self):
        return _prod(d.n for d in self.J)

    @property
    def k(self):
        return _prod(d.n for d in self.P)


def _prod(it):
    r = 1
    for v in it:
        r *= v
    return r


def classify(labA: str, labB: str, labC: str):
    """Return the label sets (I, J, P) of Section 4 as strings in the order the
    labels appear in C (I, J) and in A (P).  Raises LabelError when a label is
    in one tensor only, in all three, or twice in one tensor."""
    for lab in (labA, labB, labC):
        if len(set(lab)) != len(lab):
            raise LabelError(f"label repeated within {lab!r}")
    sa, sb, sc = set(labA), set(labB), set(labC)
    for x in sa | sb | sc:
        if (x in sa) + (x in sb) + (x in sc) != 2:
            raise LabelError(f"label {x!r} must occur in exactly two tensors")
    I = "".join(x for x in labC if x in sa)
    J = "".join(x for x in labC if x in sb)
    P = "".join(x for x in labA if x in sb)
    return I, J, P


def _dims(A, B, C):
    """A, B, C: (labels, lens, strides).  Build the Dim lists per bundle."""
    (la, na, sa), (lb, nb, sb), (lc, nc, sc) = A, B, C
    I, J, P = classify(la, lb, lc)
    ext, st = {}, {"A": {}, "B": {}, "C": {}}
    for name, (lab, ns, ss) in (("A", A), ("B", B), ("C", C)):
        for x, n, s in zip(lab, ns, ss):
            if x in ext and ext[x] != int(n):
                raise ExtentError(f"label {x!r} has extents {ext[x]} and {n}")
            ext[x] = int(n)
            st[name][x] = int(s)
    def mk(labels, names):
        return [Dim((x,), ext[x], {t: st[t][x] for t in names}) for x in labels]
    return mk(I, "AC"), mk(J, "BC"), mk(P, "AB")


def _fold(dims: List[Dim]) -> List[Dim]:
    dims = list(dims)
    merged = True
    while merged:
        merged = False
        for i in range(len(dims)):
            for j in range(len(dims)):
                if i == j:
                    continue
                x, y = dims[i], dims[j]
                if all(y.s[t] == x.s[t] * x.n for t in x.s):
                    dims[i] = Dim(x.labels + y.labels, x.n * y.n, dict(x.s))
                    del dims[j]
                    merged = True
                    break
            if merged:
                break
    return dims


def normalize(A, B, C) -> Bundles:
    """A, B, C are (labels, lens, strides) triples.  Returns the bundles after
    the five steps of Section 7.3 (names 'A' and 'B' in Dim.s refer to the
    tensors *after* any swap)."""
    I, J, P = _dims(A, B, C)
    # 1. discard length-1 dims
    I = [d for d in I if d.n != 1]
    J = [d for d in J if d.n != 1]
    P = [d for d in P if d.n != 1]
    # 2. merge dims that are sequentially contiguous in both tensors
    I, J, P = _fold(I), _fold(J), _fold(P)
    # 3. order I and J by stride in C
    I = sorted(I, key=lambda d: abs(d.s["C"]))
    J = sorted(J, key=lambda d: abs(d.s["C"]))
    # 4. swap A with B and I with J if the first J dimension has unit stride in C
    swapped = False
    if J and J[0].s["C"] == 1:
        swapped = True
        I, J = J, I
        I = [Dim(d.labels, d.n, {"A": d.s["B"], "C": d.s["C"]}) for d in I]
        J = [Dim(d.labels, d.n, {"B": d.s["A"], "C": d.s["C"]}) for d in J]
        P = [Dim(d.labels, d.n, {"A": d.s["B"], "B": d.s["A"]}) for d in P]
    # 5. order P by stride in A
    P = sorted(P, key=lambda d: abs(d.s["A"]))
    return Bundles(I, J, P, swapped)
