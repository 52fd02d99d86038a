"""Seeded synthetic workloads (shapes, layouts, value distributions).

This module holds no arithmetic of the method: it only defines the contraction
shapes the benchmarks and tests use and draws their inputs from seeded
generators, in FP64 on the host.  The same host arrays feed both the CUDA path
and the CPU oracle.

Layout convention: "column-major" means general column-major order (Section 5):
the first index has stride 1 and each further stride is the product of the
lengths before it.
"""
from dataclasses import dataclass, field
from typing import Dict, List, Optional, Tuple

import numpy as np
import torch


@dataclass
class Spec:
    name: str
    labA: str
    labB: str
    labC: str
    ext: Dict[str, int]
    dtype: torch.dtype
    alpha: float
    beta: float
    dist: str = "uniform"          # uniform[-1,1] | normal | uniform_spiky
    c_init: str = "zeros"          # zeros | uniform | nan
    mode: str = "f64"

    def shape(self, lab: str) -> Tuple[int, ...]:
        return tuple(self.ext[x] for x in lab)

    def flops(self) -> float:
        return 2.0 * float(np.prod([self.ext[x] for x in set(self.labA + self.labB + self.labC)]))


# The five workload shapes measured by bench.py and the tests.
SPECS = {
    # FP64, abcd <- aebf . dfce, every extent 16 (256^3 as a matrix product)
    "small_f64": Spec("small_f64", "aebf", "dfce", "abcd", dict.fromkeys("abcdef", 16),
                      torch.float64, 1.0, 0.0),
    # FP64 coupled-cluster-style abij <- cadb . icjd, a..d = 96, i, j = 24
    "cc4x4_f64": Spec("cc4x4_f64", "cadb", "icjd", "abij",
                      dict(a=96, b=96, c=96, d=96, i=24, j=24), torch.float64, 0.5, 1.0,
                      c_init="uniform"),
    # FP32 abcd <- eafb . cfde, all 64, 1% of entries scaled by 1e3, BF16x3 mode
    "spiky_f32": Spec("spiky_f32", "eafb", "cfde", "abcd", dict.fromkeys("abcdef", 64),
                      torch.float32, 1.0, 0.0, dist="uniform_spiky", mode="bf16x3"),
    # FP32 ijk <- ilmj . mkl, i, j, k = 128, l, m = 64, normal inputs, forward + backward
    "grad_f32": Spec("grad_f32", "ilmj", "mkl", "ijk", dict(i=128, j=128, k=128, l=64, m=64),
                     torch.float32, 1.0, 0.0, dist="normal", mode="bf16x3"),
}


def colmajor(flat: torch.Tensor, shape) -> torch.Tensor:
    """View a flat tensor as `shape` in general column-major order."""
    r = len(shape)
    if r == 0:
        return flat.reshape(())
    return flat.reshape(tuple(reversed(shape))).permute(*reversed(range(r)))


def _draw(g: torch.Generator, n: int, dist: str) -> torch.Tensor:
    if dist == "uniform":
        return torch.rand(n, generator=g, dtype=torch.float64) * 2 - 1
    if dist == "normal":
        return torch.randn(n, generator=g, dtype=torch.float64)
    if dist == "uniform_spiky":
        x = torch.rand(n, generator=g, dtype=torch.float64) * 2 - 1
        mask = torch.rand(n, generator=g, dtype=torch.float64) < 0.01
        return torch.where(mask, x * 1e3, x)
    if dist == "int":
        return torch.randint(-8, 9, (n,), generator=g).to(torch.float64)
    raise ValueError(dist)


def make_inputs(spec: Spec, seed: int, dist: Optional[str] = None):
    """Host FP64 arrays (column-major) for A, B and the initial C, already
    rounded to spec.dtype (so the oracle sees exactly the device values)."""
    g = torch.Generator().manual_seed(seed)
    dist = dist or spec.dist
    out = {}
    for name, lab in (("A", spec.labA), ("B", spec.labB)):
        shape = spec.shape(lab)
        n = int(np.prod(shape)) if shape else 1
        out[name] = colmajor(_draw(g, n, dist).to(spec.dtype).to(torch.float64), shape)
    shape = spec.shape(spec.labC)
    n = int(np.prod(shape)) if shape else 1
    if spec.c_init == "zeros":
        c = torch.zeros(n, dtype=torch.float64)
    elif spec.c_init == "nan":
        c = torch.full((n,), float("nan"), dtype=torch.float64)
    else:
        c = _draw(g, n, "uniform" if dist != "int" else "int")
    out["C"] = colmajor(c.to(spec.dtype).to(torch.float64), shape)
    return out


# ---- random contractions (batch workloads, parity sweeps) ---------------------------

LETTERS = "abcdefghijklmnopqrstuvwxyzABCDEFGHIJKLMNOPQRSTUVWXYZ"


@dataclass
class RandomProblem:
    labA: str
    labB: str
    labC: str
    ext: Dict[str, int]
    # per-tensor dimension order of the storage (a permutation of the labels),
    # giving a dense layout with randomly permuted strides
    orderA: str = ""
    orderB: str = ""
    orderC: str = ""
    alpha: float = 1.0
    beta: float = 0.0

    def flops(self):
        return 2.0 * float(np.prod([self.ext[x] for x in set(self.labA + self.labB + self.labC)]))


def random_problem(rng: np.random.Generator, dI=(1, 3), dJ=(1, 3), dP=(1, 3), ext=(8, 64),
                   max_rank: int = 6, max_elems: int = 1 << 22, max_flops: float = 2.0 ** 34,
                   allow_zero_bundles: bool = False) -> RandomProblem:
    """Draw a contraction with d_I, d_J, d_P dims, extents uniform in `ext`,
    random label orders in A, B, C and randomly permuted dense strides.
    Redraws until every operand has at most `max_elems` elements and the flop
    count is at most `max_flops`."""
    lo = 0 if allow_zero_bundles else 1
    while True:
        nP = int(rng.integers(dP[0], dP[1] + 1))
        nI = int(rng.integers(max(lo, dI[0]), dI[1] + 1))
        nJ = int(rng.integers(max(lo, dJ[0]), dJ[1] + 1))
        if nI + nP > max_rank or nJ + nP > max_rank or nI + nJ > max_rank:
            continue
        labs = list(rng.permutation(list(LETTERS[:nI + nJ + nP])))
        I, J, P = labs[:nI], labs[nI:nI + nJ], labs[nI + nJ:]
        e = {x: int(rng.integers(ext[0], ext[1] + 1)) for x in labs}
        A = "".join(rng.permutation(I + P)) if I + P else ""
        B = "".join(rng.permutation(P + J)) if P + J else ""
        C = "".join(rng.permutation(I + J)) if I + J else ""
        size = lambda s: int(np.prod([e[x] for x in s])) if s else 1
        if max(size(A), size(B), size(C)) > max_elems:
            continue
        fl = 2.0 * size(I) * size(J) * size(P)
        if fl > max_flops:
            continue
        oA = "".join(rng.permutation(list(A))) if A else ""
        oB = "".join(rng.permutation(list(B))) if B else ""
        oC = "".join(rng.permutation(list(C))) if C else ""
        return RandomProblem(A, B, C, e, oA, oB, oC)


def dense_permuted(flat: torch.Tensor, labels: str, order: str, ext: Dict[str, int]) -> torch.Tensor:
    """View `flat` as a tensor indexed by `labels` whose storage is column-major
    in the label order `order`."""
    if not labels:
        return flat.reshape(())
    base = colmajor(flat, tuple(ext[x] for x in order))
    perm = [order.index(x) for x in labels]
    return base.permute(*perm)


def make_random_inputs_on(p: RandomProblem, seed: int, dtype, device):
    """As make_random_inputs with uniform[-1, 1] values, drawn on `device`
    from its own seeded generator (large workloads: no host round trip).
    Returns tensors of `dtype` on the device."""
    g = torch.Generator(device=device).manual_seed(seed)
    out = {}
    for name, lab, order in (("A", p.labA, p.orderA), ("B", p.labB, p.orderB), ("C", p.labC, p.orderC)):
        n = int(np.prod([p.ext[x] for x in lab])) if lab else 1
        flat = (torch.rand(n, generator=g, dtype=torch.float64, device=device) * 2 - 1).to(dtype)
        out[name] = dense_permuted(flat, lab, order or lab, p.ext)
    return out


def make_random_inputs(p: RandomProblem, seed: int, dtype=torch.float64, dist: str = "uniform"):
    g = torch.Generator().manual_seed(seed)
    out = {}
    for name, lab, order in (("A", p.labA, p.orderA), ("B", p.labB, p.orderB), ("C", p.labC, p.orderC)):
        n = int(np.prod([p.ext[x] for x in lab])) if lab else 1
        flat = _draw(g, n, dist).to(dtype).to(torch.float64)
        out[name] = dense_permuted(flat, lab, order or lab, p.ext)
    return out


# ---- the batch workload: 512 independent contractions ---------------------------------

def batch_problems(seed: int = 1004, count: int = 512):
    """Random contractions of the paper's random-contraction generator shape:
    1-3 contracted indices, ranks 2-6 per operand (d_I + d_P <= 6,
    d_P + d_J <= 6, d_I, d_J >= 1), extents uniform in 8..64, random label
    orders and randomly permuted dense layouts; a draw whose operand exceeds
    2^22 elements or whose flop count exceeds 2^34 is redrawn."""
    rng = np.random.default_rng(seed)
    return [random_problem(rng, dI=(1, 5), dJ=(1, 5), dP=(1, 3), ext=(8, 64), max_rank=6,
                           max_elems=1 << 22, max_flops=2.0 ** 34) for _ in range(count)]


# ---- contractions shaped like a given matrix multiplication ---------------------------
# Section 9's randomly generated contractions: for a matrix shape (m, n, k),
# each of the bundles I, J, P gets one to three tensor dims whose extents
# multiply to about m, n and k; the label order inside each tensor and each
# tensor's storage order are random permutations.  Results are reported
# against "effective" matrix lengths derived from the flops f actually
# performed: m = n = k = (f / 2)^(1/3) for square shapes, k = f / (2 m n)
# for rank-k updates with the prescribed m and n.

def split_extent(rng: np.random.Generator, target: int, nd: int, min_ext: int = 2) -> List[int]:
    """`nd` extents (each >= min_ext) whose product is close to `target`: the
    first nd - 1 drawn within +-25 % of target^(1/nd), the last making up the
    rest."""
    if nd == 1:
        return [max(min_ext, int(target))]
    base = float(target) ** (1.0 / nd)
    ext = [max(min_ext, int(round(base * rng.uniform(0.75, 1.25)))) for _ in range(nd - 1)]
    ext.append(max(min_ext, int(round(target / float(np.prod(ext))))))
    return ext


def shaped_problem(rng: np.random.Generator, m: int, n: int, k: int,
                   dims=(1, 3)) -> RandomProblem:
    """One random contraction shaped like an m x n x k matrix multiplication."""
    nd = [int(rng.integers(dims[0], dims[1] + 1)) for _ in range(3)]
    labs = [str(x) for x in rng.permutation(list(LETTERS[:sum(nd)]))]
    I, J, P = labs[:nd[0]], labs[nd[0]:nd[0] + nd[1]], labs[nd[0] + nd[1]:]
    e = {}
    for bundle, target in ((I, m), (J, n), (P, k)):
        for x, v in zip(bundle, split_extent(rng, target, len(bundle))):
            e[x] = v
    perm = lambda xs: "".join(str(x) for x in rng.permutation(list(xs)))  # noqa: E731
    A, B, C = perm(I + P), perm(P + J), perm(I + J)
    return RandomProblem(A, B, C, e, perm(A), perm(B), perm(C))


def effective_square(flops: float) -> float:
    """Effective m = n = k of a square-shaped contraction: (f / 2)^(1/3)."""
    return (flops / 2.0) ** (1.0 / 3.0)


def effective_rank_k(flops: float, m: int, n: int) -> float:
    """Effective k of a rank-k-shaped contraction with prescribed m and n: f / (2 m n)."""
    return flops / (2.0 * m * n)


# The two shape families of the paper's random-contraction experiments at
# GB300-sized lengths: three contractions per shape (seeded).
PAPER_SHAPES = {
    "paper_square_f64": dict(m=4096, n=4096, k=4096, seed=1101, count=3),
    "paper_rankk_f64": dict(m=16000, n=16000, k=256, seed=1102, count=3),
}


def paper_problems(name: str) -> List[RandomProblem]:
    s = PAPER_SHAPES[name]
    rng = np.random.default_rng(s["seed"])
    return [shaped_problem(rng, s["m"], s["n"], s["k"]) for _ in range(s["count"])]


# ---- the Tensor Contraction Benchmark's contraction strings (Section 9.3) ------------
# The 24 contractions the paper runs from the Tensor Contraction Benchmark, as
# printed on its benchmark figure: index strings C-A-B ("abc-adec-ebd" is
# C_abc := A_adec B_ebd), from the communication-bound to the compute-bound
# end.  The paper gives no extents and no data.  Synthetic stand-ins: every
# index of a contraction gets the same extent e, the integer nearest to
# (F / 2)^(1 / L) for L distinct indices, so that each contraction performs
# about F flops (2 e^L); the label structure alone then decides the matrix
# shape (a lone contracted index makes a rank-k-like update, two indices per
# bundle a square-like product).  Every tensor is column-major in its own
# label order (the first index has stride 1); values uniform[-1, 1].
TCCG_STRINGS = [
    "abcde-efbad-cf", "abcde-efcad-bf", "abcd-dbea-ec", "abcde-ecbfa-fd", "abcd-deca-be",
    "abc-bda-dc", "abcd-ebad-ce", "abcdef-dega-gfbc", "abcdef-dfgb-geac", "abcdef-degb-gfac",
    "abcdef-degc-gfab", "abc-dca-bd", "abcd-ea-ebcd", "abcd-eb-aecd", "abcd-ec-abed",
    "abc-adec-ebd", "ab-cad-dcb", "ab-acd-dbc", "abc-acd-db", "abc-adc-bd", "ab-ac-cb",
    "abcd-aebf-fdec", "abcd-eafd-fbec", "abcd-aebf-dfce",
]


def tccg_problem(index_string: str, flops: float = 2.0 ** 34) -> RandomProblem:
    """One contraction of the benchmark's strings with the synthetic extents
    described above (column-major storage in each tensor's label order)."""
    labC, labA, labB = index_string.split("-")
    labels = sorted(set(labA + labB + labC))
    e = max(2, int(round((flops / 2.0) ** (1.0 / len(labels)))))
    return RandomProblem(labA, labB, labC, {x: e for x in labels}, labA, labB, labC)


def tccg_problems(flops: float = 2.0 ** 34) -> List[RandomProblem]:
    return [tccg_problem(s, flops) for s in TCCG_STRINGS]
