"""The seeded workload generators (no GPU): Section 9's contractions shaped
like a given matrix multiplication, and the effective lengths the paper
reports them at."""
import numpy as np
import pytest

from paper_1607_00291_gb300 import workloads as W


def bundles(p):
    I = [x for x in p.labC if x in p.labA]
    J = [x for x in p.labC if x in p.labB]
    P = [x for x in p.labA if x in p.labB]
    return I, J, P


def size(p, xs):
    return int(np.prod([p.ext[x] for x in xs])) if xs else 1


@pytest.mark.parametrize("mnk", [(4096, 4096, 4096), (16000, 16000, 256), (300, 200, 20)])
def test_shaped_problems_follow_the_recipe(mnk):
    rng = np.random.default_rng(5)
    m, n, k = mnk
    for _ in range(50):
        p = W.shaped_problem(rng, m, n, k)
        I, J, P = bundles(p)
        # every label in exactly two tensors; one to three dims per bundle
        for x in p.ext:
            assert (x in p.labA) + (x in p.labB) + (x in p.labC) == 2
        assert all(1 <= len(b) <= 3 for b in (I, J, P))
        assert sorted(p.labA) == sorted(I + P) and sorted(p.labB) == sorted(P + J)
        # storage orders are permutations of each tensor's labels
        for lab, order in ((p.labA, p.orderA), (p.labB, p.orderB), (p.labC, p.orderC)):
            assert sorted(lab) == sorted(order)
        # bundle products close to the matrix lengths
        for b, target in ((I, m), (J, n), (P, k)):
            assert abs(size(p, b) / target - 1) < 0.3, (b, size(p, b), target)
        assert p.flops() == 2.0 * size(p, I) * size(p, J) * size(p, P)


def test_effective_lengths():
    assert W.effective_square(2.0 * 4096 ** 3) == pytest.approx(4096)
    assert W.effective_rank_k(2.0 * 16000 * 16000 * 256, 16000, 16000) == pytest.approx(256)


def test_paper_problem_sets_are_seeded():
    for name in W.PAPER_SHAPES:
        a, b = W.paper_problems(name), W.paper_problems(name)
        assert [(p.labA, p.labB, p.labC, p.ext) for p in a] == [(p.labA, p.labB, p.labC, p.ext) for p in b]
        assert len(a) == W.PAPER_SHAPES[name]["count"]


def test_benchmark_strings_parse_and_follow_the_extent_rule():
    import oracle.bundle as ob
    assert len(W.TCCG_STRINGS) == 24
    for s in W.TCCG_STRINGS:
        p = W.tccg_problem(s)
        labC, labA, labB = s.split("-")
        assert (p.labA, p.labB, p.labC) == (labA, labB, labC)
        I, J, P = ob.classify(labA, labB, labC)  # each label in exactly two tensors
        assert I and J and P
        L = len(set(labA + labB + labC))
        e = p.ext[labC[0]]
        assert set(p.ext.values()) == {e}
        # the integer extent nearest to (2^33)^(1/L): about 2^34 flops
        assert abs(e - 2 ** (33 / L)) <= 0.5
        assert 0.5 * 2 ** 34 < p.flops() < 2 * 2 ** 34
    # the small form of the same rule
    assert all(W.tccg_problem(s, 2.0 ** 16).flops() < 2 ** 18 for s in W.TCCG_STRINGS)
