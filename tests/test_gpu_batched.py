"""Batched contractions (K6 persistent launch, K7 autotuner, graph replay)
against the CPU oracle, problem by problem, in every mode."""
import os

import numpy as np
import pytest
import torch

import paper_1607_00291_gb300 as tc
from paper_1607_00291_gb300 import workloads as W

from helpers import norm_err, oracle_ref, to_device

pytestmark = pytest.mark.gpu
TOLS = {"f64": 1e-12, "bf16x3": 3 * 2.0 ** -16 + 8 * 2.0 ** -24, "bf16x6": 1e-5}


def make_batch(seed, count, ext=(1, 30), mode="f64"):
    rng = np.random.default_rng(seed)
    dt = torch.float64 if mode == "f64" else torch.float32
    host, dev = [], []
    for i in range(count):
        p = W.random_problem(rng, dI=(1, 3), dJ=(1, 3), dP=(1, 3), ext=ext, max_elems=1 << 16,
                             max_flops=2.0 ** 24)
        h = W.make_random_inputs(p, seed=seed * 1000 + i, dtype=dt)
        alpha = float(rng.uniform(-2, 2))
        beta = float(rng.choice([0.0, 1.0, rng.uniform(-2, 2)]))
        host.append((p, h, alpha, beta))
        dev.append((to_device(h["A"], dt), p.labA, to_device(h["B"], dt), p.labB,
                    to_device(h["C"], dt), p.labC, alpha, beta))
    return host, dev


def check_batch(host, dev, mode):
    worst = 0.0
    for (p, h, alpha, beta), d in zip(host, dev):
        ref, mag = oracle_ref(alpha, h["A"], p.labA, h["B"], p.labB, beta, h["C"], p.labC)
        e = norm_err(d[4].cpu().double().numpy(), ref, mag)
        worst = max(worst, e)
    assert worst <= TOLS[mode], worst
    return worst


@pytest.mark.parametrize("mode", ["f64", "bf16x3", "bf16x6"])
def test_batch_matches_oracle(mode):
    host, dev = make_batch(11, 40, mode=mode)
    tc.contract_batched(dev, mode=mode)
    assert tc.device_error() == 0
    check_batch(host, dev, mode)


@pytest.mark.parametrize("mode", ["f64", "bf16x3"])
def test_plan_graph_capture_and_replay(mode):
    host, dev = make_batch(12, 24, mode=mode)
    C0 = [d[4].clone() for d in dev]
    plan = tc.Plan(dev, mode=mode)
    plan.execute()  # first run outside capture (one-time per-device set-up)
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        plan.execute()
    # capture does not run the kernels; each replay performs the batch once
    for d, c0 in zip(dev, C0):
        d[4].copy_(c0)
    torch.cuda.synchronize()
    g.replay()
    torch.cuda.synchronize()
    assert tc.device_error() == 0
    check_batch(host, dev, mode)
    for d, c0 in zip(dev, C0):
        d[4].copy_(c0)
    g.replay()
    torch.cuda.synchronize()
    check_batch(host, dev, mode)
    plan.close()


@pytest.mark.parametrize("mode", ["f64", "bf16x6"])
def test_batch_degenerate_members(mode):
    dt = torch.float64 if mode == "f64" else torch.float32
    g = torch.Generator().manual_seed(13)
    r = lambda *s: (torch.rand(*s, generator=g, dtype=torch.float64) * 2 - 1).to(dt).double()
    cases = [
        (0.0, torch.full((9, 7), float("nan"), dtype=torch.float64), "ip", r(7, 5), "pj", 2.0, r(9, 5), "ij"),
        (1.0, torch.zeros(9, 0, dtype=torch.float64), "ip", torch.zeros(0, 5, dtype=torch.float64), "pj", 0.5, r(9, 5), "ij"),
        (1.0, r(0, 4), "ip", r(4, 5), "pj", 1.0, torch.zeros(0, 5, dtype=torch.float64), "ij"),
        (1.0, r(33), "p", r(33, 70), "pj", 0.0, torch.full((70,), float("nan"), dtype=torch.float64), "j"),
        (1.0, r(130), "i", r(70), "j", 0.0, torch.zeros(70, 130, dtype=torch.float64), "ji"),
        (1.5, r(7, 9), "ab", r(9, 7), "ba", -1.0, r(()), ""),
    ]
    dev = [(to_device(A, dt), la, to_device(B, dt), lb, to_device(C, dt), lc, al, be)
           for (al, A, la, B, lb, be, C, lc) in cases]
    tc.contract_batched(dev, mode=mode)
    assert tc.device_error() == 0
    for (al, A, la, B, lb, be, C, lc), d in zip(cases, dev):
        got = d[4].cpu().double().numpy()
        if al == 0.0:
            assert np.array_equal(got, (be * C).to(dt).double().numpy())
            continue
        ref, mag = oracle_ref(al, A, la, B, lb, be, C, lc)
        assert norm_err(got, ref, mag) <= TOLS[mode]


def test_autotuned_batch(monkeypatch, tmp_path):
    cache = tmp_path / "tune.txt"
    monkeypatch.setenv("TC_AUTOTUNE", "1")
    monkeypatch.setenv("TC_AUTOTUNE_CACHE", str(cache))
    host, dev = make_batch(14, 12, ext=(8, 40), mode="bf16x3")
    tc.contract_batched(dev, mode="bf16x3")
    assert tc.device_error() == 0
    check_batch(host, dev, "bf16x3")
    lines = cache.read_text().strip().splitlines()
    assert lines and all(l.split()[0] in ("tile", "balance") for l in lines)
    assert any(l.startswith("balance ") for l in lines)


def _cm_strides(shape):
    st, acc = [], 1
    for n in shape:
        st.append(acc)
        acc *= n
    return tuple(st)


def _tile_key(mode_code, pl):
    lg = lambda x: 0 if x <= 1 else int(round(np.log2(x)))  # noqa: E731
    return (f"{mode_code} {lg(pl['m'])} {lg(pl['n'])} {lg(pl['k'])} "
            f"{int(pl['a_k_contig'])} {int(pl['b_k_contig'])}")


@pytest.mark.parametrize("mode", ["f64", "bf16x3"])
def test_cached_tile_record_changes_the_choice(monkeypatch, tmp_path, mode):
    # three problems of one shape class (200 x 100 x 96 as given; the planner
    # swaps A and B for the row-major C): the estimate takes the
    # least-padding FP64 tile or the tensor-core tile covering n; a cached
    # record of the class overrides it, and the results still match the oracle
    dt = torch.float64 if mode == "f64" else torch.float32
    g = torch.Generator().manual_seed(5)
    r = lambda *s: (torch.rand(*s, generator=g, dtype=torch.float64) * 2 - 1).to(dt).double()  # noqa: E731
    cases = [(r(200, 96), r(96, 100), r(200, 100)) for _ in range(3)]
    dev = [(to_device(A, dt), "ip", to_device(B, dt), "pj", to_device(C, dt), "ij", 1.0, 0.5)
           for A, B, C in cases]
    monkeypatch.delenv("TC_AUTOTUNE", raising=False)
    monkeypatch.delenv("TC_AUTOTUNE_CACHE", raising=False)
    est = tc.Plan(dev, mode=mode)
    pl = tc.plan_describe(dev[0][0], "ip", dev[0][2], "pj", dev[0][4], "ij")
    mcode = {"f64": 0, "bf16x3": 1}[mode]
    m, n = pl["m"], pl["n"]  # the matrix view (C row-major: A and B trade roles)
    if mode == "f64":
        tiles = {0: (64, 64), 1: (32, 64), 2: (64, 32)}  # the FP64 tile classes
        pad = lambda t: -(-m // t[0]) * t[0] * (-(-n // t[1]) * t[1])  # noqa: E731
        got = (est.config(0)["bm"], est.config(0)["bn"])
        assert got == min(tiles.values(), key=pad)  # the least-padding estimate
        forced = next(c for c, t in tiles.items() if t != got)
        want = tiles[forced]
    else:
        assert est.config(0)["bn"] == min(128, -(-n // 16) * 16)  # the tile covering n
        forced, want = 64, (128, 64)
    est.close()
    cache = tmp_path / "tune.txt"
    cache.write_text(f"tile {_tile_key(mcode, pl)} {forced}\n")
    monkeypatch.setenv("TC_AUTOTUNE_CACHE", str(cache))
    plan = tc.Plan(dev, mode=mode)
    for i in range(3):
        c = plan.config(i)
        assert (c["bm"], c["bn"]) == want
    plan.execute()
    torch.cuda.synchronize()
    assert tc.device_error() == 0
    for (A, B, C0), d in zip(cases, dev):
        ref, mag = oracle_ref(1.0, A, "ip", B, "pj", 0.5, C0, "ij")
        assert norm_err(d[4].cpu().double().numpy(), ref, mag) <= TOLS[mode]
    plan.close()


@pytest.mark.parametrize("mode", ["f64", "bf16x3"])
def test_balance_divisor_is_tuned_and_cached(monkeypatch, tmp_path, mode):
    # forty problems and two with a long contracted range: the tuner
    # times the batch with D = 2, 4, 8, 16 and records its choice; a cached
    # D then decides how finely the long problems are split
    dt = torch.float64 if mode == "f64" else torch.float32
    g = torch.Generator().manual_seed(6)
    r = lambda *s: (torch.rand(*s, generator=g, dtype=torch.float64) * 2 - 1).to(dt).double()  # noqa: E731
    cases = [(r(128, 2048), r(2048, 256), torch.zeros(128, 256, dtype=torch.float64)) for _ in range(40)]
    cases += [(r(96, 20000), r(20000, 80), torch.zeros(96, 80, dtype=torch.float64)) for _ in range(2)]
    dev = [(to_device(A, dt), "ip", to_device(B, dt), "pj", to_device(C, dt), "ij", 1.0, 0.0)
           for A, B, C in cases]
    cache = tmp_path / "tune.txt"
    monkeypatch.setenv("TC_AUTOTUNE_CACHE", str(cache))
    tuned = tc.Plan(dev, mode=mode)
    bal = [l for l in cache.read_text().splitlines() if l.startswith("balance ")]
    assert len(bal) == 1
    sig, d = bal[0].split()[1:]
    assert int(d) in (2, 4, 8, 16) and tuned.config(0)["balance"] == int(d)
    tuned.close()
    splits = {}
    for D in (2, 16):
        f = tmp_path / f"tune{D}.txt"
        f.write_text(f"balance {sig} {D}\n")
        monkeypatch.setenv("TC_AUTOTUNE_CACHE", str(f))
        plan = tc.Plan(dev, mode=mode)
        c = plan.config(len(cases) - 1)
        assert c["balance"] == D
        splits[D] = c["splits"]
        for d_ in dev:
            d_[4].zero_()
        plan.execute()
        torch.cuda.synchronize()
        assert tc.device_error() == 0
        for (A, B, C0), d_ in zip(cases, dev):
            ref, mag = oracle_ref(1.0, A, "ip", B, "pj", 0.0, C0, "ij")
            assert norm_err(d_[4].cpu().double().numpy(), ref, mag) <= TOLS[mode]
        plan.close()
    assert splits[16] > splits[2] >= 1


@pytest.mark.parametrize("mode", ["f64", "bf16x3"])
def test_batch512_workload_every_element(mode):
    # the 512-problem workload at full size, every output element of every
    # problem against the oracle (every tile class, every k-split)
    import oracle
    dt = torch.float64 if mode == "f64" else torch.float32
    probs = W.batch_problems(seed=1004)
    host, dev = [], []
    for i, p in enumerate(probs):
        h = W.make_random_inputs(p, seed=5000 + i, dtype=dt)
        host.append((p, h))
        dev.append((to_device(h["A"], dt), p.labA, to_device(h["B"], dt), p.labB,
                    to_device(h["C"], dt), p.labC, 1.0, 0.0))
    tc.contract_batched(dev, mode=mode)
    assert tc.device_error() == 0
    worst = 0.0
    for (p, h), d in zip(host, dev):
        got = d[4].cpu().double().numpy()
        c = np.array(h["C"].numpy(), copy=True)
        mag = oracle.contract_(1.0, h["A"].numpy(), p.labA, h["B"].numpy(), p.labB, 0.0, c, p.labC)
        worst = max(worst, norm_err(got, c, mag))
    assert worst <= TOLS[mode], worst


@pytest.mark.parametrize("mode", ["f64", "bf16x3"])
def test_dynamic_items_many_small_and_empty(mode):
    # 300 problems, every third with an empty contracted range (C = beta * C
    # alone): many more work items than CTAs, most of them short, so the
    # persistent CTAs claim items from the shared counter many times over and
    # the tensor-core kernel's item queue wraps around repeatedly
    dt = torch.float64 if mode == "f64" else torch.float32
    g = torch.Generator().manual_seed(17)
    r = lambda *s: (torch.rand(*s, generator=g, dtype=torch.float64) * 2 - 1).to(dt).double()
    cases = []
    for i in range(300):
        m, n = 5 + (i * 7) % 150, 3 + (i * 11) % 140
        k = 0 if i % 3 == 0 else 1 + (i * 13) % 90
        cases.append((1.0 - 0.01 * i, r(m, k), "ip", r(k, n), "pj", 0.5, r(m, n), "ij"))
    dev = [(to_device(A, dt), la, to_device(B, dt), lb, to_device(C, dt), lc, al, be)
           for (al, A, la, B, lb, be, C, lc) in cases]
    for rep in range(2):  # a second execution of the same plan reuses the counter
        for d, c in zip(dev, cases):
            d[4].copy_(c[6].to(dt))
        tc.contract_batched(dev, mode=mode)
        assert tc.device_error() == 0
        worst = 0.0
        for (al, A, la, B, lb, be, C, lc), d in zip(cases, dev):
            ref, mag = oracle_ref(al, A, la, B, lb, be, C, lc)
            worst = max(worst, norm_err(d[4].cpu().double().numpy(), ref, mag))
        assert worst <= TOLS[mode], (rep, worst)
