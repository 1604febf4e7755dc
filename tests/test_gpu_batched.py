"""Batched form: tensors of uneven order, size and rank sketched by one
persistent launch and finalized together; per-item parity with the oracle,
equality with single-tensor plans, CUDA-graph capture and the autotuner.

Batch recipe (uneven shapes as in the batched workload: d in {3..6},
n in {8..32} clamped so that n^d stays under the entry cap, ranks in {2..16}
per bond, 1e-7 relative noise); item b uses data seed 1000 + b and
test-matrix seed 1000 + b; eps = 1e-5, p = 5, rmax = 16."""
import numpy as np
import pytest
import torch

import ttinputs as ti
from oracle import pstt2 as OP, tt as OT
from paper_2111_10448_gb300 import TTSketch

EPS, P, RMAX = 1e-5, 5, 16


def make_batch(count, cap, seed=5, dtype=np.float64):
    specs = ti.batch_specs(count=count, seed=seed, cap=cap)
    xs, probs = [], []
    for b, (dims, r) in enumerate(specs):
        xs.append(ti.random_tt(dims, r, seed=1000 + b, noise=1e-7, dtype=dtype))
        probs.append(dict(dims=dims, eps=EPS, rmax=RMAX, p=P, seed=1000 + b))
    return xs, probs


def run_batched(xs, probs, prec="fp64", x_dtype=torch.float64):
    t = TTSketch(None, batch=probs, x_dtype=x_dtype, prec=prec)
    dev = [torch.tensor(x, dtype=x_dtype, device="cuda") for x in xs]
    t.batched(dev)
    torch.cuda.synchronize()
    return t, dev


def full(cores):
    return OT.tt_full([np.asarray(G) for G in cores])


@pytest.mark.gpu
def test_batched_fp64_matches_oracle_per_item():
    xs, probs = make_batch(12, cap=20_000)
    t, _ = run_batched(xs, probs)
    st, ranks = t.status()
    assert st in (0, 7)
    worst = 0.0
    for b, (x, pr) in enumerate(zip(xs, probs)):
        o = OP.pstt2(x, pr["dims"], eps=EPS, rmax=RMAX, p=P, seed=pr["seed"], passes=1)
        got = full(t.core_list(b))
        err = np.linalg.norm(got - OT.tt_full(o["cores"])) / np.linalg.norm(x)
        worst = max(worst, err)
        assert err <= 1e-10, (b, pr["dims"], err)
    print(f"batched FP64 vs oracle: worst {worst:.2e} over {len(xs)} items")


@pytest.mark.gpu
def test_batched_bf16_within_10eps_of_oracle():
    xs, probs = make_batch(10, cap=30_000, seed=7, dtype=np.float32)
    t, _ = run_batched(xs, probs, prec="bf16", x_dtype=torch.float32)
    for b, (x, pr) in enumerate(zip(xs, probs)):
        x64 = x.astype(np.float64)
        o = OP.pstt2(x64, pr["dims"], eps=EPS, rmax=RMAX, p=P, seed=pr["seed"], passes=1)
        got = full(t.core_list(b))
        err = np.linalg.norm(got - OT.tt_full(o["cores"])) / np.linalg.norm(x64)
        assert err <= 10 * EPS, (b, pr["dims"], err)


@pytest.mark.gpu
def test_batched_equals_single_tensor_plans():
    xs, probs = make_batch(24, cap=200_000, seed=11)
    t, dev = run_batched(xs, probs)
    for b, (x, pr) in enumerate(zip(xs, probs)):
        s = TTSketch(pr["dims"], eps=EPS, rmax=RMAX, p=P, seed=pr["seed"], x_dtype=torch.float64)
        s.pstt2(dev[b])
        torch.cuda.synchronize()
        a, c = full(t.core_list(b)), full(s.core_list(0))
        assert np.linalg.norm(a - c) <= 1e-11 * np.linalg.norm(x), b


@pytest.mark.gpu
def test_batched_graph_capture_replays():
    xs, probs = make_batch(16, cap=100_000, seed=13)
    t, dev = run_batched(xs, probs)          # first call: tables go to the workspace
    ref_cores, ref_ranks = t.cores.clone(), t.ranks.clone()
    refs = [full(t.core_list(b)) for b in range(len(xs))]
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        t.batched(dev, stream=torch.cuda.current_stream())
    for _ in range(2):
        t.cores.fill_(float("nan"))
        t.ranks.fill_(-1)
        g.replay()
        torch.cuda.synchronize()
        assert torch.equal(t.ranks, ref_ranks)
        for b in range(len(xs)):
            got = full(t.core_list(b))
            assert np.linalg.norm(got - refs[b]) <= 1e-11 * np.linalg.norm(refs[b]), b
    del ref_cores


@pytest.mark.gpu
def test_autotuner_picks_a_candidate_and_keeps_results():
    xs, probs = make_batch(32, cap=300_000, seed=17)
    t, dev = run_batched(xs, probs)
    refs = [full(t.core_list(b)) for b in range(len(xs))]
    best = t.autotune(dev)
    assert best[0] in (32, 64) and best[1] in (1, 4, 16) and best[2] in (2, 4, 8), best
    for b in range(len(xs)):
        assert np.linalg.norm(full(t.core_list(b)) - refs[b]) <= 1e-11 * np.linalg.norm(refs[b]), b
    t.batched(dev)
    torch.cuda.synchronize()
    for b in range(len(xs)):
        assert np.linalg.norm(full(t.core_list(b)) - refs[b]) <= 1e-11 * np.linalg.norm(refs[b]), b
    print("autotuned batched launch shape (ta, chunk, ctas/SM):", best)


@pytest.mark.gpu
@pytest.mark.parametrize("prec", ["bf16", "tf32", "fp16"])
def test_batched_small_plane_matches_single_plans_and_oracle(prec):
    """Mixed-precision batch whose items all fit the small-plane kernel
    (n_1, n_d <= 32): each item within 10 eps of the FP64 oracle and of its
    own single-tensor plan (the two differ only in FP32 accumulation order).
    FP16 items carry their own scale (each item's largest |X|)."""
    xs, probs = make_batch(24, cap=200_000, seed=19, dtype=np.float32)
    if prec == "fp16":
        for x, pr in zip(xs, probs):
            pr["x_scale_log2"] = 15 - int(np.frexp(float(np.max(np.abs(x))))[1])
    t, dev = run_batched(xs, probs, prec=prec, x_dtype=torch.float32)
    st, _ = t.status()
    assert st in (0, 7)
    for b, (x, pr) in enumerate(zip(xs, probs)):
        x64 = x.astype(np.float64)
        s = TTSketch(pr["dims"], eps=EPS, rmax=RMAX, p=P, seed=pr["seed"], x_dtype=torch.float32, prec=prec,
                     x_scale_log2=pr.get("x_scale_log2", 0))
        s.pstt2(dev[b])
        torch.cuda.synchronize()
        got, single = full(t.core_list(b)), full(s.core_list(0))
        o = OP.pstt2(x64, pr["dims"], eps=EPS, rmax=RMAX, p=P, seed=pr["seed"], passes=1)
        nx = np.linalg.norm(x64)
        assert np.linalg.norm(got - OT.tt_full(o["cores"])) <= 10 * EPS * nx, (b, pr["dims"])
        assert np.linalg.norm(got - single) <= 10 * EPS * nx, (b, pr["dims"])


@pytest.mark.gpu
def test_batched_bf16_graph_capture_replays():
    xs, probs = make_batch(16, cap=100_000, seed=23, dtype=np.float32)
    t, dev = run_batched(xs, probs, prec="bf16", x_dtype=torch.float32)
    ref_ranks = t.ranks.clone()
    refs = [full(t.core_list(b)) for b in range(len(xs))]
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        t.batched(dev, stream=torch.cuda.current_stream())
    for _ in range(2):
        t.cores.fill_(float("nan"))
        t.ranks.fill_(-1)
        g.replay()
        torch.cuda.synchronize()
        assert torch.equal(t.ranks, ref_ranks)
        for b in range(len(xs)):
            got = full(t.core_list(b))
            # the same launch replayed: FP32 slot sums are added into the FP64
            # sketches by atomics, so only their order may differ
            assert np.linalg.norm(got - refs[b]) <= 1e-6 * np.linalg.norm(refs[b]), b


@pytest.mark.gpu
def test_autotuner_small_plane_block_shape():
    """BF16 small-plane batch: the autotuner picks a block shape (largest kR
    count per 16-plane block) and units per grab among its candidates, and
    the decomposition it leaves stays within 10 eps of the oracle."""
    xs, probs = make_batch(20, cap=200_000, seed=29, dtype=np.float32)
    t, dev = run_batched(xs, probs, prec="bf16", x_dtype=torch.float32)
    best = t.autotune(dev)
    assert best[0] in (1, 2, 4, 8) and best[1] in (1, 4, 8) and best[2] == 1, best
    for b, (x, pr) in enumerate(zip(xs, probs)):
        x64 = x.astype(np.float64)
        o = OP.pstt2(x64, pr["dims"], eps=EPS, rmax=RMAX, p=P, seed=pr["seed"], passes=1)
        err = np.linalg.norm(full(t.core_list(b)) - OT.tt_full(o["cores"])) / np.linalg.norm(x64)
        assert err <= 10 * EPS, (b, pr["dims"], err)
    print("autotuned small-plane batched shape (kR per block, chunk, ctas/SM):", best)


@pytest.mark.gpu
@pytest.mark.parametrize("shape", [1, 2, 4, 8])
def test_batched_small_plane_every_block_shape(shape):
    """Every block shape of the small-plane batched kernel (largest number of
    kR values per 16-plane block, so one-kR blocks of items with several kR
    values too) gives a decomposition within 10 eps of the oracle."""
    xs, probs = make_batch(16, cap=200_000, seed=31, dtype=np.float32)
    t = TTSketch(None, batch=probs, x_dtype=torch.float32, prec="bf16")
    t.batch_config(shape, 4, 1)
    dev = [torch.tensor(x, dtype=torch.float32, device="cuda") for x in xs]
    t.batched(dev)
    torch.cuda.synchronize()
    for b, (x, pr) in enumerate(zip(xs, probs)):
        x64 = x.astype(np.float64)
        o = OP.pstt2(x64, pr["dims"], eps=EPS, rmax=RMAX, p=P, seed=pr["seed"], passes=1)
        err = np.linalg.norm(full(t.core_list(b)) - OT.tt_full(o["cores"])) / np.linalg.norm(x64)
        assert err <= 10 * EPS, (shape, b, pr["dims"], err)


@pytest.mark.gpu
def test_autotuner_cache(tmp_path, monkeypatch):
    """TT_TUNE_CACHE: the first call tunes and appends one line; a second plan
    of the same batch takes the stored shape without timing (a planted line,
    a valid candidate, wins over the tuned one) and still leaves a valid
    decomposition."""
    xs, probs = make_batch(12, cap=100_000, seed=29, dtype=np.float32)
    cache = tmp_path / "tune.txt"
    monkeypatch.setenv("TT_TUNE_CACHE", str(cache))
    dev = [torch.tensor(x, dtype=torch.float32, device="cuda") for x in xs]
    t = TTSketch(None, batch=probs, x_dtype=torch.float32, prec="bf16")
    best = t.autotune(dev)
    lines = cache.read_text().split("\n")
    lines = [l for l in lines if l]
    assert len(lines) == 1 and tuple(int(v) for v in lines[0].split()[1:]) == best
    key = lines[0].split()[0]
    if best[0] in (1, 2, 4, 8):   # small-plane batch: (kR values per block, blocks per grab, 1)
        planted = (1, 1, 1) if best != (1, 1, 1) else (1, 4, 1)
    else:                         # generic tile kernel: (64, tiles per grab, CTAs per SM)
        planted = (64, 1, 2) if best != (64, 1, 2) else (64, 4, 4)
    with open(cache, "a") as f:
        f.write(f"{key} {planted[0]} {planted[1]} {planted[2]}\n")
    t2 = TTSketch(None, batch=probs, x_dtype=torch.float32, prec="bf16")
    assert t2.autotune(dev) == planted
    assert len([l for l in cache.read_text().split("\n") if l]) == 2
    torch.cuda.synchronize()
    for b in range(len(xs)):
        g1, g2 = full(t.core_list(b)), full(t2.core_list(b))
        assert np.linalg.norm(g1 - g2) <= 1e-5 * np.linalg.norm(xs[b])
