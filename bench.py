"""Benchmark of the PSTT2-onepass hot path on GB300 (one JSON line on stdout).

Workload (the large streaming configuration): X is the Hilbert-type tensor
1/(x_{i1}+x_{i2}+x_{i3}+x_{i4}), x on a uniform grid of [1, 2], d = 4,
n = 256 (4.29e9 FP32 entries, 17.18 GB), eps = 1e-6, p = 10, rmax = 6.
One step = the whole hot path on one tensor: zero the sketches, sketch every
unfolding in one pass over X (the fused multi-sketch kernel), and form the
TT cores (FP64 TSQR/CPQR, rank rule, least-squares middle core, core
products).  `value` = entries/s with X resident in HBM; `e2e` = the same
through the C ABI with X in pinned HOST memory, copied to the device in 1 GiB
slabs inside the timed region, and the cores copied back.

Arms: default = this library (mixed BF16 tensor-core sketch; the FP64 GPU path
is timed beside it); --impl reference = the FP64 CPU oracle on a bounded
sample of the same workload (there is no other implementation of the method).
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "PSTT2 tensor entries/s and HBM roofline fraction, mixed vs FP64 GPU at eps=1e-6"
WORKLOAD = dict(dims=[256, 256, 256, 256], eps=1e-6, p=10, rmax=6, seed=1)
SLAB = 16  # last-mode slices per 1 GiB slab (256^3 * 4 B * 16 = 1 GiB)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--prec", default="bf16", choices=["bf16", "tf32"])
    ap.add_argument("--n", type=int, default=256, help="mode size (default: the 17 GB workload)")
    ap.add_argument("--mid", type=int, default=0,
                    help="size of the two middle modes (default n); a smaller value keeps the kernel's "
                         "tile shape on a smaller tensor (profiling)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--batch", type=int, default=512, help="tensors in the batched workload")
    ap.add_argument("--batched-only", action="store_true",
                    help="run only the batched workload (profiling); prints its own JSON line")
    ap.add_argument("--batch-prec", default="bf16,fp64", help="precisions of the batched workload")
    ap.add_argument("--batch-shape", default="",
                    help="fixed launch shape 'ta,chunk,ctas_per_sm' instead of the autotuner")
    return ap.parse_args()


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, mx, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [v.strip() for v in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
                power.append(float(f[3]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm),
                "power_w_max": max(power) if power else None}


# ------------------------------------------------------------------- peaks
def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d.get("hbm_gbs"), "measured"
    return 6800.0, "fallback"


def traffic_record(kernel_tag):
    """DRAM bytes per launch from the committed ncu summary, when it was taken
    on the current source of that kernel (else None)."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        rec = json.load(f)
    r = rec.get(kernel_tag)
    if not r:
        return None
    try:
        import hashlib
        src = open(os.path.join(ROOT, r["source"]), "rb").read()
        if hashlib.sha256(src).hexdigest()[:16] != r["source_sha"]:
            return None
    except OSError:
        return None
    return r["dram_bytes_per_launch"]


# -------------------------------------------------------------- CPU oracle
def cpu_sample(steps=1, n=128):
    """The FP64 oracle as it stands, on a bounded sample of the workload: the
    same Hilbert-type function at d = 4 with a smaller n (n = 128: 268M
    entries), same eps, p, rmax, one-pass.  Returns entries/s, the threads
    used, the sample description and the per-step times."""
    import numpy as np
    import ttinputs as ti
    from oracle import pstt2 as OP
    dims = [n] * 4
    x = ti.hilbert_type(dims, np.float32).astype(np.float64)
    times = []
    for _ in range(steps):
        t0 = time.perf_counter()
        OP.pstt2(x, dims, eps=WORKLOAD["eps"], rmax=WORKLOAD["rmax"], p=WORKLOAD["p"], seed=WORKLOAD["seed"],
                 passes=1)
        times.append(time.perf_counter() - t0)
    try:
        from threadpoolctl import threadpool_info
        cores = max([i.get("num_threads", 1) for i in threadpool_info()] + [1])
    except Exception:
        cores = os.cpu_count()
    return n ** 4 / statistics.median(times), cores, (
        f"oracle.pstt2 one-pass on the Hilbert-type tensor at d=4, n={n} ({n ** 4} entries), eps=1e-6, "
        f"p=10, rmax=6; entries/s = entries / wall time"), times


def reference_sample_n(steps, budget_s=150.0):
    """Largest sample size n in {32, 48, 64, 96, 128} whose `steps` oracle
    runs fit the time budget (cost scales with n^4; measured at n = 32)."""
    t32 = cpu_sample(1, 32)[3][0]
    best = 32
    for n in (48, 64, 96, 128):
        if t32 * (n / 32) ** 4 * steps <= budget_s:
            best = n
    return best


def run_reference(a):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    steps = max(1, a.steps)
    n = reference_sample_n(steps + min(a.warmup, 1))
    for _ in range(min(a.warmup, 1)):
        cpu_sample(1, n)
    v, cores, sample, times = cpu_sample(steps, n)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "entries/s", "n_gpus": a.gpus,
            "steps": steps, "warmup": a.warmup, "ms_per_step": 1e3 * statistics.median(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": f"Hilbert-type d=4 n=256 FP32 (bounded sample per step: n={n})",
                       "sample": sample},
            "cpu_baseline": {"value": v, "unit": "entries/s", "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": "entries/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- GPU arm
def batched_inputs(count, dev, seed=5):
    """The batched workload on the device: `count` FP32 tensors, d in {3..6},
    n in {8..32} (n^d <= 2e6), random N(0,1) TT cores of ranks in {2..16}
    (data seed 1000 + b), plus 1e-7 relative Gaussian noise; eps = 1e-5,
    p = 5, rmax = 16, test-matrix seed 1000 + b."""
    import numpy as np
    import torch
    import ttinputs as ti
    xs, probs = [], []
    gen = torch.Generator(device=dev)
    gen.manual_seed(seed)
    for b, (dims, r) in enumerate(ti.batch_specs(count=count, seed=seed, cap=2_000_000)):
        L = torch.ones(1, 1, dtype=torch.float64, device=dev)
        for G in ti.random_tt_cores(dims, r, seed=1000 + b):
            a_, n_, c_ = G.shape
            Gd = torch.from_numpy(np.asfortranarray(G).reshape(a_, n_ * c_, order="F")).to(dev)
            L = (L @ Gd).T.reshape(c_, n_, -1).permute(1, 2, 0).reshape(-1, c_)  # rows u + N i
        x = L[:, 0]
        e = torch.randn(x.numel(), dtype=torch.float64, device=dev, generator=gen)
        x = x + e * (1e-7 * x.norm() / e.norm())
        xs.append(x.to(torch.float32).contiguous())
        probs.append(dict(dims=dims, eps=1e-5, rmax=16, p=5, seed=1000 + b))
    return xs, probs


def run_batched(a, dev, P, stream):
    """Batched workload: one plan, one persistent sketch launch over all
    tensors + batched finalize, per precision; autotuned launch shape."""
    import numpy as np
    import torch
    import ttinputs as ti
    xs, probs = batched_inputs(a.batch, dev)
    ntot = sum(x.numel() for x in xs)
    out = {"workload": f"{a.batch} FP32 tensors, d in 3..6, n in 8..32 (n^d <= 2e6), TT ranks 2..16 + 1e-7 noise; "
                       f"eps=1e-5 p=5 rmax=16; {ntot} entries ({ntot * 4 / 1e9:.2f} GB)", "entries": ntot}
    for prec in a.batch_prec.split(","):
        t = P.TTSketch(None, batch=probs, x_dtype=torch.float32, prec=prec)
        if a.batch_shape:
            best = tuple(int(v) for v in a.batch_shape.split(","))
            t.batch_config(*best)
        else:
            best = t.autotune(xs, stream)
        stream.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        k = max(3, min(a.steps, 10))
        t.batched(xs, stream)
        e0.record(stream)
        for _ in range(k):
            t.batched(xs, stream)
        e1.record(stream)
        stream.synchronize()
        ms = e0.elapsed_time(e1) / k
        # accuracy on a sample of items (host contraction of the cores)
        errs = []
        for b in range(0, len(xs), max(1, len(xs) // 8)):
            xt = ti.contract_tt(t.core_list(b))
            xh = xs[b].double().cpu().numpy()
            errs.append(float(np.linalg.norm(xt - xh) / np.linalg.norm(xh)))
        out[prec] = {"value": ntot / (ms * 1e-3), "unit": "entries/s", "ms_per_step": ms,
                     "launch_shape": {"ta": best[0], "chunk": best[1], "ctas_per_sm": best[2]},
                     "max_rel_err_sampled": max(errs), "items_sampled": len(errs)}
        del t
    return out


def whole_job(ms_local, units_local, world, device=None):
    """Whole-job rate over `world` ranks: the step time is the MAX over ranks,
    the units are the SUM over ranks.  Returns (ms, units, units/s)."""
    if world > 1:
        import torch
        import torch.distributed as dist
        t = torch.tensor([ms_local], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        u = torch.tensor([float(units_local)], dtype=torch.float64, device=device)
        dist.all_reduce(u, op=dist.ReduceOp.SUM)
        ms_local, units_local = float(t.item()), float(u.item())
    return ms_local, units_local, units_local / (ms_local * 1e-3)


def run_batched_only(a):
    import torch
    import paper_2111_10448_gb300 as P
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", "0")))
    torch.cuda.set_device(dev)
    stream = torch.cuda.Stream(device=dev)
    out = run_batched(a, dev, P, stream)
    print(json.dumps({"batched": out}), flush=True)


def run_gpu(a):
    import torch
    import paper_2111_10448_gb300 as P
    from paper_2111_10448_gb300 import _native as N
    import ctypes as C

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    L = P.lib()
    n = a.n
    m = a.mid or n
    dims = [n, m, m, n]
    ntot = n * m * m * n
    Nd1 = n * m * m
    stream = torch.cuda.Stream(device=dev)
    sp = C.c_void_p(stream.cuda_stream)

    # X resident in HBM (generated on the device, not timed)
    X = torch.empty(ntot, dtype=torch.float32, device=dev)
    nn = (C.c_int64 * 4)(*dims)
    N.check(L.tt_generate_hilbert_type(4, nn, 0, n, C.c_void_p(X.data_ptr()), N.TT_F32, sp), "gen")
    stream.synchronize()

    kw = dict(eps=WORKLOAD["eps"], rmax=WORKLOAD["rmax"], p=WORKLOAD["p"], seed=WORKLOAD["seed"] + rank,
              x_dtype=torch.float32, device=dev)
    t = P.TTSketch(dims, prec=a.prec, **kw)

    def step(ev=None):
        t.begin(stream)
        if ev is not None:
            ev[0].record(stream)
        t.accumulate(X, 0, n, stream)
        if ev is not None:
            ev[1].record(stream)
        t.finalize(stream)

    for _ in range(a.warmup):
        step()
    stream.synchronize()
    if world > 1:
        torch.distributed.barrier()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(a.steps)]
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clk = ClockSampler(torch.cuda.get_device_properties(dev).index if hasattr(torch.cuda.get_device_properties(dev), "index") else local)
    clk.start()
    time.sleep(0.3)
    l0 = L.tt_kernel_launches()
    torch.cuda.synchronize(dev)
    if world > 1:
        torch.distributed.barrier()
    e0.record(stream)
    for i in range(a.steps):
        step(evs[i])
    e1.record(stream)
    torch.cuda.synchronize(dev)
    if world > 1:
        torch.distributed.barrier()
    l1 = L.tt_kernel_launches()
    clocks = clk.stop()
    ms, _, value = whole_job(e0.elapsed_time(e1) / a.steps, ntot, world, dev)
    sketch_ms = statistics.mean(s.elapsed_time(e) for s, e in evs)
    st, ranks = t.status(stream)

    # accuracy of this run: ||X - X~|| / ||X|| on the device
    err2 = t.error(X, stream)
    stream.synchronize()
    err2 = err2.cpu().numpy()
    rel_err = float((err2[0] / err2[1]) ** 0.5)

    out = {}
    # ---- FP64 GPU path, same eps (one step after one warm-up)
    if not a.no_fp64:
        f = P.TTSketch(dims, prec="fp64", **kw)
        f.pstt2(X, stream)
        stream.synchronize()
        g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        g0.record(stream)
        f.pstt2(X, stream)
        g1.record(stream)
        torch.cuda.synchronize(dev)
        f_ms = g0.elapsed_time(g1)
        fe = f.error(X, stream)
        # mixed vs FP64: ||X~_mixed - X~_fp64|| / ||X||
        Xf = f.reconstruct(torch.float32, stream=stream)
        d2 = t.error(Xf, stream)
        stream.synchronize()
        fe, d2 = fe.cpu().numpy(), d2.cpu().numpy()
        del Xf
        out["fp64_gpu"] = {"value": ntot / (f_ms * 1e-3), "unit": "entries/s", "ms_per_step": f_ms,
                           "rel_err_vs_X": float((fe[0] / fe[1]) ** 0.5),
                           "mixed_vs_fp64_rel": float((d2[0] / err2[1]) ** 0.5),
                           "ranks": f.status(stream)[1]}
        del f

    # ---- e2e: X from pinned host memory in 1 GiB slabs, cores back to host
    if not a.no_e2e:
        Xh = torch.empty(ntot, dtype=torch.float32, pin_memory=True)
        Xh.copy_(X)
        Xd = torch.empty_like(X)
        cores_h = torch.empty(t.cores.numel(), dtype=torch.float64, pin_memory=True)
        ranks_h = torch.empty(t.ranks.numel(), dtype=torch.int32, pin_memory=True)
        copy = torch.cuda.Stream(device=dev)
        slab = SLAB * Nd1
        group = 128 if n % 128 == 0 else n   # slices per accumulate (tensor-core M tile)

        def e2e_step():
            done = []
            for s0 in range(0, n, SLAB):
                with torch.cuda.stream(copy):
                    Xd[s0 * Nd1:(s0 + SLAB) * Nd1].copy_(Xh[s0 * Nd1:(s0 + SLAB) * Nd1], non_blocking=True)
                    ev = torch.cuda.Event()
                    ev.record(copy)
                done.append(ev)
            t.begin(stream)
            for g0_ in range(0, n, group):
                stream.wait_event(done[(g0_ + group) // SLAB - 1])
                t.accumulate(Xd[g0_ * Nd1:(g0_ + group) * Nd1], g0_, group, stream)
            t.finalize(stream)
            with torch.cuda.stream(stream):
                cores_h.copy_(t.cores, non_blocking=True)
                ranks_h.copy_(t.ranks, non_blocking=True)

        e2e_step()
        torch.cuda.synchronize(dev)
        h0 = time.perf_counter()
        k = max(1, min(a.steps, 3))
        for _ in range(k):
            e2e_step()
        torch.cuda.synchronize(dev)
        e_ms = (time.perf_counter() - h0) * 1e3 / k
        out["e2e"] = {"value": world * ntot / (e_ms * 1e-3), "unit": "entries/s", "ms_per_step": e_ms,
                      "h2d_bytes_per_step": ntot * 4,
                      "d2h_bytes_per_step": t.cores.numel() * 8 + t.ranks.numel() * 4}
        del Xh, Xd

    peak, peak_kind = measured_peaks()
    achieved = ntot * 4 / (sketch_ms * 1e-3) / 1e9
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": traffic_record(f"sketch_{a.prec}_{n}x{m}x{m}x{n}"), "peak_kind": f"{peak_kind} hbm_gbs",
                "kernel_ms": sketch_ms, "algorithmic_bytes": ntot * 4}

    if not a.no_batched:
        out["batched"] = run_batched(a, dev, P, stream)

    cpu = None
    if rank == 0 and not a.no_cpu:
        v, cores, sample, _ = cpu_sample(1)
        cpu = {"value": v, "unit": "entries/s", "cores": cores, "kind": "oracle", "sample": sample}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "entries/s", "n_gpus": world, "steps": a.steps,
                "warmup": a.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": a.prec, "data": "synthetic",
                "config": {"workload": f"Hilbert-type d=4 dims={dims} FP32 ({ntot * 4 / 1e9:.2f} GB) one-pass PSTT2, "
                                       f"eps=1e-6 p=10 rmax=6, {a.prec} tensor-core sketch with X split hi+lo, "
                                       "FP64 solves",
                           "l2": "inputs larger than L2 (no flush needed)",
                           "ranks": ranks, "status": st, "rel_err_vs_X": rel_err,
                           "parallelism": "replicas" if world > 1 else "single GPU"},
                "roofline": roofline, "cpu_baseline": cpu, "e2e": out.get("e2e"),
                "gpu_launches": int(l1 - l0), "clocks": clocks, "fp64_gpu": out.get("fp64_gpu"),
                "batched": out.get("batched")}
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def main():
    a = parse()
    if a.impl == "reference":
        run_reference(a)
    elif a.batched_only:
        run_batched_only(a)
    else:
        run_gpu(a)


if __name__ == "__main__":
    main()
