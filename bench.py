"""Throughput of BrawsCPD / AdawsCPD iterations on one or more GB300s.

A step is one SGD iteration of the whole path (mode draw, importance
sampling, sampled KRP rows, fiber gather, weighted gradient, AdaGrad step,
CDF refresh) on the 1000^3 BF16 tensor, R = 50, B = 2048, Euclidean
sampling. Before the timed region the gradient engine and CTA cap are
chosen by cpd_autotune (timing the applicable candidates). Inputs are synthetic (lognormal-scaled N(0,1) factors, 1e-2
noise), generated on the device; the three mode replicas (6 GB) are far
larger than L2, so no flush is needed between iterations.

Prints one JSON line (rank 0). --impl reference times the FP64 CPU oracle on
the same workload instead (rank 0 only).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import time

import torch

# The serving workload runs one stream per request; with CUDA's default of 8
# hardware work queues, streams beyond the eighth share queues and serialise.
# Must be set before the CUDA context exists.
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "SGD iters/s & fiber-gather GB/s vs HBM peak; batched solves/s, p99 @ equal fit"
DEFAULT_WORKLOAD = "c4_1000cube_bf16"
# The sources each engine's gradient kernel is compiled from: a committed traffic
# figure applies while their hash is the one recorded beside it.
_CSRC = "paper_2103_04081_gb300/csrc/"
_COMMON = [_CSRC + "cpd_device.cuh", _CSRC + "cpd_tcgen05.cuh", _CSRC + "cpd_internal.h"]
KERNEL_SOURCES = {"cluster": [_CSRC + "cpd_tcc.cu"] + _COMMON, "tensor": [_CSRC + "cpd_tc.cu"] + _COMMON,
                  "persistent": [_CSRC + "cpd_pers.cu"] + _COMMON, "fused": [_CSRC + "cpd_fused.cu"] + _COMMON,
                  "simt": [_CSRC + "cpd_kernels.cu"] + _COMMON}


def kernel_hash(engine: str) -> str:
    h = hashlib.sha256()
    for p in KERNEL_SOURCES.get(engine, KERNEL_SOURCES["simt"]):
        with open(os.path.join(ROOT, p), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def measured_peaks() -> tuple[dict, str]:
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


def ncu_traffic(engine: str) -> float | None:
    """DRAM bytes per launch of the gradient kernel from the committed ncu summary,
    if that summary was taken on the current kernel sources."""
    p = os.path.join(ROOT, "profiles", f"grad_{engine}_c4_traffic.txt")
    if not os.path.exists(p):
        return None
    txt = open(p).read()
    m_hash = re.search(r"kernel_sources_sha256_16=(\w+)", txt)
    m_b = re.search(r"dram_bytes_per_full_launch=([0-9.eE+]+)", txt)
    if not m_hash or not m_b or m_hash.group(1) != kernel_hash(engine):
        return None
    return float(m_b.group(1))


class Clocks:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.idx = device_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.proc:
            time.sleep(0.2)
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.out, _ = self.proc.communicate()

    def summary(self) -> dict:
        rows = []
        for line in (self.out or "").strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) >= 9:
                rows.append(f)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[q] for r in rows for q in range(4) if r[5 + q].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def dist_setup():
    """One process per GPU (replicas: every rank runs its own decomposition).
    NCCL when GPUs are present, gloo otherwise (host-side tests)."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
            dist.init_process_group("nccl")
        else:
            dist.init_process_group("gloo")
        return dist, rank, world, local
    return None, 0, 1, 0


def max_over_ranks(dist, value: float, device: str) -> float:
    """The slowest rank's time: the job is done when every replica is."""
    if not dist:
        return value
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world: int, steps: int, max_ms: float) -> float:
    """Iterations per second over all replicas (weak scaling: each rank runs
    `steps` iterations of its own decomposition)."""
    return world * steps / (max_ms / 1e3)


def make_inputs(w: dict, rank: int, device: str):
    from paper_2103_04081_gb300 import inputs as IN
    A = IN.factors(w["dims"], w["R"], w["data_seed"] + rank, congruence=w["congruence"],
                   lognormal_rows=w["lognormal_rows"], device=device)
    X = IN.cp_tensor(A, w["noise"], w["data_seed"] + rank, w["x_dtype"])
    A0 = IN.init_factors(w["dims"], w["R"], w["init_seed"] + rank,
                         dtype=torch.float64 if w["x_dtype"] == "f64" else torch.float32)
    if X.is_cuda:
        # X is written on torch's current stream; cpd_init reads it on the
        # side stream the context is built on, which is not ordered after it
        torch.cuda.synchronize()
    return X, A0


def cfg_kwargs(w: dict, rank: int, engine: str) -> dict:
    return dict(dims=w["dims"], R=w["R"], B=w["B"], x_dtype=w["x_dtype"], sampling=w["sampling"],
                step=w["step"], alpha=w.get("alpha", 0.1), eta=w.get("eta", 0.1), b=w.get("b", 1e-12),
                seed=w["sample_seed"] + rank, engine=engine)


def _oracle_rate(O, ocfg, xb, A0: list, budget_s: float, omp: bool) -> tuple[float, int, float]:
    """Consecutive oracle iterations from A0 for about budget_s seconds."""
    import numpy as np
    A = [a.double().numpy().copy() for a in A0]
    S = [np.zeros_like(a) for a in A]
    O.run(ocfg, 0, 1, None, A, S, xbuf=xb, omp=omp)          # warm-up iteration
    it, t1 = 0, time.time()
    while time.time() - t1 < budget_s or it < 2:
        st = O.run(ocfg, 1 + it, 1, None, A, S, xbuf=xb, omp=omp)
        assert st == O.OK, st
        it += 1
    el = time.time() - t1
    return it / el, it, el


def oracle_baseline(w: dict, X_dev: torch.Tensor, A0: list, budget_s: float, all_cores: bool = True) -> dict:
    """The FP64 CPU oracle, as it stands, on a bounded sample of the workload:
    consecutive iterations from the same initial factors for about budget_s
    seconds, single-threaded (the checker build); then the timing-only build
    of the same source that spreads the fiber gather and the contraction rows
    over every host core."""
    import numpy as np

    from oracle import oracle as O
    t0 = time.time()
    if X_dev.dtype == torch.bfloat16:
        xb = X_dev.cpu().view(torch.int16).numpy().view(np.uint16)
    else:
        xb = X_dev.cpu().numpy()
    ocfg = O.Config(dims=tuple(w["dims"]), R=w["R"], B=w["B"], sampling=w["sampling"], step=w["step"],
                    x_dtype=w["x_dtype"], alpha=w.get("alpha", 0.1), eta=w.get("eta", 0.1),
                    b=w.get("b", 1e-12), seed=w["sample_seed"])
    prep = time.time() - t0
    rate, it, el = _oracle_rate(O, ocfg, xb, A0, budget_s, omp=False)
    ncores = os.cpu_count() or 1
    out = {"value": rate, "unit": "iters/s", "cores": 1, "cores_used": 1, "cores_on_box": ncores,
           "kind": "oracle", "iterations": it,
           "sample": f"{it} consecutive oracle iterations of the {w['name']} workload "
                     f"({el:.1f} s single-threaded FP64 C; host copy {prep:.1f} s not timed)"}
    if all_cores:
        os.environ.setdefault("OMP_NUM_THREADS", str(ncores))
        r2, it2, el2 = _oracle_rate(O, ocfg, xb, A0, budget_s / 2, omp=True)
        out["all_cores"] = {"value": r2, "unit": "iters/s", "cores_used": int(os.environ["OMP_NUM_THREADS"]),
                            "iterations": it2,
                            "sample": f"{it2} consecutive iterations, {el2:.1f} s, the OpenMP build of the "
                                      "same oracle source (fiber gather and contraction rows over the cores)"}
    return out


def error_vs_oracle(C, dev: str, stream, kw: dict, steps_tf: int = 3, free_iters: int = 500) -> dict:
    """Error of the GPU path against the FP64 oracle, stated beside the numbers:
    (1) at the bench workload, teacher-forced iterations in the bench's launch
    configuration (the oracle starts from the GPU's state at t): indices and
    probabilities bit-exact, the gradient's relative Frobenius error and its
    largest row error against the row's componentwise scale, the updated
    factor's largest relative row error; (2) on the 120^4 BF16 workload (the
    tensor-core path), free runs of both from the same start near the solution
    for free_iters iterations, compared by the oracle's Tol routine."""
    import math

    import numpy as np

    from oracle import oracle as O
    from paper_2103_04081_gb300 import inputs as IN
    res = {}
    w = dict(IN.WORKLOADS[DEFAULT_WORKLOAD])
    X, A0 = make_inputs(w, 0, dev)
    with torch.cuda.stream(stream):
        dec = C.Decomposition(X, [a.to(dev) for a in A0], stream=stream, **kw)
    xb = X.cpu().view(torch.int16).numpy().view(np.uint16) if X.dtype == torch.bfloat16 else X.cpu().numpy()
    del X
    dec.sgd_iters(50, stream)
    torch.cuda.synchronize()
    ocfg = O.Config(dims=tuple(w["dims"]), R=w["R"], B=w["B"], sampling=w["sampling"], step=w["step"],
                    x_dtype=w["x_dtype"], eta=w["eta"], b=w["b"], seed=w["sample_seed"])
    worst = {"G_frobenius": 0.0, "G_row_scaled": 0.0, "A_row": 0.0}
    exact = True
    for _ in range(steps_tf):
        t = dec.t
        A = [a.double().numpy().copy() for a in dec.factors("cpu", stream)]
        Ap = [a.copy() for a in A]
        S = [s.numpy().copy() for s in dec.adagrad()]
        out = O.step(ocfg, t, None, A, S, xbuf=xb)
        dec.sgd_iters(1, stream)
        torch.cuda.synchronize()    # the reads below use the default stream
        n, idx, p = dec.last_sample()
        _, G = dec.last_gradient()
        exact = exact and n == out["n"] and bool(np.array_equal(idx.numpy().astype(np.int64), out["idx"])) \
            and bool(np.array_equal(p.numpy(), out["p"]))
        Gg = G.numpy().astype(np.float64)
        sc = O.grad_row_scale(w["dims"], n, out["idx"], out["p"], Ap, xb, w["x_dtype"], w["B"])
        An = dec.factors("cpu", stream)[n].double().numpy()
        worst["G_frobenius"] = max(worst["G_frobenius"],
                                   float(np.linalg.norm(Gg - out["G"]) / np.linalg.norm(out["G"])))
        worst["G_row_scaled"] = max(worst["G_row_scaled"],
                                    float(np.max(np.linalg.norm(Gg - out["G"], axis=1) / sc)))
        den = np.maximum(np.linalg.norm(A[n], axis=1), np.linalg.norm(Ap[n], axis=1))
        worst["A_row"] = max(worst["A_row"], float(np.max(np.linalg.norm(An - A[n], axis=1) / den)))
    res["teacher_forced"] = {"workload": DEFAULT_WORKLOAD, "engine": dec.describe()["engine"],
                             "iterations": steps_tf, "indices_and_probabilities_bit_exact": exact, **worst}
    dec.close()
    del xb
    # free runs on the 120^4 BF16 workload
    w3 = dict(IN.WORKLOADS["c3_120pow4_bf16"])
    A3 = IN.factors(w3["dims"], w3["R"], w3["data_seed"], device=dev)
    X3 = IN.cp_tensor(A3, w3["noise"], w3["data_seed"], "bf16")
    # start 10% off the true factors, eta = 0.1: the regime near the solution
    # where the BF16 path's rounding matters most
    g3 = torch.Generator().manual_seed(w3["init_seed"])
    A30 = [(a.cpu() * (1.0 + 0.1 * torch.randn(a.shape, generator=g3, dtype=torch.float64))).float() for a in A3]
    eta3 = 0.1
    with torch.cuda.stream(stream):
        d3 = C.Decomposition(X3, [a.to(dev) for a in A30], stream=stream, dims=w3["dims"], R=w3["R"],
                             B=w3["B"], x_dtype="bf16", sampling=w3["sampling"], step=w3["step"],
                             eta=eta3, b=w3["b"], seed=w3["sample_seed"])
    xb3 = X3.cpu().view(torch.int16).numpy().view(np.uint16)
    del X3
    d3.sgd_iters(free_iters, stream)
    Ag = [a.double().numpy() for a in d3.factors("cpu", stream)]
    eng3 = d3.describe()["engine"]
    d3.close()
    oc3 = O.Config(dims=tuple(w3["dims"]), R=w3["R"], B=w3["B"], sampling=w3["sampling"], step=w3["step"],
                   x_dtype="bf16", eta=eta3, b=w3["b"], seed=w3["sample_seed"])
    Ao = [a.double().numpy().copy() for a in A30]
    So = [np.zeros_like(a) for a in Ao]
    assert O.run(oc3, 0, free_iters, None, Ao, So, xbuf=xb3, omp=True) == O.OK
    tg, _ = O.tol_blas(xb3, w3["dims"], Ag, "bf16")
    to, _ = O.tol_blas(xb3, w3["dims"], Ao, "bf16")
    res["free_run"] = {"workload": "c3_120pow4_bf16", "engine": eng3, "iterations": free_iters,
                       "start": "true factors x (1 + 0.1 N(0,1)), eta 0.1",
                       "fit_gpu": 1 - math.sqrt(tg), "fit_oracle": 1 - math.sqrt(to),
                       "fit_diff": (1 - math.sqrt(tg)) - (1 - math.sqrt(to)),
                       "factor_drift": max(float(np.linalg.norm(a - b) / np.linalg.norm(b))
                                           for a, b in zip(Ag, Ao))}
    return res


def fit_pass(C, dec, w: dict, stream, reps: int = 5) -> dict:
    """The stop check of Sec. 5.2 (one pass over the mode-1 replica): mean
    device time of cpd_fit_start's launches (operand preparation, the pass,
    the fold) over `reps` passes, CUDA events on the launching stream, and the
    replica bytes it reads per pass against the measured copy peak."""
    esize = {"bf16": 2, "f32": 4, "f64": 8}[w["x_dtype"]]
    I0 = w["dims"][0]
    J = 1
    for d in w["dims"][1:]:
        J *= d
    rbytes = J * ((I0 + 7) // 8 * 8) * esize
    C.cpd_fit_start(dec.ctx, stream)
    while C.cpd_fit_poll(dec.ctx) is None:
        time.sleep(1e-4)
    ms = _event_ms(stream, lambda: [C.cpd_fit_start(dec.ctx, stream) for _ in range(reps)]) / reps
    while C.cpd_fit_poll(dec.ctx) is None:
        time.sleep(1e-4)
    peaks, _ = measured_peaks()
    gbs = rbytes / (ms * 1e-3) / 1e9
    return {"kernel": "k_fit_tc" if dec.describe().get("fit_pass") == "tensor" else "k_fit",
            "ms_per_pass": ms, "replica_bytes_read": rbytes, "gbs": gbs, "frac": gbs / peaks["hbm_gbs"],
            "note": "read-only pass, against the copy peak (read + write)"}


def _event_ms(stream, fn) -> float:
    """Device time of fn's work on `stream` (CUDA events on that stream)."""
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    fn()
    e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1)


def gather_per_mode(C, X, A0: list, w: dict, dev: str, stream, peak: float, K: int = 32, reps: int = 10) -> dict:
    """The fiber gather in bulk, per mode: cpd_skrp draws K = 32 mini-batches
    of one mode (Alg. 3) and gathers their K B fibers (Alg. 1) in one launch
    over every SM, (a) writing the fibers only and (b) also p_f, the
    multi-indices and the sampled KRP rows. The fibers are read once and
    written once, like the measured copy peak, so `frac` = (bytes read +
    bytes written) / time / peak; `gather_gbs` counts the useful fiber bytes
    (K B I_n elem) alone. CUDA events over `reps` launches with fresh draws
    each, on the launching stream; the replicas are far larger than L2."""
    kw = cfg_kwargs(w, 0, "auto")
    with torch.cuda.stream(stream):
        dec = C.Decomposition(X, [a.to(dev) for a in A0], stream=stream, **kw)
    esize = {"bf16": 2, "f32": 4, "f64": 8}[w["x_dtype"]]
    tdt = {"bf16": torch.bfloat16, "f32": torch.float32}[w["x_dtype"]]
    N, B, R = len(w["dims"]), w["B"], w["R"]
    out = {"K": K, "B": B, "launches_timed": reps, "kernel": "k_skrp",
           "peak": "hbm_gbs of MEASURED_PEAKS.json (a copy: bytes read + bytes written)", "modes": []}
    idx = torch.empty(K * B, N, dtype=torch.int32, device=dev)
    p = torch.empty(K * B, dtype=torch.float64, device=dev)
    Z = torch.empty(K * B, R, dtype=torch.float32, device=dev)
    side = K * B * (N * 4 + 8 + R * 4)          # idx, p and Z written
    t0 = K
    for n, In in enumerate(w["dims"]):
        ld = (In + 7) // 8 * 8
        Xs = torch.empty(K * B * ld, dtype=tdt, device=dev)
        fib = K * B * ld * esize                  # fiber bytes read (= written)
        row = {"mode": n, "I_n": In, "useful_bytes_per_launch": K * B * In * esize}
        # fibers only (the draws and the gather), then every output of Alg. 3 + Alg. 1
        for name, outs, moved in (("fibers_only", (None, None, None), 2 * fib), ("all_outputs", (idx, p, Z), 2 * fib + side)):
            C.cpd_skrp(dec.ctx, n, 0, K, *outs, Xs, stream)
            ms = _event_ms(stream, lambda: [C.cpd_skrp(dec.ctx, n, t0 + K * r, K, *outs, Xs, stream)
                                            for r in range(reps)]) / reps
            t0 += K * reps
            row[name] = {"ms_per_launch": ms, "bytes_moved_per_launch": moved,
                         "gather_gbs": row["useful_bytes_per_launch"] / (ms * 1e-3) / 1e9,
                         "copy_equivalent_gbs": moved / (ms * 1e-3) / 1e9,
                         "frac": moved / (ms * 1e-3) / 1e9 / peak}
        out["modes"].append(row)
        del Xs
    dec.close()
    return out


def batched_form(C, X, A0: list, w: dict, dev: str, stream, peak: float, G: int, cs: int,
                 iters: int) -> dict:
    """The batched form: G decompositions of the workload (own seeds) advanced by
    one grouped persistent launch per call (one thread-block cluster each);
    aggregate iterations/s and the fiber-gather GB/s they imply (B I_n elem per
    iteration), steady state after 100 untimed iterations."""
    decs = []
    for q in range(G):
        kw = cfg_kwargs(w, 0, "persistent")
        kw["max_ctas"] = cs
        kw["seed"] = w["sample_seed"] + 1000 + q
        with torch.cuda.stream(stream):
            decs.append(C.Decomposition(X, [a.to(dev) for a in A0], stream=stream, **kw))
    grp = C.cpd_group_create([d.ctx for d in decs], stream)
    C.cpd_group_iters(grp, 100, stream)
    ms = _event_ms(stream, lambda: C.cpd_group_iters(grp, iters, stream))
    C.cpd_group_destroy(grp)
    fits = [d.fit(stream)[0] for d in decs]
    for d in decs:
        d.close()
    esize = {"bf16": 2, "f32": 4, "f64": 8}[w["x_dtype"]]
    In = sum(w["dims"]) / len(w["dims"])
    agg = G * iters / (ms * 1e-3)
    gbs = agg * w["B"] * In * esize / 1e9
    return {"decompositions": G, "cluster": cs, "iterations_each": iters, "launches": 1,
            "aggregate_iters_per_s": agg, "gather_gbs": gbs, "frac": gbs / peak,
            "mean_fit_after": statistics.fmean(fits)}


def run_reference(args, w: dict) -> None:
    dist, rank, world, local = dist_setup()
    if rank != 0:
        return
    dev = f"cuda:{local}" if torch.cuda.is_available() else "cpu"
    X, A0 = make_inputs(w, 0, dev)
    budget = max(10.0, min(60.0, 1.0 * args.steps))
    base = oracle_baseline(w, X, A0, budget, all_cores=False)
    line = {"impl": "reference", "metric": METRIC, "value": base["value"], "unit": "iters/s",
            # a step is one oracle iteration; the number timed is bounded by a time
            # budget (10-60 s of single-core CPU work) rather than by --steps
            "n_gpus": args.gpus, "steps": base["iterations"], "warmup": 1, "ms_per_step": 1000.0 / base["value"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config_block(w, "oracle"),
            "cpu_baseline": base,
            "e2e": {"value": base["value"], "unit": "iters/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# B = 512 and eta = 0.2: the pair with the most requests reaching the target and
# the fewest iterations in a sweep of B in {256, 512, 1024, 2048} x eta in
# {0.1, 0.2} over the first 24 requests, each run alone.
SERVE = dict(requests=512, rate=200.0, stop_fit=0.98, max_iters=20000, fit_every=256,
             sampling="euclidean", step="adagrad", eta=0.2, b=1e-12, B=512, max_ctas=8,
             engine_r16="tensor", grouping=True, engine="classic", cluster=2,
             client_gb=64.0, strided_fraction=0.25, plain_sample=128, match=1e-3)


def serve_batch(q: dict) -> int:
    """Mini-batch size of a serving request (fibers per iteration)."""
    return SERVE["B"]


def serve_cfg(q: dict, x_dtype: str, engine: str = "auto", max_ctas: int = 0):
    from paper_2103_04081_gb300 import cpd as C
    return C.make_config(dims=q["dims"], R=q["R"], B=serve_batch(q), x_dtype=x_dtype,
                         sampling=SERVE["sampling"], step=SERVE["step"], eta=SERVE["eta"],
                         b=SERVE["b"], seed=q["sample_seed"], engine=engine, max_ctas=max_ctas)


def pct(v: list, q: float) -> float:
    v = sorted(v)
    k = min(len(v) - 1, max(0, int(round(q / 100.0 * (len(v) - 1)))))
    return v[k]


class TensorRing:
    """Device buffer from which the client carves each request's BF16 tensor
    while it waits for admission (the server copies it into its own layout at
    admission, after which the space is free again); allocations are released
    in about the order they were made, as a ring."""

    def __init__(self, nbytes: int, dev: str):
        self.buf = torch.empty(nbytes, dtype=torch.uint8, device=dev)
        self.cap, self.live = nbytes, []          # [offset, size, released] in allocation order
        self.head = 0                             # next free offset

    def _first(self) -> int:
        while self.live and self.live[0][2]:
            self.live.pop(0)
        return self.live[0][0] if self.live else -1

    def alloc(self, nbytes: int):
        nbytes = (nbytes + 255) // 256 * 256
        first = self._first()
        if first < 0:
            self.head = 0
            off = 0 if nbytes <= self.cap else -1
        elif self.head > first:                   # free: [head, cap) and [0, first)
            off = self.head if self.head + nbytes <= self.cap else (0 if nbytes <= first else -1)
        else:                                     # free: [head, first)
            off = self.head if self.head + nbytes <= first else -1
        if off < 0:
            return None, None
        rec = [off, nbytes, False]
        self.live.append(rec)
        self.head = off + nbytes
        return self.buf[off:off + nbytes], rec

    @staticmethod
    def release(rec) -> None:
        rec[2] = True


def serve_materialize(q: dict, dev: str, out: torch.Tensor | None = None):
    """A request's BF16 tensor (one pass on the device) and initial factors."""
    from paper_2103_04081_gb300 import inputs as IN
    A = IN.factors(q["dims"], q["R"], q["data_seed"], device=dev)
    X = IN.cp_tensor_streamed(A, q["noise"], q["data_seed"], "bf16", out=out)
    A0 = [a.to(dev) for a in IN.init_factors(q["dims"], q["R"], q["init_seed"])]
    return X, A0


def serve_bench(dev: str, n_req: int, n_plain: int, max_active: int) -> dict:
    """The serving workload: a Poisson stream of 3- and 4-way BF16 requests,
    every mode size uniform in [50, 400], served concurrently by the native
    server under an HBM budget. A request's tensor is generated on the device
    as soon as it has arrived and there is room (the client carves it from a
    64 GB ring and releases it once the server has admitted the request and
    copied it); its time-to-fit runs from its arrival to its stop, so time
    spent waiting for admission or generation counts. A request whose replicas
    would take more than a quarter of the budget runs with the strided layout
    on the CUDA-core engine.

    Then a seeded random sample of n_plain requests runs in the plain GPU form:
    one decomposition at a time, the engine and grid chosen for the whole GPU
    (no CTA cap), the same stopping rule. The comparison is at equal final
    fit: a sampled request counts when both forms stop within 1e-3 of each
    other or both reach the fit target."""
    from collections import deque

    import numpy as np

    from paper_2103_04081_gb300 import cpd as C
    from paper_2103_04081_gb300 import inputs as IN
    reqs = IN.serve_requests(n_req, rate=SERVE["rate"], seed=0)
    torch.cuda.synchronize()
    free, _ = torch.cuda.mem_get_info()
    ring = TensorRing(int(SERVE["client_gb"] * (1 << 30)), dev)
    budget = int(0.85 * (free - ring.cap))
    strided_mb = int(budget * SERVE["strided_fraction"]) >> 20
    srv = C.cpd_server_create(hbm_budget=budget, max_active=max_active, fit_every=SERVE["fit_every"],
                              grouping=SERVE["grouping"], strided_above_mb=strided_mb)

    sms = torch.cuda.get_device_properties(dev).multi_processor_count

    def engine_of(q):
        """Engine and CTA cap of a request: small requests share the GPU in
        grouped lanes with a cap of max_ctas; a request whose replicas let
        only `conc` such requests fit the budget at once gets about 2 x SMs /
        conc CTAs (a multiple of 8), so that the few large ones that run
        together still cover the GPU."""
        if SERVE["engine"] == "persistent":   # one thread-block cluster per request, grouped launches
            return "persistent", SERVE["cluster"]
        reps = 2 * sum(int(np.prod(q["dims"])) // d * ((d + 7) // 8 * 8) for d in q["dims"])
        conc = max(1, budget // max(reps, 1))
        cap = min(sms, max(SERVE["max_ctas"], ((2 * sms + conc - 1) // conc + 7) // 8 * 8))
        return (SERVE["engine_r16"] if q["R"] >= 16 else "simt"), cap

    gen_stream = torch.cuda.Stream()
    pending, arrived = deque(reqs), deque()
    live, done, gen_s = {}, {}, 0.0
    t0 = time.perf_counter()
    while pending or arrived or live:
        now = time.perf_counter() - t0
        while pending and pending[0]["arrival"] <= now:
            arrived.append(pending.popleft())
        moved = False
        # every arrived request is generated and submitted as soon as the ring
        # has room for its tensor: the server admits whichever fit its budget,
        # so a large request waiting for memory does not hold up small ones
        if arrived:
            q = arrived[0]
            nbytes = 2 * int(np.prod(q["dims"]))
            buf, rec = ring.alloc(nbytes)
            if buf is not None:
                # generated on a stream of its own and synchronised on that
                # stream alone: the server's worker may be capturing graphs,
                # which a device-wide synchronisation would break
                g0 = time.perf_counter()
                with torch.cuda.stream(gen_stream):
                    X, A0 = serve_materialize(q, dev, out=buf[:nbytes].view(torch.bfloat16))
                gen_stream.synchronize()
                gen_s += time.perf_counter() - g0
                eng, cap = engine_of(q)
                tk = C.cpd_submit(srv, serve_cfg(q, "bf16", eng, cap), X, A0, SERVE["stop_fit"], SERVE["max_iters"])
                live[tk] = [q, rec, A0, time.perf_counter() - t0]
                arrived.popleft()
                moved = True
        for tk in list(live):
            st, d = C.cpd_poll(srv, tk)
            entry = live[tk]
            if entry[1] is not None and d["t_start"] > 0:   # admitted: the server holds its own copy
                ring.release(entry[1])
                entry[1] = None
                moved = True
            if d["done"]:
                if entry[1] is not None:
                    ring.release(entry[1])
                done[tk] = (entry[0], st, d, entry[3])
                del live[tk]
                moved = True
        if not moved:
            time.sleep(2e-4)
    t1 = time.perf_counter()
    C.cpd_server_destroy(srv)
    del ring
    torch.cuda.empty_cache()

    ok = [(q, d, sub) for q, st, d, sub in done.values() if st == C.OK]
    # time-to-fit from arrival: the client's wait before submission plus the
    # server's submission-to-stop time (each on its own clock)
    ttf = [(sub - q["arrival"]) + (d["t_done"] - d["t_submit"]) for q, d, sub in ok]
    qwait = [(sub - q["arrival"]) + (d["t_start"] - d["t_submit"]) for q, d, sub in ok]
    span = t1 - t0
    by_i = {q["i"]: d for q, d, _ in ok}
    served = {"requests": n_req, "completed": len(ok), "solves_per_s": len(ok) / span, "wall_s": span,
              "ttf_p50_s": pct(ttf, 50), "ttf_p99_s": pct(ttf, 99), "queue_p50_s": pct(qwait, 50),
              "queue_p99_s": pct(qwait, 99), "reached": sum(d["reached"] for _, d, _ in ok) / max(1, len(ok)),
              "mean_fit": statistics.fmean(d["fit"] for _, d, _ in ok),
              "iters_total": sum(d["iters"] for _, d, _ in ok),
              "iters_per_s": sum(d["iters"] for _, d, _ in ok) / span,
              "strided_layout": sum(d["layout"] == 1 for _, d, _ in ok),
              "four_way": sum(q["N"] == 4 for q, _, _ in ok),
              "generation_s": gen_s}
    for name, sel in (("three_way", lambda q, d: q["N"] == 3),
                      ("four_way_replicas", lambda q, d: q["N"] == 4 and d["layout"] == 0),
                      ("strided", lambda q, d: d["layout"] == 1)):
        run = [d["t_done"] - d["t_start"] for q, d, _ in ok if sel(q, d)]
        if run:
            served["run_s_" + name] = {"n": len(run), "mean": statistics.fmean(run), "max": max(run)}
    out = {"workload": "serve_poisson200_3or4way_dims50to400_bf16", "served": served,
           "budget_gb": budget / 2**30, "strided_above_gb": strided_mb / 1024}
    if n_plain < 1:
        return out

    # plain GPU form on a seeded random sample, one decomposition at a time
    pick = sorted(np.random.default_rng(1).choice(len(reqs), size=min(n_plain, len(reqs)), replace=False))
    stream = torch.cuda.Stream()
    rows = []
    for i in pick:
        q = reqs[i]
        X, A0 = serve_materialize(q, dev)
        torch.cuda.synchronize()
        p0 = time.perf_counter()
        # the server's rule: replicas above the threshold -> the strided layout
        reps = 2 * sum(int(np.prod(q["dims"])) // d * ((d + 7) // 8 * 8) for d in q["dims"])
        cfg = serve_cfg(q, "bf16")
        if reps > strided_mb << 20:
            cfg.x_layout, cfg.engine = 1, 1
        with torch.cuda.stream(stream):
            ctx = C.cpd_init(cfg, X, A0, stream)
        del X
        it, fit = 0, 0.0
        while it < SERVE["max_iters"]:
            step = min(SERVE["fit_every"], SERVE["max_iters"] - it)
            C.cpd_sgd_iters(ctx, step, stream)
            it += step
            fit, _ = C.cpd_fit(ctx, stream)
            if fit >= SERVE["stop_fit"]:
                break
        C.cpd_destroy(ctx)
        rows.append((q["i"], time.perf_counter() - p0, fit, it))
        torch.cuda.empty_cache()
    sec = [r[1] for r in rows]
    matched = [r for r in rows if r[0] in by_i and (
        abs(by_i[r[0]]["fit"] - r[2]) <= SERVE["match"] or
        (by_i[r[0]]["fit"] >= SERVE["stop_fit"] and r[2] >= SERVE["stop_fit"]))]
    plain = {"requests": len(rows), "sample": "seeded random sample (numpy default_rng(1)) of the stream",
             "solves_per_s": len(rows) / sum(sec), "reached": sum(r[2] >= SERVE["stop_fit"] for r in rows) / len(rows),
             "mean_fit": statistics.fmean(r[2] for r in rows), "iters_total": sum(r[3] for r in rows),
             "served_mean_fit_same_requests": statistics.fmean(by_i[r[0]]["fit"] for r in rows if r[0] in by_i),
             "served_reached_same_requests": statistics.fmean(float(by_i[r[0]]["reached"]) for r in rows
                                                              if r[0] in by_i)}
    eq = {"rule": "final fits within %g, or both at the fit target %g" % (SERVE["match"], SERVE["stop_fit"]),
          "matched": len(matched), "of": len(rows)}
    if matched:
        eq["plain_solves_per_s_matched"] = len(matched) / sum(r[1] for r in matched)
        eq["served_over_plain"] = served["solves_per_s"] / eq["plain_solves_per_s_matched"]
    out.update({"plain_gpu_sequential": plain, "equal_fit": eq,
                "rule": {"stop_fit": SERVE["stop_fit"], "max_iters": SERVE["max_iters"],
                         "fit_every": SERVE["fit_every"], "sampling": SERVE["sampling"],
                         "step": SERVE["step"], "eta": SERVE["eta"], "B": SERVE["B"],
                         "max_ctas": SERVE["max_ctas"], "max_active": max_active,
                         "engine": ("persistent cluster of %d CTAs per request" % SERVE["cluster"]
                                    if SERVE["engine"] == "persistent" else
                                    "per-CTA tensor cores for R >= 16 (%s), CUDA cores below" % SERVE["engine_r16"]),
                         "grouped_launches": SERVE["grouping"],
                         "plain": "automatic engine, no CTA cap, one request at a time"}})
    return out


def config_block(w: dict, engine: str) -> dict:
    return {"workload": w["name"], "dims": list(w["dims"]), "R": w["R"], "B": w["B"],
            "x_dtype": w["x_dtype"], "sampling": w["sampling"], "step": w["step"], "engine": engine,
            "l2": "no flush: the mode-major tensor replicas (%.1f GB) are larger than L2" % (
                len(w["dims"]) * torch.tensor(w["dims"]).prod().item() * (2 if w["x_dtype"] == "bf16" else 4) / 1e9)}


def main() -> None:
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20000)
    ap.add_argument("--warmup", type=int, default=500)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD)
    ap.add_argument("--engine", default="auto", choices=["auto", "simt", "tensor", "cluster", "persistent", "fused"])
    ap.add_argument("--max-ctas", type=int, default=0, help="CTA cap of the gradient launch (0: none)")
    ap.add_argument("--sampling", default=None)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-autotune", action="store_true",
                    help="skip cpd_autotune (by default the applicable engines and CTA caps are timed first, "
                         "outside the timed region, and the fastest is used)")
    ap.add_argument("--no-gather-legs", action="store_true", help="skip the bulk gather and batched-form legs")
    ap.add_argument("--only-gather", action="store_true", help="run only the bulk gather leg (--steps launches per mode)")
    ap.add_argument("--only-fit", action="store_true", help="run only the stop-check pass (--steps passes)")
    ap.add_argument("--only-serving", action="store_true", help="run only the serving leg")
    ap.add_argument("--batch-g", type=int, default=15, help="decompositions in the batched-form leg")
    ap.add_argument("--batch-cs", type=int, default=8, help="cluster size of the batched-form leg")
    ap.add_argument("--batch-iters", type=int, default=1000)
    ap.add_argument("--serve-requests", type=int, default=SERVE["requests"])
    ap.add_argument("--serve-plain", type=int, default=SERVE["plain_sample"])
    ap.add_argument("--serve-active", type=int, default=64)
    ap.add_argument("--serve-engine", default=SERVE["engine"], choices=["classic", "persistent"])
    ap.add_argument("--serve-cluster", type=int, default=SERVE["cluster"])
    ap.add_argument("--serve-strided-fraction", type=float, default=SERVE["strided_fraction"],
                    help="requests whose replicas need more than this fraction of the budget run strided")
    args = ap.parse_args()
    SERVE["strided_fraction"] = args.serve_strided_fraction

    from paper_2103_04081_gb300 import inputs as IN
    w = dict(IN.WORKLOADS[args.workload])
    w["name"] = args.workload
    if args.sampling:
        w["sampling"] = args.sampling
    if args.impl == "reference":
        run_reference(args, w)
        return

    from paper_2103_04081_gb300 import cpd as C
    dist, rank, world, local = dist_setup()
    torch.cuda.set_device(local)
    dev = f"cuda:{local}"
    if args.only_serving:
        SERVE["engine"], SERVE["cluster"] = args.serve_engine, args.serve_cluster
        print(json.dumps({"serving": serve_bench(dev, args.serve_requests, args.serve_plain, args.serve_active)}),
              flush=True)
        return
    X, A0 = make_inputs(w, rank, dev)
    if args.only_fit:      # the stop-check pass alone (e.g. for a counter capture)
        kwf = cfg_kwargs(w, rank, "auto")
        with torch.cuda.stream(stream0 := torch.cuda.Stream()):
            decf = C.Decomposition(X, [a.to(dev) for a in A0], stream=stream0, **kwf)
        decf.sgd_iters(20, stream0)
        print(json.dumps({"fit_pass": fit_pass(C, decf, w, stream0, reps=args.steps)}), flush=True)
        decf.close()
        return
    if args.only_gather:   # the bulk gather leg alone (e.g. for a counter capture)
        peaks, _ = measured_peaks()
        print(json.dumps({"gather_per_mode": gather_per_mode(C, X, A0, w, dev, torch.cuda.Stream(),
                                                             peaks["hbm_gbs"], reps=args.steps)}), flush=True)
        return
    kw = cfg_kwargs(w, rank, args.engine)
    kw["max_ctas"] = args.max_ctas
    stream = torch.cuda.Stream()
    tuned = None
    if not args.no_autotune and args.engine == "auto" and args.max_ctas == 0:
        best, rate = C.cpd_autotune(C.make_config(**kw), X, [a.to(dev) for a in A0], iters=300, stream=stream)
        tuned = {"engine": {1: "simt", 2: "tensor", 3: "cluster", 4: "persistent", 5: "fused"}[best.engine], "max_ctas": best.max_ctas,
                 "tile_rows": best.tile_rows, "tile_fibers": best.tile_fibers, "tuning_iters_per_s": rate}
        kw["engine"], kw["max_ctas"] = tuned["engine"], tuned["max_ctas"]
        kw["tile_rows"], kw["tile_fibers"] = tuned["tile_rows"], tuned["tile_fibers"]
    with torch.cuda.stream(stream):
        dec = C.Decomposition(X, [a.to(dev) for a in A0], stream=stream, **kw)
    desc = dec.describe()
    engine = desc["engine"]
    launches_per_iter = (1 if engine == "fused" else 2) + (2 if w["sampling"] == "leverage" else 0)
    if engine == "persistent":   # one launch per call of cpd_sgd_iters (up to 2^20 iterations)
        launches_per_iter = 1.0 / args.steps

    # warm-up (W iterations), the graphs a K-iteration call replays captured
    # ahead (nothing runs), then exactly K timed iterations
    dec.sgd_iters(args.warmup, stream)
    C.cpd_prepare(dec.ctx, args.steps, stream)
    C.cpd_sync(dec.ctx, stream)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with Clocks(local) as clk:
        ev0.record(stream)
        dec.sgd_iters(args.steps, stream)
        ev1.record(stream)
        ev1.synchronize()
    ms = ev0.elapsed_time(ev1)
    C.cpd_sync(dec.ctx, stream)
    ms = max_over_ranks(dist, ms, dev)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = clk.summary()

    # per-kernel duration of the gradient kernel: CUDA events around each launch
    # on the launching stream, over a pass of the same iterations
    C.cpd_profile(dec.ctx, True)
    nprof = min(args.steps, 2000)
    dec.sgd_iters(nprof, stream)
    nlaunch, grad_ms, upd_ms = C.cpd_profile_read(dec.ctx, stream)
    C.cpd_profile(dec.ctx, False)
    fit, tol = dec.fit(stream)
    fit_leg = fit_pass(C, dec, w, stream)
    dec.close()

    iters_per_s = whole_job_rate(world, args.steps, ms)
    esize = {"bf16": 2, "f32": 4, "f64": 8}[w["x_dtype"]]
    In = sum(w["dims"]) / len(w["dims"])           # modes drawn uniformly
    gather_bytes = w["B"] * In * esize               # algorithmic HBM bytes per gradient launch
    peaks, src = measured_peaks()
    achieved = gather_bytes / (grad_ms / 1e3) / 1e9
    traffic = ncu_traffic(engine)

    # end to end through the C-ABI with host buffers: upload X and A0 from pinned
    # memory (cpd_init), K iterations, Tol, factors back to host
    e2e = None
    if rank == 0 or world > 1:
        Xh = X.cpu().pin_memory()
        A0h = [a.contiguous().pin_memory() for a in A0]
        del X
        torch.cuda.empty_cache()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        with torch.cuda.stream(stream):
            d2 = C.Decomposition(Xh, A0h, stream=stream, **kw)
        d2.sgd_iters(args.steps, stream)
        _, tol2 = d2.fit(stream)
        Ah = d2.factors("cpu", stream)
        t1 = time.perf_counter()
        d2.close()
        h2d = Xh.numel() * Xh.element_size() + sum(a.numel() * a.element_size() for a in A0h)
        d2h = sum(a.numel() * a.element_size() for a in Ah) + 8
        e2e = {"value": args.steps / (t1 - t0), "unit": "iters/s",
               "h2d_bytes_per_step": h2d / args.steps, "d2h_bytes_per_step": d2h / args.steps,
               "seconds": t1 - t0, "note": "cpd_init from pinned host X + K iterations + cpd_fit + "
                                           "cpd_get_factors to host, per iteration"}

    if rank != 0:
        return
    line = {
        "metric": METRIC, "value": iters_per_s, "unit": "iters/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "bf16" if engine in ("tensor", "cluster", "persistent", "fused") else ("f64" if w["x_dtype"] == "f64" else "f32"),
        "data": "synthetic", "config": config_block(w, engine),
        "gather_gbs_in_loop": gather_bytes * args.steps / (ms / 1e3) / 1e9,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                     "frac": achieved / peaks["hbm_gbs"], "traffic": traffic,
                     "kernel": {"tensor": "k_grad_tc", "cluster": "k_grad_tcc", "persistent": "k_pers",
                                "fused": "k_fused"}.get(engine, "k_grad_simt"),
                     "algorithmic_bytes_per_launch": gather_bytes, "mean_launch_ms": grad_ms,
                     "timed_launches": nlaunch, "peak_source": src + " (hbm_gbs, of " + src + ")",
                     "update_mean_ms": upd_ms},
        "clocks": clocks, "gpu_launches": int(round(launches_per_iter * args.steps)),
        "e2e": e2e, "final_tol": tol, "launch": desc, "fit_pass": fit_leg,
    }
    if tuned:
        line["autotuned"] = tuned
    if world == 1 and w["x_dtype"] == "bf16" and not args.no_gather_legs:
        try:
            Xg, A0g = make_inputs(w, 0, dev)
            line["gather_per_mode"] = gather_per_mode(C, Xg, A0g, w, dev, stream, peaks["hbm_gbs"])
            line["batched"] = batched_form(C, Xg, A0g, w, dev, stream, peaks["hbm_gbs"], G=args.batch_g,
                                           cs=args.batch_cs, iters=args.batch_iters)
            del Xg
            torch.cuda.empty_cache()
        except Exception as exc:  # reported, not hidden
            line["gather_per_mode_error"] = repr(exc)
    SERVE["engine"], SERVE["cluster"] = args.serve_engine, args.serve_cluster
    if not args.no_serving and world == 1:
        try:
            line["serving"] = serve_bench(dev, args.serve_requests, args.serve_plain, args.serve_active)
        except Exception as exc:  # reported, not hidden: the iteration numbers above stand
            line["serving"] = {"error": repr(exc)}
    if not args.no_cpu_baseline and world == 1:
        Xc, A0c = make_inputs(w, 0, dev)
        line["cpu_baseline"] = oracle_baseline(w, Xc, A0c, args.cpu_budget)
        del Xc
        torch.cuda.empty_cache()
        if w["name"] == DEFAULT_WORKLOAD:
            try:
                line["error_vs_oracle"] = error_vs_oracle(C, dev, stream, kw)
            except Exception as exc:  # reported, not hidden
                line["error_vs_oracle"] = {"error": repr(exc)}
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
