"""Sampling studies on the GPU path (Sec. 5): iterations to a target Tol and
the gradient variance along a run, for uniform (Alg. 2, BrasCPD / AdasCPD),
Euclidean and leverage sampling (Alg. 4 / Alg. 5).

    python -m paper_2103_04081_gb300.studies --data data3 --iters 20000

prints one JSON line per sampling distribution:
  * iterations and GPU seconds until Tol <= --tol (checked every --every
    iterations), the paper's stopping rule (Sec. 5.2, Tables 2-5);
  * E||G - E[G]||^2 of mode 0 at the checkpoints (Thm 10; the curves of
    Fig. 3), from cpd_grad_variance.
Data: the variance-study tensors (Data II / Data III), noiseless, R = 10,
|F_n| = 18 as in the paper's synthetic runs; random N(0,1) initial factors.
"""
from __future__ import annotations

import argparse
import json
import time

import torch

from . import cpd as C
from . import inputs as IN


def run(which: str, sampling: str, *, I: int, R: int, B: int, step: str, eta: float, alpha: float,
        tol: float, iters: int, every: int, seed: int, x_dtype: str, engine: str = "auto") -> dict:
    A = IN.variance_study_factors(which, I, R, seed, device="cuda")
    X = IN.cp_tensor(A, 0.0, seed, x_dtype)
    A0 = [a.cuda() for a in IN.init_factors((I, I, I), R, seed + 1,
                                             dtype=torch.float64 if x_dtype == "f64" else torch.float32)]
    dec = C.Decomposition(X, A0, dims=(I, I, I), R=R, B=B, x_dtype=x_dtype, sampling=sampling, step=step,
                          eta=eta, alpha=alpha, seed=seed, engine=engine)
    trace, reached, done, diverged = [], None, 0, False
    gpu_s = 0.0
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    desc = dec.describe()
    try:
        while done < iters:
            v, m = dec.grad_variance(0)
            f, t = dec.fit()
            trace.append({"iter": done, "tol": t, "var_mode0": v, "mean_norm2_mode0": m})
            if t <= tol:
                reached = done
                break
            k = min(every, iters - done)
            ev0.record()
            dec.sgd_iters(k)
            ev1.record()
            ev1.synchronize()
            gpu_s += ev0.elapsed_time(ev1) / 1e3
            done += k
        if reached is None:
            f, t = dec.fit()
            if t <= tol:
                reached = done
            trace.append({"iter": done, "tol": t})
    except C.CpdError as e:               # a step size too large for the data
        if e.status not in (C.ENONFINITE, C.EDEGENERATE):
            raise
        diverged = True
        trace.append({"iter": done, "tol": float("nan")})
    dec.close()
    return {"data": which, "sampling": sampling, "step": step, "eta": eta, "alpha": alpha, "I": I, "R": R,
            "B": B, "tol_target": tol, "iters_to_tol": reached, "iters_run": done, "diverged": diverged,
            "gpu_seconds": gpu_s, "final_tol": trace[-1]["tol"], "engine": desc["engine"], "trace": trace}


def main() -> None:
    ap = argparse.ArgumentParser()
    ap.add_argument("--data", default="data2", choices=["data2", "data3"])
    ap.add_argument("--I", type=int, default=300)
    ap.add_argument("--R", type=int, default=10)
    ap.add_argument("--B", type=int, default=18)
    ap.add_argument("--step", default="adagrad")
    ap.add_argument("--eta", type=float, default=0.1)
    ap.add_argument("--alpha", type=float, default=0.1)
    ap.add_argument("--tol", type=float, default=1e-5)
    ap.add_argument("--iters", type=int, default=20000)
    ap.add_argument("--every", type=int, default=100)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--x-dtype", default="f32")
    ap.add_argument("--samplings", default="uniform,euclidean,leverage")
    args = ap.parse_args()
    for s in args.samplings.split(","):
        t0 = time.time()
        out = run(args.data, s, I=args.I, R=args.R, B=args.B, step=args.step, eta=args.eta,
                  alpha=args.alpha, tol=args.tol, iters=args.iters, every=args.every, seed=args.seed,
                  x_dtype=args.x_dtype)
        out["wall_seconds"] = time.time() - t0
        print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
