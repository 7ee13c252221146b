"""Benchmark: time to a rank-k approximation on one GB300 (and the CPU oracle beside it).

Workload (noisy exponential decay): dense A 65536 x 16384 float32,
sigma_i = exp(-i/200) between Haar factors plus 1e-3 N(0,1) noise, target rank
k = 1000, sparse sign sketch of size r1 = 2000 with s = 8 non-zeros per row,
q = 2 power steps.  One step = one full Randomized SVD through the C ABI
(sketch apply, power iteration, re-orthonormalisation, Q^T A, core SVD,
U and V^T) in the mixed-precision mode; the sketch tables are built once.

Printed: one JSON line with the metric, the plain-FP64 GPU form's time and
residual at the same q (the accuracy target), the stage breakdown, the
roofline of the dominant kernel, an end-to-end number with host buffers, and
the CPU oracle timed on a bounded row sample.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "time to rank-k approx at fixed rel. residual vs plain FP64 GPU; HBM GB/s"

# DRAM bytes (read + write) per launch measured by ncu for the sketch-apply kernel, per
# element of A and per element of A~ at the capture's shape; scaled to the run's shape
# (traffic grows with m n and m r1).  None until a capture of the current kernel exists.
NCU_TRAFFIC = {
    # profiles/k_sketch_sched_8192x16384_r2000.md (the kernel with A's split written in the
    # same pass): 538.3 MB read + 555.1 MB written at m = 8192, n = 16384, r1 = 2000; A~'s
    # share taken as its algorithmic 65.5 MB, the rest per element of A
    "k_sketch_sched": {"per_a": (538.251264e6 + 555.143936e6 - 65.536e6) / (8192 * 16384),
                       "per_out": 65.536e6 / (8192 * 2000)},
}


def ncu_traffic(kernel, m, n, r1):
    t = NCU_TRAFFIC.get(kernel)
    if not t:
        return None
    return t["per_a"] * m * n + t["per_out"] * m * r1


def max_over_ranks(x, dist, device):
    """x on this rank -> the largest x over the ranks of the default process group."""
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def per_approximation_ms(ms_total, steps, world):
    """Whole-job time per rank-k approximation: each of `world` ranks runs `steps`
    of them within ms_total (the slowest rank's time)."""
    return ms_total / (steps * world)


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--m", type=int, default=65536)
    p.add_argument("--n", type=int, default=16384)
    p.add_argument("--r1", type=int, default=2000)
    p.add_argument("--k", type=int, default=1000)
    p.add_argument("--s", type=int, default=8)
    p.add_argument("--q", type=int, default=2)
    p.add_argument("--noise", type=float, default=1e-3)
    p.add_argument("--scaled-noise", action="store_true",
                   help="noise matrix scaled by 1/sqrt(n): E = noise * G / sqrt(n)")
    p.add_argument("--no-fp64", action="store_true", help="skip the plain FP64 GPU reference run")
    p.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--final-passes", type=int, default=3)
    p.add_argument("--power-passes", type=int, default=3)
    p.add_argument("--cpu-rows", type=int, default=2048)
    p.add_argument("--autotune", action="store_true",
                   help="rsvd: time each product's split-K candidates in the warm-up and "
                        "keep the fastest (spm_set_autotune)")
    p.add_argument("--sketch", default="sparse", choices=["sparse", "dense", "srht"],
                   help="sketch family of Lemma 3.2 (item 2, 1 or 3) for the rsvd workload")
    p.add_argument("--trials", type=int, default=5, help="polydecay: trials (the paper: 25)")
    p.add_argument("--poly-l", default="800,1200,1600", help="polydecay: sketch sizes l")
    p.add_argument("--q-sketched", type=int, default=15)
    p.add_argument("--no-poly-alg2", dest="poly_alg2", action="store_false",
                   help="polydecay: skip the Algorithm 2 vs generalized Nystrom comparison")
    p.add_argument("--q-classical", type=int, default=5)
    p.add_argument("--poly-target", type=float, default=0.1,
                   help="polydecay: relative spectral error the time is measured to")
    p.add_argument("--workload", default="rsvd", choices=["rsvd", "batched", "csr", "nystrom",
                                                          "polydecay"],
                   help="rsvd: the 65536 x 16384 RandSVD (default); batched: 512 uneven "
                        "problems in one graph-captured spm_rsvd_batched call; csr: the "
                        "10^6 x 2*10^5 sparse matrix with a planted rank-200 term; nystrom: the "
                        "40000-point Gaussian kernel")
    p.add_argument("--nys-n", type=int, default=40000, help="nystrom: number of points")
    p.add_argument("--batch", type=int, default=512)
    p.add_argument("--nstreams", type=int, default=16)
    p.add_argument("--batch-precision", default="mixed", choices=["mixed", "fp32"])
    p.add_argument("--batch-auto", action="store_true",
                   help="batched: spm_rsvd_batched_auto (selector network + residual judge) "
                        "at --target instead of the fixed (q, r1)")
    p.add_argument("--target", type=float, default=1.05,
                   help="batched --batch-auto: residual ratio target")
    return p.parse_args()


def workload_name(a):
    sk = {"sparse": f"sparse sign sketch r1={a.r1} s={a.s}", "dense": f"dense sign sketch r1={a.r1}",
          "srht": f"SRHT sketch r1={a.r1}"}[getattr(a, "sketch", "sparse")]
    noise = (f"{a.noise:g}*N(0,1)/sqrt(n)" if getattr(a, "scaled_noise", False)
             else f"{a.noise:g}*N(0,1)")
    return (f"dense {a.m}x{a.n} f32, sigma_i=exp(-i/200) + {noise} noise, "
            f"k={a.k}, {sk}, q={a.q}, RandSVD")


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self):
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100", "-i", os.environ.get("LOCAL_RANK", "0"), "-f", self.path],
                stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": []}
        if self.proc is None:
            return out
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        try:
            for line in open(self.path):
                f = [x.strip() for x in line.split(",")]
                if len(f) < 9:
                    continue
                try:
                    sm.append(float(f[1]))
                    mx.append(float(f[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, f[5:9]):
                    if v.lower() == "active":
                        reasons.add(nm)
            os.unlink(self.path)
        except Exception:
            pass
        if sm:
            busy = [v for v in sm if v > 0.5 * max(sm)] or sm
            out = {"sm_mhz": statistics.median(busy), "sm_max_mhz": max(mx),
                   "reasons": sorted(reasons), "samples": len(sm)}
        return out


# ------------------------------------------------------------------ CPU oracle leg
def cpu_oracle_ms(A_rows, a, seed_s=42, seed_o=43):
    """Oracle Randomized SVD on a row sample; returns the time in ms."""
    from oracle import algorithms as alg
    from oracle import sketch as osk
    n = A_rows.shape[1]
    So = osk.Sketch(n, a.r1, a.s, seed_s)
    Om = osk.gaussian(a.r1, a.k, seed_o)
    t0 = time.perf_counter()
    alg.rsvd(A_rows, So, Om, a.q, a.k)
    return (time.perf_counter() - t0) * 1e3


def cpu_oracle_fit(A_rows, a):
    """The oracle at the full m from two row samples (the first half of A_rows and
    all of it): its time is linear in m, t(m) = t0 + slope m, the constant part
    being the m-independent work (the SVD of the k x n matrix B, the r2 x r2
    Choleskies), so only the slope is extrapolated.  Returns (estimate ms, time of
    the small sample, time of the large one, rows of the small one)."""
    rows = A_rows.shape[0] // 2
    t1 = cpu_oracle_ms(A_rows[:rows], a)
    t2 = cpu_oracle_ms(A_rows, a)
    slope = max(t2 - t1, 0.0) / rows
    return t2 + slope * (a.m - 2 * rows), t1, t2, rows


def reference_main(a):
    """--impl reference: the CPU oracle, as it stands, on bounded row samples."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    rows = max(a.cpu_rows, a.k)
    # row samples of the same workload, generated on the host
    from paper_2605_09755_gb300 import workloads as wl
    noise = a.noise / (a.n ** 0.5) if a.scaled_noise else a.noise
    A, _ = wl.noisy_exp_numpy(2 * rows, a.n, seed=1002, noise=noise)
    for _ in range(a.warmup):
        cpu_oracle_ms(A[:rows], a)
    fits = [cpu_oracle_fit(A, a) for _ in range(a.steps)]
    v = statistics.mean(f[0] for f in fits)
    t1 = statistics.mean(f[1] for f in fits)
    t2 = statistics.mean(f[2] for f in fits)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "ms",
            "n_gpus": a.gpus, "steps": a.steps, "warmup": a.warmup, "ms_per_step": v,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": workload_name(a)},
            "cpu_baseline": {"value": v, "unit": "ms", "cores": os.cpu_count(), "kind": "oracle",
                             "sample": f"oracle RandSVD on {rows} and {2 * rows} of {a.m} rows: "
                                       f"{t1:.0f} and {t2:.0f} ms; the difference extrapolated "
                                       f"linearly in m (the SVD of B and other m-independent "
                                       f"work counted once)"},
            "e2e": {"value": v, "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ GPU leg
def residual(A, U, sg, Vt, chunk=4096):
    import torch
    tot = 0.0
    Vs = (Vt.float() * 1.0)
    Us = U.float() * sg.float()
    for i in range(0, A.shape[0], chunk):
        R = A[i:i + chunk] - Us[i:i + chunk] @ Vs
        tot += float((R.double() ** 2).sum())
    return tot ** 0.5


def batched_auto_main(a):
    """The same 512 problems through spm_rsvd_batched_auto at a residual target
    (default 1.05 x the Eckart-Young optimum): the selector network picks (q, r1)
    per problem from its q = 0 probe, the batch runs, and the residual judge adds
    power steps (or an FP32 re-run) where the estimate has not settled.  One step =
    one spm_rsvd_batched_auto call (eager: it reads the predictions and the judge's
    estimates on the host).  Reported: time, the share of problems within the
    target, the ratio distribution, against the fixed (q = 2, r1 = 2k) path and the
    network's picks without the judge."""
    import numpy as np
    import torch
    from paper_2605_09755_gb300 import _build, spm
    from paper_2605_09755_gb300 import selector as sel
    from paper_2605_09755_gb300 import workloads as wl
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    _build.build()
    lib = spm.lib()
    params = sel.load_params()
    specs = wl.batch_specs(a.batch)
    probs, opts = [], []
    for sp in specs:
        A, sig = sel.make_matrix(sp)
        probs.append(dict(A=A, k=sp["k"], seed=42))
        opts.append(float(np.sqrt(np.sum(np.sort(np.asarray(sig))[::-1][sp["k"]:] ** 2))))
    torch.cuda.synchronize()
    prec = {"mixed": spm.PREC_MIXED, "fp32": spm.PREC_FP32}[a.batch_precision]

    def ratios(batch):
        out = []
        for p, opt, (U, sg, Vt) in zip(probs, opts, batch.outputs):
            R = p["A"] - (U * sg) @ Vt
            out.append(float(torch.linalg.norm(R.double())) / opt if opt > 0 else 1.0)
        return np.array(out)

    # problems whose optimal residual is at least 1.4% of |A|_F: there the judge's
    # estimate resolves the target's margin; below it the estimate is too coarse,
    # and the optimum itself approaches the working precision's floor
    fro = [float(torch.linalg.norm(p["A"].double())) for p in probs]
    judgeable = np.array([o >= 0.014 * f for o, f in zip(opts, fro)])

    def stats(r):
        out = {"share_within_target": float(np.mean(r <= a.target)), "median": float(np.median(r)),
               "p90": float(np.quantile(r, 0.9)), "max": float(np.max(r))}
        if judgeable.any():
            out["share_within_target_opt_ge_1.4pct"] = float(np.mean(r[judgeable] <= a.target))
            out["median_opt_ge_1.4pct"] = float(np.median(r[judgeable]))
        if (~judgeable).any():
            out["median_opt_lt_1.4pct"] = float(np.median(r[~judgeable]))
        return out

    batch = spm.Batch(probs, precision=prec, nstreams=a.nstreams)
    for _ in range(a.warmup):
        picks = batch.run_auto(a.target, params)
    torch.cuda.synchronize()
    c0 = lib.spm_launch_count()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler()
    clocks.start()
    torch.cuda.synchronize()
    e0.record()
    for _ in range(a.steps):
        picks = batch.run_auto(a.target, params)
    e1.record()
    torch.cuda.synchronize()
    clk = clocks.stop()
    launches = int(lib.spm_launch_count() - c0)
    batch.check_status()
    ms = e0.elapsed_time(e1) / a.steps
    judged = ratios(batch)
    kept = batch.item_params()
    # the network's picks alone (no judge), and the fixed path, for comparison
    pick_probs = [dict(A=p["A"], k=p["k"], seed=42, q=q, r1=min(c * p["k"], p["A"].shape[1]),
                       s=min(8, min(c * p["k"], p["A"].shape[1]))) for p, (q, c) in zip(probs, picks)]
    pb = spm.Batch(pick_probs, precision=prec, nstreams=a.nstreams)
    pb.run()
    torch.cuda.synchronize()
    e0.record()
    pb.run()
    e1.record()
    torch.cuda.synchronize()
    pick_ms = e0.elapsed_time(e1)
    picked = ratios(pb)
    del pb
    fixed_probs = [dict(A=p["A"], k=p["k"], seed=42, q=2, r1=min(2 * p["k"], p["A"].shape[1]),
                        s=min(8, min(2 * p["k"], p["A"].shape[1]))) for p in probs]
    fb = spm.Batch(fixed_probs, precision=prec, nstreams=a.nstreams)
    fb.run()
    torch.cuda.synchronize()
    e0.record()
    fb.run()
    e1.record()
    torch.cuda.synchronize()
    fixed_ms = e0.elapsed_time(e1)
    fixed = ratios(fb)
    del fb
    a_bytes = sum(p["A"].numel() * 4 for p in probs)
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    ach = 2.0 * a_bytes / (pick_ms * 1e-3) / 1e9
    line = {
        "metric": f"time to rank-k approximations within {a.target:g} x optimal (batched, "
                  f"selector + residual judge)", "value": ms, "unit": "ms", "n_gpus": 1,
        "steps": a.steps, "warmup": a.warmup, "ms_per_step": ms, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "bf16x3+f32" if a.batch_precision == "mixed" else "f32",
        "data": "synthetic (seeded)",
        "config": {"workload": f"{len(probs)} uneven dense problems (m in [512, 8192], n in "
                               f"[256, 4096], k in [16, 256], decay i^-alpha or exp(-i/tau)); "
                               f"spm_rsvd_batched_auto at target {a.target:g}",
                   "precision": a.batch_precision, "nstreams": a.nstreams},
        "accuracy": {"judged": stats(judged), "network_pick_only": stats(picked),
                     "fixed_q2_r1_2k": stats(fixed)},
        "problems_opt_ge_1.4pct_of_fro": int(judgeable.sum()),
        "q_raised_by_judge": int(sum(1 for (qk, _, _), (q, _) in zip(kept, picks) if qk > q)),
        "r1_raised_by_judge": int(sum(1 for (_, rk, _), (q, c), p in zip(kept, picks, probs)
                                      if rk > min(c * p["k"], p["A"].shape[1]))),
        "network_pick_only_ms": pick_ms, "fixed_ms": fixed_ms,
        "roofline": {"kernel": "whole batch at the network's picks (two passes over every A: "
                               "A S and Q^T A)", "bound": "hbm", "achieved": ach, "peak": hbm_peak,
                     "unit": "GB/s", "frac": ach / hbm_peak, "traffic": None,
                     "peak_source": "MEASURED_PEAKS.json hbm_gbs, of measured"},
        "e2e": None, "cpu_baseline": None, "gpu_launches": launches, "clocks": clk,
    }
    print(json.dumps(line), flush=True)


def batched_main(a):
    """512 uneven dense problems (m in [512, 8192], n in [256, 4096] log-uniform,
    k in [16, 256], sigma ~ i^-alpha or exp(-i/tau)); r1 = 2k, s = 8, q = 2.
    One step = one replay of the CUDA graph captured around one
    spm_rsvd_batched call over all problems."""
    import numpy as np
    import torch
    from paper_2605_09755_gb300 import _build, spm
    from paper_2605_09755_gb300 import selector as sel
    from paper_2605_09755_gb300 import workloads as wl
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    _build.build()
    lib = spm.lib()
    specs = wl.batch_specs(a.batch)
    probs, sigmas = [], []
    for sp in specs:
        A, sig = sel.make_matrix(sp)
        r1 = min(2 * sp["k"], sp["n"])
        probs.append(dict(A=A, k=sp["k"], r1=r1, q=a.q, s=min(a.s, r1), seed=42))
        sigmas.append(sig)
    torch.cuda.synchronize()
    prec = {"mixed": spm.PREC_MIXED, "fp32": spm.PREC_FP32}[a.batch_precision]
    batch = spm.Batch(probs, precision=prec, nstreams=a.nstreams)
    for _ in range(a.warmup):
        batch.run()
    torch.cuda.synchronize()
    batch.check_status()
    c0 = lib.spm_launch_count()
    batch.run()
    torch.cuda.synchronize()
    launches = int(lib.spm_launch_count() - c0)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    batch.run()
    e1.record()
    torch.cuda.synchronize()
    eager_ms = e0.elapsed_time(e1)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        batch.run()
    graph.replay()
    torch.cuda.synchronize()
    clocks = ClockSampler()
    clocks.start()
    torch.cuda.synchronize()
    e0.record()
    for _ in range(a.steps):
        graph.replay()
    e1.record()
    torch.cuda.synchronize()
    clk = clocks.stop()
    batch.check_status()
    ms = e0.elapsed_time(e1) / a.steps
    # accuracy: residual / Eckart-Young optimum per problem
    ratios = []
    for p, sig, (U, sg, Vt) in zip(probs, sigmas, batch.outputs):
        opt = float(np.sqrt(np.sum(np.sort(sig)[::-1][p["k"]:] ** 2)))
        R = p["A"] - (U * sg) @ Vt
        ratios.append(float(torch.linalg.norm(R.double())) / opt if opt > 0 else 1.0)
    a_bytes = sum(p["A"].numel() * 4 for p in probs)
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    ach = 2.0 * a_bytes / (ms * 1e-3) / 1e9
    roof = {"kernel": "whole batch (two passes over every A: A S and Q^T A)", "bound": "hbm",
            "achieved": ach, "peak": hbm_peak, "unit": "GB/s", "frac": ach / hbm_peak,
            "traffic": None, "peak_source": "MEASURED_PEAKS.json hbm_gbs, of measured"}
    # end to end: host copies of every A into the captured call's input buffers,
    # one replay of the captured batched call, every U, sigma, V^T copied out
    hostA = [p["A"].cpu().pin_memory() for p in probs]
    hostO = [tuple(t.cpu().pin_memory() for t in o) for o in batch.outputs]
    e2e_ms = []
    for _ in range(2):
        torch.cuda.synchronize()
        e0.record()
        for hA, p in zip(hostA, probs):
            p["A"].copy_(hA, non_blocking=True)
        graph.replay()
        for ho, o in zip(hostO, batch.outputs):
            for h, d in zip(ho, o):
                h.copy_(d, non_blocking=True)
        e1.record()
        torch.cuda.synchronize()
        e2e_ms.append(e0.elapsed_time(e1))
    batch.check_status()
    e2e = {"value": e2e_ms[-1], "unit": "ms", "h2d_bytes_per_step": int(a_bytes),
           "d2h_bytes_per_step": int(sum(sum(t.numel() * 4 for t in o) for o in batch.outputs))}
    cpu = None
    if not a.no_cpu:
        from oracle import algorithms as alg
        from oracle import sketch as osk
        rng = np.random.default_rng(3)
        sample = sorted(rng.choice(len(probs), size=min(12, len(probs)), replace=False).tolist())
        work = [float(p["A"].shape[0]) * p["A"].shape[1] * p["k"] for p in probs]
        t0 = time.perf_counter()
        for i in sample:
            p = probs[i]
            A = p["A"].double().cpu().numpy()
            n = A.shape[1]
            alg.rsvd(A, osk.Sketch(n, p["r1"], p["s"], 42), osk.gaussian(p["r1"], p["k"], 43), p["q"],
                     p["k"])
        t = (time.perf_counter() - t0) * 1e3
        scale = sum(work) / sum(work[i] for i in sample)
        cpu = {"value": t * scale, "unit": "ms", "cores": os.cpu_count(), "kind": "oracle",
               "sample": f"oracle RandSVD of {len(sample)} of the {len(probs)} problems, time "
                         f"scaled by total m n k ({scale:.1f}x)"}
    line = {
        "metric": "time to rank-k approx of a batch of 512 uneven dense matrices", "value": ms,
        "unit": "ms", "n_gpus": 1, "steps": a.steps, "warmup": a.warmup, "ms_per_step": ms,
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
        "dtype": "bf16x3+f32" if prec == spm.PREC_MIXED else "f32", "data": "synthetic (seeded)",
        "config": {"workload": f"batched RandSVD: {len(probs)} matrices m in [512, 8192], n in "
                               f"[256, 4096] log-uniform, k in [16, 256], r1 = 2k, s = {a.s}, "
                               f"q = {a.q}, one CUDA graph replay per step",
                   "precision": a.batch_precision, "nstreams": a.nstreams,
                   "l2": f"inputs ({a_bytes / 1e9:.1f} GB) larger than L2; no flush"},
        "matrices_per_s": len(probs) / (ms * 1e-3), "eager_ms": eager_ms,
        "accuracy": {"median_ratio_vs_optimal": float(np.median(ratios)),
                     "max_ratio_vs_optimal": float(np.max(ratios))},
        "roofline": roof, "e2e": e2e, "cpu_baseline": cpu, "gpu_launches": launches * a.steps,
        "clocks": clk,
    }
    print(json.dumps(line), flush=True)


def csr_main(a):
    """The sparse workload: A = A_csr + U diag(100 i^-1/2) V^T, 10^6 x 2*10^5 with 20
    N(0, 1) non-zeros per row, planted rank 200 kept as factors; r1 = 400, k = 200,
    s = 8, q = 2, mixed precision through spm_rsvd_csr.  One step = one call."""
    import numpy as np
    import torch
    from paper_2605_09755_gb300 import _build, spm
    from paper_2605_09755_gb300 import workloads as wl
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    _build.build()
    lib = spm.lib()
    m, n, nnz_row, p, r1, k = 1_000_000, 200_000, 20, 200, 400, 200
    indptr, indices, values, U, sig, V = wl.sparse_planted(m, n, nnz_row, p, seed=1003)
    f32 = lambda x: torch.tensor(x, dtype=torch.float32, device="cuda")
    A = spm.CsrMatrix(torch.tensor(indptr, device="cuda"),
                      torch.tensor(indices, dtype=torch.int32, device="cuda"), f32(values), n,
                      U=f32(U), sig=f32(sig), V=f32(V))
    del indices, values, U, V
    S = spm.Sketch(n, r1, a.s, 42)
    step = lambda timing=False: spm.rsvd_csr(S, A, k, a.q, k, precision=spm.PREC_MIXED,
                                            timing=timing)
    for _ in range(a.warmup):
        step()
    torch.cuda.synchronize()
    c0 = lib.spm_launch_count()
    _, _, _, inf = step(timing=True)
    torch.cuda.synchronize()
    launches = int(lib.spm_launch_count() - c0)
    # the CSR sketch kernel alone (the sparse part, no low-rank term), for its
    # roofline: rowptr, colind and values read, A~ written (the sketch tables sit in L2)
    Asp = spm.CsrMatrix(A.rowptr, A.colind, A.vals, n)
    At = torch.empty(m, r1, device="cuda")
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    for _ in range(3):
        spm.sketch_apply_csr(S, Asp, out=At)
    e0.record()
    for _ in range(a.steps):
        spm.sketch_apply_csr(S, Asp, out=At)
    e1.record()
    torch.cuda.synchronize()
    sk_ms = e0.elapsed_time(e1) / a.steps
    sk_bytes = (m + 1) * 8 + m * nnz_row * 8 + m * r1 * 4
    del At
    clocks = ClockSampler()
    clocks.start()
    torch.cuda.synchronize()
    e0.record()
    for _ in range(a.steps):
        step()
    e1.record()
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1) / a.steps
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    ach = sk_bytes / (sk_ms * 1e-3) / 1e9
    line = {
        "metric": "time to rank-k approx of a sparse CSR matrix with a planted low-rank term",
        "value": ms, "unit": "ms", "n_gpus": 1, "steps": a.steps, "warmup": a.warmup,
        "ms_per_step": ms, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
        "dtype": "bf16x3+f32", "data": "synthetic (seeded)",
        "config": {"workload": f"CSR {m}x{n}, {nnz_row} N(0,1) non-zeros per row, planted "
                               f"U diag(100 i^-1/2) V^T of rank {p} as factors, r1 = {r1}, "
                               f"k = {k}, s = {a.s}, q = {a.q}, RandSVD",
                   "precision": "mixed", "l2": "A~ (1.6 GB) larger than L2; no flush"},
        "stage_ms": inf["stage_ms"],
        "roofline": {"kernel": "k_csr_sketch (A_csr S)", "bound": "hbm",
                     "achieved": ach, "peak": hbm_peak, "unit": "GB/s", "frac": ach / hbm_peak,
                     "traffic": None, "peak_source": "MEASURED_PEAKS.json hbm_gbs, of measured"},
        "e2e": None,
        "cpu_baseline": {"value": None, "unit": "ms", "cores": os.cpu_count(), "kind": "oracle",
                         "sample": "not run: the oracle's RandSVD needs the dense 10^6 x 2*10^5 "
                                   "matrix (1.6 TB in FP64)"},
        "gpu_launches": launches * a.steps, "clocks": clk,
    }
    print(json.dumps(line), flush=True)


def formed_kernel(a, spm, S, K64, k, q, e0, e1, rel_err):
    """The Nystrom approximation of the same kernel from a formed FP32 K in HBM
    (spm_nystrom_eig): its time, stage times and error, and the FP64 error."""
    import torch
    K = K64.float()
    formed = lambda: spm.nystrom_eig(S, K, k, q, precision=spm.PREC_MIXED)
    formed()
    torch.cuda.synchronize()
    e0.record()
    for _ in range(a.steps):
        formed()
    e1.record()
    torch.cuda.synchronize()
    formed_ms = e0.elapsed_time(e1) / a.steps
    Uk, lk, inf_k = spm.nystrom_eig(S, K, k, q, precision=spm.PREC_MIXED, timing=2)
    e_formed = rel_err(Uk, lk, K64)
    del K, Uk, lk
    U64, lam64, _ = spm.nystrom_eig(S, K64, k, q, precision=spm.PREC_FP64)
    e_fp64 = rel_err(U64, lam64, K64)
    return formed_ms, inf_k, e_formed, e_fp64


def nystrom_main(a):
    """Nystrom (Algorithm 3, factored form) of the Gaussian kernel over 40000 points of
    an 8-component mixture in R^16 (means N(0, 3^2 I), unit covariance), h = the lower
    median of the pairwise distances; r1 = 1000, k = 500, s = 8, q = 1, mixed precision.
    One step = one spm_nystrom_gauss call: K is generated inside the product K S and
    never stored.  The same approximation from a formed FP32 K (spm_nystrom_eig, the
    6.4 GB matrix read from HBM) is timed beside it."""
    import numpy as np
    import torch
    from paper_2605_09755_gb300 import _build, spm
    from paper_2605_09755_gb300 import workloads as wl
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    _build.build()
    lib = spm.lib()
    n, d, r1, k, q = a.nys_n, 16, 1000, 500, 1
    X = wl.gmm_points(n, d, 8, seed=1004)
    Xd = torch.tensor(X, dtype=torch.float64, device="cuda")
    sq = (Xd * Xd).sum(1)
    D2 = (sq[:, None] + sq[None, :] - 2.0 * (Xd @ Xd.T)).clamp_min_(0.0)
    # lower median over the pairs i < j: every pair appears twice off the diagonal
    npairs = n * (n - 1) // 2
    D2.fill_diagonal_(float("inf"))
    kth = 2 * ((npairs - 1) // 2) + 1
    h2 = float(torch.kthvalue(D2.reshape(-1), kth).values)
    h = h2 ** 0.5
    D2.fill_diagonal_(0.0)
    K64 = torch.exp(D2 / (-2.0 * h2))
    del D2
    K64 = 0.5 * (K64 + K64.T)
    Xf = Xd.float()
    S = spm.Sketch(n, r1, a.s, 42)
    step = lambda timing=False: spm.nystrom_gauss(S, Xf, h, k, q, precision=spm.PREC_MIXED,
                                                  timing=timing)
    for _ in range(a.warmup):
        step()
    torch.cuda.synchronize()
    c0 = lib.spm_launch_count()
    U, lam, inf = step(timing=2)
    torch.cuda.synchronize()
    launches = int(lib.spm_launch_count() - c0)
    clocks = ClockSampler()
    clocks.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(a.steps):
        step()
    e1.record()
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1) / a.steps
    U, lam, _ = step()
    # the fused product alone (its two table/point preparation launches included)
    spm.gauss_sketch(S, Xf, h)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(a.steps):
        spm.gauss_sketch(S, Xf, h)
    e1.record()
    torch.cuda.synchronize()
    ks_ms = e0.elapsed_time(e1) / a.steps

    # end to end through the public call with host buffers: X in, U and lam out
    Xh = Xf.cpu().pin_memory()
    Uh = torch.empty(n, k, dtype=torch.float32).pin_memory()
    lh = torch.empty(k, dtype=torch.float32).pin_memory()

    def e2e_step():
        Xg = Xh.to("cuda", non_blocking=True)
        Ug, lg, _ = spm.nystrom_gauss(S, Xg, h, k, q, precision=spm.PREC_MIXED)
        Uh.copy_(Ug, non_blocking=True)
        lh.copy_(lg, non_blocking=True)

    e2e_step()
    torch.cuda.synchronize()
    e0.record()
    for _ in range(a.steps):
        e2e_step()
    e1.record()
    torch.cuda.synchronize()
    e2e_ms = e0.elapsed_time(e1) / a.steps

    def rel_err(U, lam, Kref):
        U64, l64 = U.double(), lam.double()
        err2, ref2 = 0.0, 0.0
        for i0 in range(0, n, 4096):       # ||K - U diag(lam) U^T||_F in row blocks
            blk = Kref[i0:i0 + 4096] - (U64[i0:i0 + 4096] * l64) @ U64.T
            err2 += float((blk * blk).sum())
            ref2 += float((Kref[i0:i0 + 4096] ** 2).sum())
        return (err2 / ref2) ** 0.5

    e_fused = rel_err(U, lam, K64)
    formed_ms, inf_k, e_formed, e_fp64 = None, {"stage_ms": None}, None, None
    if a.no_fp64:
        del K64
    else:
        formed_ms, inf_k, e_formed, e_fp64 = formed_kernel(a, spm, S, K64, k, q, e0, e1, rel_err)
        del K64
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    # ALU roofline of the fused product: per pair (i, j), d subtractions and d
    # multiply-adds for the squared distance, one multiply for the exponent and s
    # multiplies by the signed 1/sqrt(s): 2 d + 1 + s FP32 lane operations (the
    # exponential runs on the special-function unit, the additions into the
    # accumulators in shared memory).  Peak: 128 FP32 lanes per SM per clock.
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    mhz = clk.get("sm_max_mhz") or 2070.0
    ops = float(n) * n * (2 * d + 1 + a.s)
    alu_peak = sms * 128 * mhz * 1e6 / 1e9
    alu_ach = ops / (ks_ms * 1e-3) / 1e9
    ks_bytes = n * d * 4 + n * r1 * 4 + 2 * n * ((a.s + 3) // 4 * 4) * 4
    cpu = None
    if not a.no_cpu:
        from oracle import algorithms as alg
        from oracle import sketch as osk
        ns = 3000
        So = osk.Sketch(ns, r1, a.s, 42)
        t0 = time.perf_counter()
        Ks = alg.gaussian_kernel(X[:ns], h)
        osk.apply_right(Ks, So)
        t_ks = (time.perf_counter() - t0) * 1e3
        t0 = time.perf_counter()
        alg.nystrom_gauss(X[:ns], h, So, osk.gaussian(r1, k, 43), q)
        t = (time.perf_counter() - t0) * 1e3
        # forming K and K S grow with n^2; everything after them (C~ Y, the finish) with n
        est = t_ks * (n / ns) ** 2 + max(t - t_ks, 0.0) * (n / ns)
        cpu = {"value": est, "unit": "ms", "cores": os.cpu_count(), "kind": "oracle",
               "sample": f"oracle factored Nystrom of the Gaussian kernel of the first {ns} of "
                         f"the {n} points (same r1, k, q, h): {t:.0f} ms, of which forming K and "
                         f"K S {t_ks:.0f} ms; those scaled by (n / {ns})^2, the rest by n / {ns}"}
    line = {
        "metric": "time to a rank-k Nystrom approximation of a PSD kernel matrix", "value": ms,
        "unit": "ms", "n_gpus": 1, "steps": a.steps, "warmup": a.warmup, "ms_per_step": ms,
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32 (kernel values and K S) + bf16x3 (C~ Y) + f64 (Cholesky)",
        "data": "synthetic (seeded)",
        "config": {"workload": f"Nystrom (factored, shifted Cholesky) of the Gaussian kernel over "
                               f"{n} points of an 8-component mixture in R^{d}, h = lower median "
                               f"distance, K generated inside K S (never stored), r1 = {r1}, "
                               f"k = {k}, s = {a.s}, q = {q}",
                   "precision": "mixed", "l2": "no flush: the fused product reads 2.6 MB of points "
                                                "and writes C~ (160 MB, larger than L2)"},
        "stage_ms": inf["stage_ms"], "gauss_sketch_ms": ks_ms,
        "formed_kernel": {"ms": formed_ms, "stage_ms": inf_k["stage_ms"],
                          "note": "same approximation from a formed FP32 K (6.4 GB) in HBM"},
        "accuracy": {"rel_fro_err_fused_mixed": e_fused, "rel_fro_err_formed_mixed": e_formed,
                     "rel_fro_err_fp64": e_fp64,
                     "ratio": e_fused / e_fp64 if e_fp64 else None, "h": h,
                     "lam_top": float(lam[0]), "lam_k": float(lam[-1])},
        "roofline": {"kernel": "k_gauss_sketch_f32 (K S, K generated)", "bound": "alu",
                     "achieved": alu_ach, "peak": alu_peak, "unit": "Gop/s",
                     "frac": alu_ach / alu_peak, "traffic": None,
                     "ops_per_pair": 2 * d + 1 + a.s,
                     "peak_source": f"{sms} SMs x 128 FP32 lanes x {mhz:.0f} MHz (derived)",
                     "hbm": {"algorithmic_bytes": ks_bytes,
                             "achieved_gbs": ks_bytes / (ks_ms * 1e-3) / 1e9, "peak": hbm_peak,
                             "frac": ks_bytes / (ks_ms * 1e-3) / 1e9 / hbm_peak}},
        "e2e": {"value": e2e_ms, "unit": "ms", "h2d_bytes_per_step": n * d * 4,
                "d2h_bytes_per_step": n * k * 4 + k * 4},
        "cpu_baseline": cpu, "gpu_launches": launches * a.steps, "clocks": clk,
    }
    print(json.dumps(line), flush=True)


def protocol_summary(records, target):
    """Section 4's curves from individual runs.

    records: dicts with method ("sketched", "classical", "alg2_sketched" or
    "alg2_generalized_nystrom"), l (sketch size; n for the classical form), q, ms
    and err (relative spectral error).  Returns
    (curves, best): curves[method:l] = [(q, mean ms, mean err, runs)] by q, and
    best[method] = the smallest mean time whose mean error is <= target, with its
    (l, q), or None when no iterate reaches the target."""
    groups = {}
    for r in records:
        groups.setdefault((r["method"], r["l"], r["q"]), []).append(r)
    curves = {}
    for (method, l, q), rs in sorted(groups.items()):
        curves.setdefault(f"{method}:{l}", []).append(
            (q, statistics.mean(x["ms"] for x in rs), statistics.mean(x["err"] for x in rs), len(rs)))
    best = {}
    for key, pts in curves.items():
        method, l = key.split(":")
        for q, ms, err, _ in pts:
            if err <= target and (best.get(method) is None or ms < best[method]["ms"]):
                best[method] = {"ms": ms, "err": err, "l": int(l), "q": q}
        best.setdefault(method, None)
    return curves, best


def polydecay_main(a):
    """Section 4's protocol on its synthetic polydecay matrix (30000 x 15000,
    sigma_i = 30000 / i between Haar factors), FP32 A, mixed precision, k = 40:
    the Sketch-Powered RandSVD with a CountSketch S (s = 1) of l columns,
    l in {800, 1200, 1600}, q = 0..15, against the classical RandSVD (S = I),
    q = 0..5, each iterate computed from scratch and timed alone (CUDA events),
    error = ||A - U S V^T||_2 / sigma_{k+1} - 1 (the spectral norm by block power
    iteration on the residual), averaged over the trials (sketch seed 42 + t,
    Omega seed 43 + t).  A sketch is built, and its gather plan made by one
    untimed call, before its iterates are timed.  With Algorithm 2 (Appendix D):
    S1 a CountSketch of l columns against S1 = I, S2 a CountSketch of the rows
    to l in both, error ||A - Y X||_2 / sigma_{k+1} - 1."""
    import torch
    from paper_2605_09755_gb300 import _build, spm
    from paper_2605_09755_gb300 import workloads as wl
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    torch.backends.cuda.matmul.allow_tf32 = False
    _build.build()
    lib = spm.lib()
    m, n, k = 30000, 15000, 40
    ls = [int(x) for x in a.poly_l.split(",")]
    A, sigma = wl.polydecay_torch(m, n, seed=1006)
    torch.cuda.synchronize()
    sig_k1 = float(sigma[k])
    U = torch.empty(m, k, device="cuda")
    sg = torch.empty(k, device="cuda")
    Vt = torch.empty(k, n, device="cuda")
    g = torch.Generator(device="cuda")

    def spectral_err(L=None, R=None):
        # block power iteration on A - L R (block 8, 40 steps); L R = U diag(sg) Vt
        # by default
        if L is None:
            L, R = U * sg, Vt
        g.manual_seed(0)
        X, _ = torch.linalg.qr(torch.randn(n, 8, device="cuda", generator=g))
        for _ in range(40):
            Y = A @ X - L @ (R @ X)
            X, _ = torch.linalg.qr(A.T @ Y - R.T @ (L.T @ Y))
        Y = A @ X - L @ (R @ X)
        return float(torch.linalg.svdvals(Y)[0]) / sig_k1 - 1.0

    def run(S, q, oseed):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        spm.rsvd(S, A, k, q, k, omega_seed=oseed, out=(U, sg, Vt), info=False,
                 precision=spm.PREC_MIXED)
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1)

    def run_lr(S1, S2, q, oseed):
        # Algorithm 2: A ~ Y X with X = (S2^T Y)^+ (S2^T A), no Q^T A product
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        Y, X, _ = spm.lowrank(S1, S2, A, k, q, omega_seed=oseed, precision=spm.PREC_MIXED)
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1), Y, X

    records = []
    ident = spm.Sketch(n, n, 1, 0, kind=spm.IDENTITY)
    run(ident, 1, 43)                                   # warm-up (kernel attributes, pool)
    Sw = spm.Sketch(n, ls[0], 1, 41)
    run(Sw, 1, 43)
    Sw.close()
    c0 = lib.spm_launch_count()
    for t in range(a.trials):
        for l in ls:
            S = spm.Sketch(n, l, 1, 42 + t)
            run(S, 0, 43 + t)          # builds the sketch's gather plan, untimed
            for q in range(a.q_sketched + 1):
                ms = run(S, q, 43 + t)
                records.append({"method": "sketched", "l": l, "q": q, "ms": ms, "err": spectral_err()})
            S.close()
        for q in range(a.q_classical + 1):
            ms = run(ident, q, 43 + t)
            records.append({"method": "classical", "l": n, "q": q, "ms": ms, "err": spectral_err()})
        if a.poly_alg2:
            # Appendix D: Algorithm 2 with S1 a CountSketch of l columns against the
            # same algorithm with S1 = I (generalized Nystrom with power
            # iterations); S2 a CountSketch of the m rows to l in both
            for l in ls:
                S2 = spm.Sketch(m, l, 1, 142 + t)
                S1 = spm.Sketch(n, l, 1, 42 + t)
                run_lr(S1, S2, 0, 43 + t)  # the gather plan, untimed
                for q in range(a.q_sketched + 1):
                    ms, Y, X = run_lr(S1, S2, q, 43 + t)
                    records.append({"method": "alg2_sketched", "l": l, "q": q, "ms": ms,
                                    "err": spectral_err(Y, X)})
                for q in range(a.q_classical + 1):
                    ms, Y, X = run_lr(ident, S2, q, 43 + t)
                    records.append({"method": "alg2_generalized_nystrom", "l": l, "q": q,
                                    "ms": ms, "err": spectral_err(Y, X)})
                del Y, X
                S1.close()
                S2.close()
    launches = int(lib.spm_launch_count() - c0)
    curves, best = protocol_summary(records, a.poly_target)
    sk, cl = best.get("sketched"), best.get("classical")
    line = {
        "metric": f"time to relative spectral error <= {a.poly_target:g} (Section 4 protocol)",
        "value": sk["ms"] if sk else None, "unit": "ms", "n_gpus": 1, "steps": len(records),
        "warmup": 1, "ms_per_step": sk["ms"] if sk else None, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "bf16x3+f32", "data": "synthetic (seeded)",
        "config": {"workload": f"polydecay {m}x{n} f32, sigma_i = {m}/i, Haar factors, k = {k}; "
                               f"CountSketch l in {ls}, q = 0..{a.q_sketched}; classical q = "
                               f"0..{a.q_classical}; {a.trials} trials" +
                               ("; Algorithm 2 (S2: CountSketch of the rows to l) with S1 = "
                                "CountSketch l vs S1 = I" if a.poly_alg2 else ""),
                   "precision": "mixed",
                   "l2": "A (1.8 GB) larger than L2; no flush"},
        "best": best, "classical_ms_to_target": cl["ms"] if cl else None,
        "speedup_vs_classical": (cl["ms"] / sk["ms"]) if (sk and cl) else None,
        "alg2_speedup_vs_generalized_nystrom": (
            best["alg2_generalized_nystrom"]["ms"] / best["alg2_sketched"]["ms"]
            if best.get("alg2_sketched") and best.get("alg2_generalized_nystrom") else None),
        "curves": curves, "roofline": None, "e2e": None, "cpu_baseline": None,
        "gpu_launches": launches,
    }
    print(json.dumps(line), flush=True)


def main():
    a = parse()
    if a.impl == "reference":
        reference_main(a)
        return
    if a.workload == "batched":
        if a.batch_auto:
            batched_auto_main(a)
        else:
            batched_main(a)
        return
    if a.workload == "csr":
        csr_main(a)
        return
    if a.workload == "nystrom":
        nystrom_main(a)
        return
    if a.workload == "polydecay":
        polydecay_main(a)
        return
    import numpy as np
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    torch.backends.cuda.matmul.allow_tf32 = False
    from paper_2605_09755_gb300 import _build, spm
    from paper_2605_09755_gb300 import workloads as wl
    _build.build()
    spm.lib()

    m, n, r1, k = a.m, a.n, a.r1, a.k
    noise = a.noise / (n ** 0.5) if a.scaled_noise else a.noise
    A, sigma = wl.noisy_exp_torch(m, n, seed=1002 + rank * 0, noise=noise)
    torch.cuda.synchronize()
    kind = {"sparse": spm.SPARSE_SIGN, "dense": spm.DENSE_SIGN, "srht": spm.SRHT}[a.sketch]
    if a.sketch != "sparse":
        # the other families are compared on the timed step and its residual only
        # (their plain FP64 form would multiply by a dense n x r1 S on CUDA cores)
        a.no_fp64 = a.no_e2e = a.no_cpu = True
    S = spm.Sketch(n, r1, a.s, seed=42, kind=kind)
    U = torch.empty(m, k, device="cuda")
    sg = torch.empty(k, device="cuda")
    Vt = torch.empty(k, n, device="cuda")
    out = (U, sg, Vt)
    mixed = dict(precision=spm.PREC_MIXED, final_passes=a.final_passes,
                 power_passes=a.power_passes)

    def step(info=False, timing=False):
        return spm.rsvd(S, A, k, a.q, k, omega_seed=43, out=out, info=info, timing=timing, **mixed)

    # plain FP64 GPU form at the same q: the accuracy target (run once, untimed loop)
    fp64 = {}
    if not a.no_fp64:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        U64, s64, V64, inf64 = spm.rsvd(S, A, k, a.q, k, omega_seed=43, precision=spm.PREC_FP64,
                                        timing=True)
        torch.cuda.synchronize()
        fp64 = {"ms": (time.perf_counter() - t0) * 1e3,
                "residual": residual(A, U64, s64, V64),
                "stage_ms": inf64["stage_ms"], "sigma": s64.double().clone()}
        del U64, s64, V64
        torch.cuda.empty_cache()

    # warm-up, then the timed region (inputs are 4.3 GB >> 129 MB L2, no flush needed);
    # with --autotune the first warm-up step measures the products' split-K choices
    if a.autotune:
        spm.set_autotune(1)
    for _ in range(a.warmup):
        step()
    torch.cuda.synchronize()
    clocks = ClockSampler()
    clocks.start()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record()
    for _ in range(a.steps):
        step()
    ev1.record()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    ms_total = ev0.elapsed_time(ev1)
    if world > 1:
        ms_total = max_over_ranks(ms_total, dist, "cuda")
    ms_step = ms_total / a.steps
    value = per_approximation_ms(ms_total, a.steps, world)

    # stage breakdown (events recorded by the library on the launching stream), in
    # the timed steps' configuration (no |A|_F sum); then |A|_F and the estimate
    _, _, _, inf = step(info=True, timing=2)
    stages = inf["stage_ms"]
    _, _, _, inf = step(info=True)
    res_mixed = residual(A, U, sg, Vt)
    launches = None
    try:
        lib = spm.lib()
        c0 = lib.spm_launch_count()
        step()
        torch.cuda.synchronize()
        launches = int(lib.spm_launch_count() - c0) * a.steps
    except Exception:
        pass

    # roofline: the sketch product A S (Algorithm 1 line 1), the step's one pass
    # over A at HBM speed, is the kernel reported; the split-precision projection
    # B = Q^T A (3 BF16 passes of 2 m n k flops) is reported beside it
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    bf16_peak = peaks.get("bf16_tflops", 1900.0)
    proj_ms = stages.get("project", 0.0)
    apply_ms = stages.get("apply", 0.0)
    proj_flops = a.final_passes * 2.0 * m * n * k
    # A read once; A~ written as BF16 (hi, and lo when the power products use
    # the split); with the fused split of A (info a_split) also A's BF16 (hi, lo)
    # for the projection, 4 bytes per element of A
    a_split = bool(inf.get("a_split")) if inf else False
    apply_bytes = ((8.0 if a_split else 4.0) * m * n
                   + (4.0 if a.power_passes > 1 else 2.0) * m * r1)
    sched_state = spm.sketch_plan(S)[0] if a.sketch == "sparse" else -1
    apply_kernel = {"sparse": "k_sketch_sched" if sched_state == 1 else "k_sketch_apply_sacc",
                    "srht": "k_srht_apply", "dense": "k_gemm_tc (A S, dense sign)"}[a.sketch]
    proj_ach = proj_flops / (proj_ms * 1e-3) / 1e12 if proj_ms else None
    roof_proj = {"kernel": "k_gemm_tc (B = Q^T A, %d BF16 passes)" % a.final_passes,
                 "bound": "tensor", "achieved": proj_ach, "peak": bf16_peak, "unit": "TFLOP/s",
                 "frac": proj_ach / bf16_peak if proj_ach else None, "traffic": None,
                 "peak_source": "MEASURED_PEAKS.json bf16_tflops (burst), of measured"}
    if a.sketch == "dense":
        # the stage also holds the BF16 split of A and of the product; the
        # contraction's flops over the stage time bound its rate from below
        flops = (2 if a.power_passes > 1 else 1) * 2.0 * m * n * r1
        ach = flops / (apply_ms * 1e-3) / 1e12
        roof = {"kernel": apply_kernel + ", apply stage", "bound": "tensor", "achieved": ach,
                "peak": bf16_peak, "unit": "TFLOP/s", "frac": ach / bf16_peak, "traffic": None,
                "peak_source": "MEASURED_PEAKS.json bf16_tflops (burst), of measured"}
    else:
        ach = apply_bytes / (apply_ms * 1e-3) / 1e9
        roof = {"kernel": apply_kernel, "bound": "hbm", "achieved": ach, "peak": hbm_peak,
                "unit": "GB/s", "frac": ach / hbm_peak,
                # the table's capture is of the kernel with the fused split
                "traffic": ncu_traffic(apply_kernel, m, n, r1) if a_split else None,
                "algorithmic_bytes": apply_bytes,
                "peak_source": "MEASURED_PEAKS.json hbm_gbs, of measured"}
    sketch_roof = {"achieved_gbs": apply_bytes / (apply_ms * 1e-3) / 1e9 if apply_ms else None,
                   "frac": (apply_bytes / (apply_ms * 1e-3) / 1e9) / hbm_peak if apply_ms else None}

    # end to end through the public call with host buffers (spm_rsvd_host:
    # A staged from page-locked host memory in row chunks, overlapped with the
    # sketch product; U, sigma, Vt copied back)
    e2e = None
    if not a.no_e2e:
        Ah = A.cpu().pin_memory()
        Uh = torch.empty(m, k).pin_memory()
        sh = torch.empty(k).pin_memory()
        Vh = torch.empty(k, n).pin_memory()
        def e2e_step():
            spm.rsvd_host(S, Ah, k, a.q, k, omega_seed=43, out=(Uh, sh, Vh), info=False, **mixed)
        for _ in range(2):
            e2e_step()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(a.steps):
            e2e_step()
        e1.record()
        torch.cuda.synchronize()
        e2e = {"value": e0.elapsed_time(e1) / a.steps, "unit": "ms",
               "h2d_bytes_per_step": int(Ah.numel() * 4),
               "d2h_bytes_per_step": int((Uh.numel() + sh.numel() + Vh.numel()) * 4)}
        del Ah

    cpu = None
    if not a.no_cpu and rank == 0 and world == 1:
        rows = max(a.cpu_rows, k)
        Ar = A[:2 * rows].double().cpu().numpy()
        cpu_oracle_ms(Ar[:min(rows, 1024)], argparse.Namespace(**{**vars(a), "k": min(k, 256),
                                                                 "r1": min(r1, 512)}))
        est, t1, t2, rows = cpu_oracle_fit(Ar, a)
        cpu = {"value": est, "unit": "ms", "cores": os.cpu_count(), "kind": "oracle",
               "sample": f"oracle RandSVD on the first {rows} and {2 * rows} of {a.m} rows (same "
                         f"n, r1, k, q): {t1:.0f} and {t2:.0f} ms; the difference extrapolated "
                         f"linearly in m (the SVD of B and other m-independent work counted once)"}

    sig_err = None
    if fp64:
        s64 = fp64.pop("sigma")
        sig_err = float(torch.max(torch.abs(sg.double() - s64)) / s64[0])

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "ms", "n_gpus": world, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": ms_step, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "bf16x3+f32",
            "data": "synthetic (seeded, generated on device)",
            "config": {"workload": workload_name(a), "sketch": a.sketch, "precision": "mixed",
                       "final_passes": a.final_passes, "power_passes": a.power_passes,
                       "autotune": bool(a.autotune), "parallelism": "replicas" if world > 1 else "1 GPU",
                       "l2": "inputs (4.3 GB) larger than L2; no flush"},
            "accuracy": {"residual_mixed": res_mixed, "residual_fp64": fp64.get("residual"),
                         "ratio": (res_mixed / fp64["residual"]) if fp64 else None,
                         "sigma_err_vs_fp64": sig_err,
                         "fro_a": inf["fro_a"], "resid_est": inf["resid_est"]},
            "fp64_gpu_ms": fp64.get("ms"), "fp64_stage_ms": fp64.get("stage_ms"),
            "speedup_vs_fp64_gpu": (fp64["ms"] / value) if fp64 else None,
            "stage_ms": stages, "sketch_apply": sketch_roof,
            "roofline": roof, "roofline_projection": roof_proj, "e2e": e2e, "cpu_baseline": cpu,
            "gpu_launches": launches,
            "clocks": clk,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
