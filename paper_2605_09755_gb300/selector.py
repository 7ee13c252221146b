"""Training data and training loop of the learned (q, sketch size) selector.

Runs of the method itself label the data: for each generated matrix with a
known spectrum, the q = 0 sketch features (spm_selector_features) are the input
and, for every candidate (q in 0..4, r1 = c k with c in {2, 4, 8}), the target
is log10(residual / optimal - 1) of the mixed-precision range finder, where
optimal is the Eckart-Young error sqrt(sum_{i>k} sigma_i^2).  Training runs on
the GPU through spm_mlp_loss_grad / spm_mlp_adam.

    python -m paper_2605_09755_gb300.selector --matrices 1334 --steps 3000
"""
import argparse
import json
import math
import os
import time

import numpy as np
import torch

from . import spm
from . import workloads as wl

HERE = os.path.dirname(os.path.abspath(__file__))
PARAMS_PATH = os.path.join(HERE, "selector_params.npy")
FLOOR = 1e-4   # ratios closer to 1 than this are all "at the optimum"


def random_spec(rng, small=True):
    """Shapes and spectrum of one training matrix (the batched workload's family)."""
    lo_m, hi_m, lo_n, hi_n = (512, 4096, 256, 2048) if small else (512, 8192, 256, 4096)
    m = int(round(math.exp(rng.uniform(math.log(lo_m), math.log(hi_m)))))
    n = int(round(math.exp(rng.uniform(math.log(lo_n), math.log(hi_n)))))
    k = int(rng.integers(16, 129 if small else 257))
    k = min(k, n // 8, m // 2)
    k = max(k, 4)
    if rng.uniform() < 0.5:
        kind, par = "poly", float(rng.uniform(0.5, 2.0))
    else:
        kind, par = "exp", float(rng.uniform(10.0, 200.0))
    return dict(m=m, n=n, k=k, kind=kind, par=par, seed=int(rng.integers(1 << 31)))


def make_matrix(spec):
    """A = U diag(sigma) V^T on the device (float32) and its sigma (float64)."""
    sigma = wl.batch_sigma(spec)
    wl.load_torch_linalg()
    g = torch.Generator(device="cuda").manual_seed(spec["seed"])
    r = sigma.size
    U, Ru = torch.linalg.qr(torch.randn(spec["m"], r, generator=g, device="cuda"))
    V, Rv = torch.linalg.qr(torch.randn(spec["n"], r, generator=g, device="cuda"))
    U *= torch.sign(torch.diagonal(Ru))
    V *= torch.sign(torch.diagonal(Rv))
    A = (U * torch.tensor(sigma, dtype=torch.float32, device="cuda")) @ V.T
    return A.contiguous(), sigma


def residual_ratio(A, Q, opt):
    R = A - Q @ (Q.T @ A)
    return float(torch.linalg.norm(R.double())) / opt


def run_candidates(A, sigma, k, seed=42):
    """Features of the q = 0 probe and the label vector over the 15 candidates."""
    m, n = A.shape
    opt = float(np.sqrt(np.sum(np.sort(sigma)[::-1][k:] ** 2)))
    r1p = min(4 * k, n)
    P = spm.Sketch(n, r1p, min(8, r1p), seed)
    feat = spm.selector_features(P, A, k, omega_seed=seed + 1).cpu().numpy()
    P.close()
    y = np.zeros(spm.MLP_OUT, dtype=np.float32)
    mask = np.ones(spm.MLP_OUT, dtype=np.float32)
    for idx, (q, c) in enumerate(spm.CANDIDATES):
        r1 = min(c * k, n)
        S = spm.Sketch(n, r1, min(8, r1), seed)
        Q, _ = spm.range_finder(S, A, k, q, omega_seed=seed + 1, precision=spm.PREC_MIXED)
        S.close()
        ratio = residual_ratio(A, Q, opt) if opt > 0 else 1.0
        y[idx] = np.log10(max(ratio - 1.0, FLOOR))
    return feat, y, mask


def generate(count, seed=7, small=True, log_every=100):
    rng = np.random.default_rng(seed)
    X, Y, M, specs = [], [], [], []
    t0 = time.time()
    for i in range(count):
        spec = random_spec(rng, small)
        A, sigma = make_matrix(spec)
        f, y, mk = run_candidates(A, sigma, spec["k"])
        X.append(f)
        Y.append(y)
        M.append(mk)
        specs.append(spec)
        if log_every and (i + 1) % log_every == 0:
            print(f"  {i + 1}/{count} matrices, {time.time() - t0:.1f} s", flush=True)
    return np.array(X, np.float32), np.array(Y, np.float32), np.array(M, np.float32), specs


def init_params(seed=0):
    rng = np.random.default_rng(seed)
    sizes = [(64, 8), (64, 64), (64, 64), (15, 64)]
    parts = []
    for o, i in sizes:
        parts.append(rng.standard_normal(o * i) * np.sqrt(2.0 / i))
        parts.append(np.zeros(o))
    return np.concatenate(parts).astype(np.float32)


def train(X, Y, M, steps=3000, lr=2e-3, seed=0, log_every=500):
    """Full-batch Adam on the GPU; returns the trained parameters (float32 numpy)."""
    p = torch.tensor(init_params(seed), device="cuda")
    m = torch.zeros_like(p)
    v = torch.zeros_like(p)
    Xd, Yd, Md = (torch.tensor(a, device="cuda") for a in (X, Y, M))
    hist = []
    for t in range(1, steps + 1):
        loss, grad = spm.mlp_loss_grad(p, Xd, Yd, Md)
        spm.mlp_adam(p, m, v, grad, t, lr=lr * (0.5 ** (t / (steps / 3))))
        if t % log_every == 0 or t == 1:
            hist.append((t, float(loss)))
    return p.cpu().numpy(), hist


def load_params(path=PARAMS_PATH):
    return torch.tensor(np.load(path).astype(np.float32), device="cuda")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--matrices", type=int, default=1334)   # x 15 candidates ~ 20k runs
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--out", default=PARAMS_PATH)
    ap.add_argument("--data-out", default="")
    a = ap.parse_args()
    from . import _build
    _build.build()
    t0 = time.time()
    X, Y, M, specs = generate(a.matrices)
    t_gen = time.time() - t0
    if a.data_out:
        np.savez(a.data_out, X=X, Y=Y, M=M)
    t0 = time.time()
    params, hist = train(X, Y, M, a.steps)
    t_train = time.time() - t0
    np.save(a.out, params)
    print(json.dumps({"matrices": a.matrices, "runs": int(M.sum()), "gen_s": t_gen,
                      "train_s": t_train, "loss": hist}), flush=True)


if __name__ == "__main__":
    main()
