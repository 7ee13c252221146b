"""GPU parity of the selector network kernels and features against the FP64 oracle."""
import numpy as np
import pytest
import torch

from oracle import mlp as omlp
from oracle import sketch as osk
from oracle import algorithms as alg
from paper_2605_09755_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def spm():
    from paper_2605_09755_gb300 import _build, spm as _spm
    _build.build()
    _spm.lib()
    return _spm


def _rand(seed, batch=37):
    rng = np.random.default_rng(seed)
    p = (omlp.init_params(seed) * 0.7).astype(np.float32).astype(np.float64)
    X = rng.standard_normal((batch, omlp.D_IN)).astype(np.float32).astype(np.float64)
    T = rng.standard_normal((batch, omlp.D_OUT)).astype(np.float32).astype(np.float64)
    M = (rng.uniform(size=(batch, omlp.D_OUT)) > 0.2).astype(np.float64)
    return p, X, T, M


def dev(a):
    return torch.tensor(np.asarray(a, dtype=np.float32), device="cuda")


def test_mlp_forward_matches_oracle(spm):
    p, X, _, _ = _rand(1, batch=300)
    Y = spm.mlp_forward(dev(p), dev(X)).double().cpu().numpy()
    Yo, _ = omlp.forward(p, X)
    assert np.max(np.abs(Y - Yo)) <= 1e-5 * max(1.0, np.abs(Yo).max())


@pytest.mark.parametrize("batch", [1, 37, 1000])
def test_mlp_loss_grad_matches_oracle(spm, batch):
    p, X, T, M = _rand(2, batch)
    loss, g = spm.mlp_loss_grad(dev(p), dev(X), dev(T), dev(M))
    lo, go = omlp.loss_grad(p, X, T, M)
    assert abs(float(loss) - lo) <= 1e-5 * max(1.0, abs(lo))
    g = g.double().cpu().numpy()
    assert np.max(np.abs(g - go)) <= 1e-4 * max(1.0, np.abs(go).max())


def test_mlp_adam_matches_oracle(spm):
    p, X, T, M = _rand(3, 64)
    pd, md, vd = dev(p), torch.zeros(omlp.N_PARAMS, device="cuda"), torch.zeros(omlp.N_PARAMS, device="cuda")
    po, mo, vo = p.copy(), np.zeros(omlp.N_PARAMS), np.zeros(omlp.N_PARAMS)
    for t in range(1, 4):
        _, g = spm.mlp_loss_grad(pd, dev(X), dev(T), dev(M))
        spm.mlp_adam(pd, md, vd, g, t, lr=1e-2)
        _, go = omlp.loss_grad(po, X, T, M)
        po, mo, vo = omlp.adam(po, mo, vo, go, t, lr=1e-2)
    assert np.max(np.abs(pd.double().cpu().numpy() - po)) <= 1e-4


def test_mlp_training_reduces_loss(spm):
    """Full-batch Adam through the library kernels fits a smooth target."""
    rng = np.random.default_rng(5)
    X = rng.uniform(-1, 1, (512, omlp.D_IN))
    T = np.stack([np.sin(X[:, 0] * (1 + j / 10)) + X[:, 1] * X[:, 2] for j in range(omlp.D_OUT)], 1)
    M = np.ones_like(T)
    p = dev(omlp.init_params(0))
    m = torch.zeros_like(p)
    v = torch.zeros_like(p)
    first = None
    for t in range(1, 401):
        loss, g = spm.mlp_loss_grad(p, dev(X), dev(T), dev(M))
        if first is None:
            first = float(loss)
        spm.mlp_adam(p, m, v, g, t, lr=3e-3)
    assert float(loss) < 0.05 * first


@pytest.mark.parametrize("m,n,r1,r2", [(600, 300, 64, 16), (1000, 512, 256, 64)])
def test_selector_features_match_oracle(spm, m, n, r1, r2):
    A, sigma = wl.dense_lowrank(m, n, 1.0 / np.arange(1, min(m, n) + 1) ** 0.8, seed=4)
    So = osk.Sketch(n, r1, 8, 42)
    Y0 = alg.sketched_power(osk.apply_right(A, So), osk.gaussian(r1, r2, 43), 0)
    fo = omlp.features_from_sketch(Y0, m, n, r1)
    S = spm.Sketch(n, r1, 8, 42)
    f = spm.selector_features(S, torch.tensor(A, dtype=torch.float32, device="cuda"), r2,
                              omega_seed=43).double().cpu().numpy()
    assert np.max(np.abs(f - fo)) <= 2e-3, (f, fo)
