"""The tensor-core surrogate network (mlp_* through the C ABI) against the
numpy oracle that reproduces its BF16 rounding points: forward outputs,
gradients of every parameter group, training."""
import numpy as np
import pytest

from oracle import mlp_oracle as M
from paper_2002_03120_gb300 import binding as B

from _gpu_common import need_gpu, rel_l2

pytestmark = pytest.mark.gpu

ORDER = ["W0", "b0", "W1", "b1", "W2", "b2", "W3", "b3", "W4", "b4"]


def flat(p):
    return np.concatenate([np.asarray(p[k], dtype=np.float64).reshape(-1) for k in ORDER])


def unflat(v, like):
    out, o = {}, 0
    for k in ORDER:
        n = like[k].size
        out[k] = v[o:o + n].reshape(like[k].shape)
        o += n
    return out


@pytest.fixture(autouse=True)
def _gpu():
    need_gpu()


def _dev(a):
    import torch
    return torch.tensor(np.asarray(a, dtype=np.float32), device="cuda")


def _params(seed):
    p = M.init_params(seed)
    rng = np.random.default_rng(seed + 100)
    for k in ORDER:
        if k.startswith("b"):
            p[k] = rng.normal(0, 0.1, size=p[k].shape)
    # the GPU holds FP32 masters: give the oracle the same values
    return {k: np.asarray(v, dtype=np.float32).astype(np.float64) for k, v in p.items()}


@pytest.mark.parametrize("n", [128, 1000])
def test_forward_matches_oracle(n):
    import torch
    p = _params(1)
    net = B.Mlp(seed=0)
    net.set_params(flat(p))
    X = np.random.default_rng(2).uniform(size=(n, 3))
    Y = torch.zeros(n, dtype=torch.float32, device="cuda")
    net.infer(_dev(X), Y)
    net.check()
    y_gpu = Y.cpu().numpy()
    y_ref, _ = M.forward(p, X.astype(np.float32).astype(np.float64), "bf16")
    assert rel_l2(y_gpu, y_ref) < 1e-3, rel_l2(y_gpu, y_ref)


@pytest.mark.parametrize("batch", [256, 200])
def test_gradients_match_oracle(batch):
    p = _params(3)
    net = B.Mlp(seed=0, batch_max=256)
    net.set_params(flat(p))
    rng = np.random.default_rng(4)
    X = rng.uniform(size=(batch, 3)).astype(np.float32)
    T = rng.normal(size=batch).astype(np.float32)
    loss = net.gradients(_dev(X), _dev(T))
    g_gpu = unflat(net.grads().astype(np.float64), p)
    y, cache = M.forward(p, X.astype(np.float64), "bf16")
    g_ref = M.backward(p, cache, y, T.astype(np.float64))
    assert loss == pytest.approx(M.loss(y, T), rel=1e-3)
    for k in ORDER:
        assert rel_l2(g_gpu[k], g_ref[k]) < 5e-3, (k, rel_l2(g_gpu[k], g_ref[k]))


def test_training_fits_a_smooth_target():
    net = B.Mlp(seed=7, batch_max=256)
    rng = np.random.default_rng(8)
    X = rng.uniform(size=(2048, 3)).astype(np.float32)
    T = (np.sin(3 * X[:, 0]) + X[:, 1] * X[:, 2]).astype(np.float32)
    Xd, Td = _dev(X), _dev(T)
    first = None
    for ep in range(150):
        for b in range(0, 2048, 256):
            l = net.train_step(Xd[b:b + 256], Td[b:b + 256], lr=2e-3, want_loss=(b == 0))
            if b == 0 and first is None:
                first = l
    import torch
    Y = torch.zeros(2048, dtype=torch.float32, device="cuda")
    net.infer(Xd, Y)
    net.check()
    mse = float(np.mean((Y.cpu().numpy() - T) ** 2))
    assert mse < 0.02 * first, (mse, first)
