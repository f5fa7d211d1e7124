"""The selector network's CUDA kernels against the float64 oracle:
forward logits, batch gradients and the Adam step agree within FP32
tolerance; training on the GPU learns a separable toy problem."""
import numpy as np
import pytest

from oracle import mlp as M

zf = pytest.importorskip("paper_2602_08190_gb300")
pytestmark = pytest.mark.gpu

RTOL, ATOL = 1e-4, 1e-5


def _close(a, b, scale=None):
    scale = np.max(np.abs(b)) if scale is None else scale
    return np.max(np.abs(np.asarray(a, np.float64) - b)) <= ATOL + RTOL * max(scale, 1.0)


def _batch(seed, B=37):
    rng = np.random.default_rng(seed)
    X = rng.normal(size=(B, M.IN)).astype(np.float32)
    y = rng.integers(0, M.OUT, B).astype(np.int32)
    mask = rng.random((B, M.OUT)) < 0.7
    mask[np.arange(B), y] = True
    return X, y, mask


def test_forward_gradient_and_adam_match_oracle():
    import torch
    net = zf.zf_mlp_create(0, 3)
    try:
        p32 = (M.he_init(3) + 0.01 * np.random.default_rng(4).normal(size=M.NPARAMS)).astype(np.float32)
        zf.zf_mlp_set_params(net, p32)
        assert np.array_equal(zf.zf_mlp_get_params(net), p32)
        p = p32.astype(np.float64)
        X, y, mask = _batch(1)
        B = len(y)
        dx = torch.from_numpy(X).cuda()
        dy = torch.from_numpy(y).cuda()
        dm = torch.from_numpy(mask.astype(np.uint8)).cuda()
        dz = torch.empty((B, M.OUT), dtype=torch.float32, device="cuda")
        dg = torch.empty(M.NPARAMS, dtype=torch.float32, device="cuda")
        dl = torch.empty(1, dtype=torch.float32, device="cuda")
        zf.zf_mlp_forward(net, dx.data_ptr(), B, dz.data_ptr())
        z_ref, _ = M.forward(p, X.astype(np.float64))
        torch.cuda.synchronize()
        assert _close(dz.cpu().numpy(), z_ref)
        zf.zf_mlp_grad(net, dx.data_ptr(), dy.data_ptr(), dm.data_ptr(), B, dg.data_ptr(), dl.data_ptr())
        loss_ref, g_ref = M.loss_grad(p, X.astype(np.float64), y, mask)
        torch.cuda.synchronize()
        assert abs(dl.item() - loss_ref) <= ATOL + RTOL * abs(loss_ref)
        g = dg.cpu().numpy()
        for name, _ in M.SHAPES:                         # per tensor
            assert _close(M.unpack(g.astype(np.float64))[name], M.unpack(g_ref)[name],
                          scale=np.max(np.abs(g_ref))), name
        zf.zf_mlp_adam(net, dg.data_ptr(), 1e-3)
        torch.cuda.synchronize()
        p_ref, _, _ = M.adam(p, g.astype(np.float64), np.zeros_like(p), np.zeros_like(p), 1, 1e-3)
        assert _close(zf.zf_mlp_get_params(net), p_ref)
    finally:
        zf.zf_mlp_destroy(net)


def test_gpu_training_learns_separable_toy_and_is_deterministic():
    rng = np.random.default_rng(7)
    centers = rng.normal(size=(M.OUT, M.IN)) * 3
    y = rng.integers(0, M.OUT, 600).astype(np.int32)
    X = (centers[y] + 0.3 * rng.normal(size=(600, M.IN))).astype(np.float32)
    mask = np.ones((600, M.OUT), np.uint8)
    params = []
    for _ in range(2):
        net = zf.zf_mlp_create(0, 11)
        try:
            losses = zf.zf_mlp_train(net, X, y, mask, 60, 64, 3e-3, seed=5)
            assert losses[-1] < losses[0] * 0.1
            assert (zf.zf_mlp_predict(net, X, mask) == y).mean() == 1.0
            m2 = mask.copy()
            m2[:, 0] = 0
            assert not np.any(zf.zf_mlp_predict(net, X, m2) == 0)
            params.append(zf.zf_mlp_get_params(net))
        finally:
            zf.zf_mlp_destroy(net)
    assert np.array_equal(params[0], params[1])
