"""The learned selector end to end on the GPU: labels measured by the
pipeline (exhaustive class search), the network trained by the library's own
kernels, and on held-out columns a small regret against the exhaustive
search -- well below the rule-based heuristic's, the method without it."""
import numpy as np
import pytest

import zf_workloads as W

zf = pytest.importorskip("paper_2602_08190_gb300")
pytestmark = pytest.mark.gpu


def test_selector_trained_on_measured_labels_beats_the_heuristic():
    import bench
    ctx = zf.zf_ctx_create(0)
    try:
        zf.zf_ctx_set_kcfg(ctx, 0, 0, 0, 16 << 20, 0)
        n_train, n_test, cap = 300, 60, 262144
        F, T, fam, dts = bench.selector_dataset(zf, ctx, range(1, n_train + n_test + 1), cap)
        assert F.shape == (n_train + n_test, 32) and T.shape == (n_train + n_test, 12)
        # every column has at least one measured class; string columns only RAW / LZ77
        assert np.all((T >= 0).any(1))
        is_bytes = F[:, 2] > 0.5
        assert np.all(T[is_bytes][:, [2, 3, 4, 5, 6, 7, 8, 9]] < 0)
        res, net = bench.selector_eval(zf, ctx, F, T, n_train)
        try:
            assert res["loss_last"] < res["loss_first"]
            assert res["regret"] <= 0.10
            heur = []
            for i, s in enumerate(range(n_train + 1, n_train + n_test + 1)):
                x, o, meta = W.selector_column(s, cap)
                p = zf.zf_plan(None, zf.Column(x, o), selector=0)
                k = p.scheme * 2 if o is None else zf.ZF_LZ77 * 2
                tt = T[n_train + i]
                if tt[k] >= 0:
                    heur.append((tt[k] - tt[tt >= 0].min()) / tt[tt >= 0].min())
            assert res["regret"] < np.mean(heur)
            # the network standardizes its inputs with the training rows' statistics
            mean, std = zf.zf_mlp_get_scaling(net)
            Ftr = F[:n_train].astype(np.float64)
            assert np.allclose(mean, Ftr.mean(0), rtol=1e-4, atol=1e-5)
            sd = Ftr.std(0)
            assert np.allclose(std, np.where(sd > 0, sd, 1.0), rtol=1e-3, atol=1e-5)
            # zf_plan with the attached network (its own scaling) makes the same choice as the batch prediction
            zf.zf_ctx_set_selector(ctx, net)
            for i in (0, 1, 3):
                x, o, meta = W.selector_column(n_train + 1 + i, cap)
                p = zf.zf_plan(ctx, zf.Column(x, o), selector=1)
                assert p.label == res["pred"][i]
                assert p.scheme == p.label // 2
            # selector 2 measures every class and keeps the fastest
            x, o, meta = W.selector_column(n_train + 2, cap)
            p = zf.zf_plan(ctx, zf.Column(x, o), selector=2)
            assert p.label >= 0 and p.predicted_ms > 0
        finally:
            zf.zf_ctx_set_selector(ctx, None)
            zf.zf_mlp_destroy(net)
    finally:
        zf.zf_ctx_destroy(ctx)
