"""Learned dispatch on the GPU: the library's MLP kernels against the float64
reference (gradient, inference), training, the autotuned table, and the gain
of the trained model over the method without it (regret on measured timings)."""
import math

import numpy as np
import pytest

import ks_inputs as gen
import oracle
from oracle import mlp_ref
from tests._gpu import assert_same, random_case, to_dev, to_host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ks():
    import __graft_entry__ as ge
    ge.build()
    import paper_0712_4046_gb300 as ks
    return ks


def _data(seed, n=300):
    rng = np.random.default_rng(seed)
    p = rng.normal(0, 0.3, mlp_ref.n_params()).astype(np.float32)
    x = rng.random((n, 5)).astype(np.float32)
    t = rng.normal(3, 2, (n, 12)).astype(np.float32)
    m = (rng.random((n, 12)) < 0.8).astype(np.float32)
    return p, x, t, m


def test_gradient_matches_cpu_reference(ks):
    for seed in (1, 2, 3):
        p, x, t, m = _data(seed)
        g_gpu, loss_gpu = ks.mlp_grad(p, x, t, m)
        loss_ref, g_ref = mlp_ref.loss_and_grad(p.astype(np.float64), x, t, m)
        assert abs(loss_gpu - loss_ref) <= 1e-4 * abs(loss_ref) + 1e-6
        scale = np.abs(g_ref).max()
        err = np.abs(g_gpu - g_ref).max()
        assert err <= 2e-5 * scale + 1e-7, (seed, err, scale)


def test_inference_kernel_matches_reference(ks):
    p, x, _, _ = _data(9, 64)
    ks.mlp_set_params(p)
    try:
        y = ks.mlp_predict(x)
    finally:
        ks.mlp_set_params(None)
    y_ref, _ = mlp_ref.forward(p.astype(np.float64), x)
    assert np.abs(y - y_ref).max() <= 1e-4 * np.abs(y_ref).max() + 1e-5


def test_training_on_gpu_fits(ks):
    from paper_0712_4046_gb300 import dispatch
    rng = np.random.default_rng(4)
    x = rng.random((400, 5)).astype(np.float32)
    w = rng.normal(0, 1, (5, 12))
    t = (np.sin(3 * x) @ w + 2).astype(np.float32)
    m = np.ones_like(t)
    p0 = dispatch.init_params(3)
    loss0 = mlp_ref.loss_only(p0.astype(np.float64), x, t, m)
    p1, loss1 = ks.mlp_train(p0, x, t, m, 1500, 3e-3)
    assert loss1 < 0.05 * loss0, (loss0, loss1)
    assert abs(loss1 - mlp_ref.loss_only(p1.astype(np.float64), x, t, m)) < 1e-3 * (1 + loss1)


def test_table_changes_the_choice_not_the_result(ks):
    f, g = random_case(1000, 1000, 48, False, 8)
    want = oracle.mul(f, g, 48, False)
    ks.dispatch_set_table([(1000, 1000, 48, 0, 3, 1)])
    try:
        info = ks.plan_info(1000, 1000, 48, False, 0, 0)
        assert (info["variant"], info["engine"]) == (3, 1)
        h = ks.mul(to_dev(f), to_dev(g), 48, False)
        ks.status_sync()
        assert_same(to_host(h), want, "table dispatch")
    finally:
        ks.dispatch_set_table([])


def test_learned_dispatch_gains_over_the_method_without_it(ks):
    """On timings the library measured (the committed tuning run), a model
    trained by the GPU kernels on 3/4 of the shapes picks, on the held-out
    quarter, configurations closer to the measured best than the library
    without it (its built-in heuristic, and fixed KS1 with the library's
    engine) and than the autotuned table."""
    from paper_0712_4046_gb300 import dispatch
    body = dispatch.load_state()
    assert body is not None, "the committed dispatch state is missing or corrupt"
    data = body["timings"]
    train_set, test_set = dispatch.split(data)
    params, _ = dispatch.train(train_set, steps=4000)
    r_mlp = dispatch.regret(test_set, dispatch.mlp_choices(params, test_set))
    dispatch.uninstall()
    try:
        r_heuristic = dispatch.regret(test_set, dispatch.library_choices(test_set))
        r_ks1 = dispatch.regret(test_set, dispatch.library_choices(test_set, variant=1))
    finally:
        dispatch.install()
    # and closer than the exhaustive table built from the same training shapes
    # (nearest measured shape, one product at a time)
    table = dispatch.choose_table(dispatch.build_table(train_set))
    r_table = dispatch.regret(test_set, [table(d) for d in test_set])
    assert r_mlp < r_heuristic, (r_mlp, r_heuristic)
    assert r_mlp < r_ks1, (r_mlp, r_ks1)
    assert r_mlp <= r_table, (r_mlp, r_table)
    assert r_mlp < 0.25, r_mlp
