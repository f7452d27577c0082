"""Host logic of the warm-start comparison (no GPU): the applies bookkeeping, the stopping rule,
the input / output scales and the seeded training set."""
import numpy as np


def test_cgls_applies_counts_the_products():
    from paper_1912_06976_gb300 import warmstart as WS

    # plain CGLS from zero: s0 = G^T d, then one G and one G^T per iteration
    assert WS.cgls_applies(0, warm=False) == 1
    assert WS.cgls_applies(7, warm=False) == 15
    # from x0: r0 = d - G x0 costs one more product
    assert WS.cgls_applies(0, warm=True) == 2
    assert WS.cgls_applies(6, warm=True) == 14


def test_iterations_to_reach_is_the_first_crossing():
    from paper_1912_06976_gb300 import warmstart as WS

    res = [5.0, 3.0, 2.0, 2.5, 1.0]
    assert WS.iterations_to_reach(res, 2.0) == 2  # equality reaches the target
    assert WS.iterations_to_reach(res, 5.0) == 0
    assert WS.iterations_to_reach(res, 0.5) is None


def test_fit_scales_are_the_reciprocal_data_rms_and_the_model_rms():
    from paper_1912_06976_gb300 import warmstart as WS

    rng = np.random.default_rng(3)
    models = rng.standard_normal((4, 2, 3, 3)).astype(np.float32) * 0.3
    data = rng.standard_normal((4, 3, 3)).astype(np.float32) * 7.0
    a, b = WS.fit_scales(models, data)
    assert np.isclose(a, 1.0 / np.sqrt(np.mean(data.astype(np.float64) ** 2)), rtol=1e-12)
    assert np.isclose(b, np.sqrt(np.mean(models.astype(np.float64) ** 2)), rtol=1e-12)


def test_training_models_do_not_depend_on_the_thread_count():
    from paper_1912_06976_gb300 import warmstart as WS

    shape = (4, 16, 16)
    one = WS.training_models(6, seed=5, shape=shape, threads=1)
    many = WS.training_models(6, seed=5, shape=shape, threads=4)
    assert one.shape == (6,) + shape and one.dtype == np.float32
    assert np.array_equal(one, many)
    assert not np.array_equal(one[0], one[1])  # each index draws its own model
    assert not np.array_equal(one, WS.training_models(6, seed=6, shape=shape, threads=2))
