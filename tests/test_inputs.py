"""The seeded input recipes (paper_1902_03070_gb300/inputs.py, serve.py):
exact mask counts, observed fractions, value ranges, the low-rank structure
each workload is built to have, the batch's shape ranges and the serving
stream's determinism and class mapping.  CPU only; the low-rank cores come
from the oracle's t-product."""
import numpy as np
import pytest

import oracle as O
from paper_1902_03070_gb300 import inputs, serve


def test_uniform_mask_exact_count():
    rng = np.random.default_rng(3)
    for shape, frac in (((7, 5, 3), 0.4), ((10, 10, 10), 0.2), ((4, 4, 4), 1.0), ((4, 4, 4), 0.0)):
        m = inputs.uniform_mask(shape, frac, rng)
        assert m.dtype == np.uint8 and m.flags.f_contiguous and m.shape == shape
        assert int(m.sum()) == int(round(frac * np.prod(shape)))
        assert set(np.unique(m)) <= {0, 1}


def test_config1_tubal_rank_and_mask():
    d = inputs.config1(O.tprod)
    T, B, mask = d["T"], d["B"], d["mask"]
    assert T.shape == (48, 48, 16)
    assert int(mask.sum()) == int(round(0.4 * T.size))
    assert np.array_equal(B, T * mask)
    # tubal rank 3: every slice of the transformed tensor has rank 3
    Tb = O.tube_transform(T)
    for k in range(T.shape[2]):
        s = np.linalg.svd(Tb[:, :, k], compute_uv=False)
        assert s[3] <= 1e-10 * s[0] and s[2] > 1e-6 * s[0]
    d2 = inputs.config1(O.tprod)
    assert np.array_equal(d2["T"], T) and np.array_equal(d2["mask"], mask)


def test_config2_recipe_small():
    d = inputs.config2(O.tprod, n1=24, n2=30, n3=20)
    T, mask = d["T"], d["mask"]
    assert T.shape == (24, 30, 20) and T.min() >= 0.0 and T.max() <= 1.0
    assert int(mask.sum()) == int(round(0.2 * T.size))
    assert np.array_equal(d["B"], T * mask)
    assert d["admm"]["max_iter"] == 200


def test_config3_spectral_rank():
    d = inputs.config3(n1=48, n2=40, n3=31)
    T = d["T"]
    assert T.shape == (48, 40, 31) and T.min() >= 0.0 and T.max() <= 1.0 + 1e-12
    assert int(d["mask"].sum()) == int(round(0.1 * T.size))
    # five spectral signatures times abundance maps: the spectral unfolding has rank 5
    s = np.linalg.svd(T.reshape(-1, 31, order="F"), compute_uv=False)
    assert s[5] <= 1e-10 * s[0] and s[4] > 1e-8 * s[0]


def test_config4_shapes_and_tau():
    shapes = inputs.config4_shapes()
    assert len(shapes) == 64
    for n1, n2, n3, r in shapes:
        assert 32 <= n1 <= 256 and 32 <= n2 <= 256 and 8 <= n3 <= 64 and 2 <= r <= 12
    assert inputs.config4_shapes() == shapes
    assert inputs.config4_tau(100, 64) == pytest.approx(2e-3 * (10 + 8))


def test_serving_stream():
    a = serve.make_stream(8, 200.0, seed=11, tprod=O.tprod, n_batch_shapes=2)
    b = serve.make_stream(8, 200.0, seed=11, tprod=O.tprod, n_batch_shapes=2)
    arr = [j["arrival"] for j in a]
    assert arr[0] == 0.0 and all(x <= y for x, y in zip(arr, arr[1:]))
    for ja, jb in zip(a, b):
        assert ja["arrival"] == jb["arrival"] and ja["cls"] == jb["cls"]
        assert np.array_equal(ja["B"], jb["B"]) and np.array_equal(ja["mask"], jb["mask"])
        assert ja["cls"] in serve.CLASSES and ja["prec"] == serve.PREC[ja["cls"]]
        assert ja["B"].dtype == (np.float64 if ja["prec"] == "fp64" else np.float32)
        assert 0.1 <= ja["observed"] <= 0.5
        assert np.all(ja["B"][ja["mask"] == 0] == 0)
        assert ja["params"]["max_iter"] == serve.ITERS[ja["cls"]] and ja["params"]["tol"] == 1e-5
