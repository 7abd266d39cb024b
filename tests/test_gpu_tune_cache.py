"""Tuning cache file (krr_tune_save / krr_tune_load): the autotuner's picks
(kernel variant and split scale per product shape) written on one handle and
read into another give the same products bit for bit; the file round-trips;
malformed files, missing files and files from a device with another SM count
are refused with KRR_ERR_INVALID_ARG.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def K():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_1408_1237_gb300 import binding
    return binding


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _tuned_handle(K):
    h = K.Handle()
    K.krr_set_option(K.KRR_OPT_AUTOTUNE, 1, handle=h)
    return h


def test_tune_cache_round_trip(K, tmp_path):
    rng = np.random.default_rng(11)
    X = _dev(rng.random((60000, 2)).astype(np.float32))
    q = _dev(rng.standard_normal(60000).astype(np.float32))
    Q = _dev(rng.standard_normal((12, 60000)).astype(np.float32))
    path = tmp_path / "tune.txt"
    h1 = _tuned_handle(K)
    try:
        for arg in (q, Q):
            K.krr_kernel_mvp(X, arg, 0.05, 1e-3, handle=h1)  # tunes this shape
        ref = [K.krr_kernel_mvp(X, arg, 0.05, 1e-3, handle=h1).cpu().numpy() for arg in (q, Q)]
        K.krr_tune_save(path, handle=h1)
    finally:
        h1.close()
    lines = path.read_text().splitlines()
    assert lines[0].startswith("krr-tune 1 sms ") and len(lines) >= 3
    h2 = _tuned_handle(K)
    try:
        K.krr_tune_load(path, handle=h2)
        got = [K.krr_kernel_mvp(X, arg, 0.05, 1e-3, handle=h2).cpu().numpy() for arg in (q, Q)]
        path2 = tmp_path / "tune2.txt"
        K.krr_tune_save(path2, handle=h2)
    finally:
        h2.close()
    for a, b in zip(ref, got):
        np.testing.assert_array_equal(a, b)
    assert path2.read_text().splitlines()[0] == lines[0]
    assert sorted(path2.read_text().splitlines()[1:]) == sorted(lines[1:])


def test_tune_cache_refuses_bad_files(K, tmp_path):
    h = K.Handle()
    try:
        good = tmp_path / "good.txt"
        K.krr_tune_save(good, handle=h)
        header = good.read_text().splitlines()[0]
        sms = int(header.split()[-1])
        cases = {
            "missing": None,
            "not_a_cache": "hello\n",
            "other_device": f"krr-tune 1 sms {sms + 1}\n",
            "bad_scale": header + "\nmvp|1|1|3|0|1|0|0|3|0|0\t-2\t1\n",
            "bad_variant": header + "\nmvp|1|1|3|0|1|0|0|3|0|0\t1\t99\n",
            "missing_field": header + "\nmvp|1|1|3|0|1|0|0|3|0|0\t1\n",
        }
        for name, text in cases.items():
            p = tmp_path / f"{name}.txt"
            if text is not None:
                p.write_text(text)
            with pytest.raises(K.KrrError) as ei:
                K.krr_tune_load(p, handle=h)
            assert ei.value.status == K.KRR_ERR_INVALID_ARG, name
        K.krr_tune_load(good, handle=h)  # an empty cache loads
    finally:
        h.close()
