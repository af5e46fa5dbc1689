"""The seeded input generator: shapes, structure and bit-for-bit determinism."""
import numpy as np
import pytest

from paper_2012_07620_gb300 import synthetic as s

# SHA-256 of (xq, xg) for the tiny workload; the same bytes must come out on
# every platform (the generator avoids libm; see the module docstring).
TINY_DIGEST_VALUE = "1b491f1d79575c3f22a106da512bb61392e50401515ccfe446dcb841c741dee8"


def test_tiny_shapes_and_labels():
    w = s.make_workload(s.TINY)
    assert w.xq.shape == (100, 128) and w.xg.shape == (900, 128)
    assert w.xq.dtype == np.float32
    np.testing.assert_allclose(np.linalg.norm(w.xq, axis=1), 1.0, atol=1e-6)
    np.testing.assert_allclose(np.linalg.norm(w.xg, axis=1), 1.0, atol=1e-6)
    counts_g = np.bincount(w.yg, minlength=50)
    assert (counts_g >= 1).all()              # every query's cluster keeps a gallery member
    assert (np.bincount(w.yq, minlength=50) + counts_g == 20).all()


def test_deterministic():
    a = s.make_workload(s.TINY)
    b = s.make_workload(s.TINY)
    assert s.array_digest(a.xq, a.xg) == s.array_digest(b.xq, b.xg)


def test_digest_pin():
    w = s.make_workload(s.TINY)
    assert s.array_digest(w.xq, w.xg) == TINY_DIGEST_VALUE


def test_cluster_sizes_market_shape():
    spec = s.MARKET_SCALE
    sizes = s._cluster_sizes(spec, spec.n - spec.n_distractors)
    assert sizes.sum() == 21100 and sizes.min() >= 8 and sizes.max() <= 30
    assert len(sizes) == 1501


def test_gaussian_moments():
    z = s.SplitMix64(7, "moments").normal(400_000)
    assert abs(z.mean()) < 0.01 and abs(z.var() - 1) < 0.01
    assert abs((z ** 4).mean() / z.var() ** 2 - 3.0) < 0.05


def test_portable_math_close_to_libm():
    u = s.SplitMix64(3, "u").uniform(10000)
    np.testing.assert_allclose(s._ln(u), np.log(u), rtol=0, atol=4e-15)
    c, sn = s._cos_sin_turns(u)
    np.testing.assert_allclose(c, np.cos(2 * np.pi * u), atol=2e-15)
    np.testing.assert_allclose(sn, np.sin(2 * np.pi * u), atol=2e-15)


def test_batched_specs():
    specs = s.batched_specs()
    assert len(specs) == 64
    for b in specs:
        sp_ = b["spec"]
        assert 500 <= sp_.n <= 8000 and sp_.dim in (256, 512, 2048)
        assert 20 <= b["k1"] <= 30 and 5 <= b["k2"] <= 7 and 1 <= b["layers"] <= 3
