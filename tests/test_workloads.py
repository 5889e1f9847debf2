"""The seeded input generators keep the recipe they document.

The generators are the one module that the CUDA path and the oracle both use.
These tests pin what a user relies on when comparing runs:
  - the same seed gives the same bits;
  - values lie in the 8-bit range;
  - the masks have the stated geometry (the loss area B is a quarter of the
    area L, with support margins);
  - each batch has the stated sizes.
"""
import numpy as np
import pytest

from paper_2204_14194_gb300 import workloads as W


def test_same_seed_same_bits_and_8bit_range():
    a, b = W.tiled_image(200, 130, 5), W.tiled_image(200, 130, 5)
    assert a.dtype == np.float64 and a.shape == (200, 130)
    assert np.array_equal(a, b)
    assert not np.array_equal(a, W.tiled_image(200, 130, 6))
    assert a.min() >= 0.0 and a.max() <= 255.0
    assert np.array_equal(W.patch(32, 9), W.patch(32, 9))
    # a tile is a function of its own stream: a bigger canvas keeps the first tile
    assert np.array_equal(W.tiled_image(64, 64, 5), W.tiled_image(128, 192, 5)[:64, :64])


@pytest.mark.parametrize("M,N", [(16, 16), (32, 32), (64, 64), (16, 32)])
def test_mask_geometry(M, N):
    c = W.centred_support(M, N)
    assert c.dtype == np.uint8 and int((c == 0).sum()) == M * N // 4
    rows, cols = np.nonzero(c == 0)
    assert (rows.min(), rows.max(), cols.min(), cols.max()) == (M // 4, M // 4 + M // 2 - 1,
                                                                N // 4, N // 4 + N // 2 - 1)
    rng = np.random.default_rng(0)
    for _ in range(20):
        r = W.rect_support(M, N, rng)
        rows, cols = np.nonzero(r == 0)
        assert int((r == 0).sum()) == M * N // 4
        assert rows.max() - rows.min() + 1 == M // 2 and cols.max() - cols.min() + 1 == N // 2
        assert rows.min() >= M // 8 and M - 1 - rows.max() >= M // 8
        assert cols.min() >= N // 8 and N - 1 - cols.max() >= N // 8
        h = W.holes_support(M, N, rng)
        assert int((h == 0).sum()) == M * N // 4
        # holes fill whole cells of the 4-aligned grid
        cells = (h == 0).reshape(M // 4, 4, N // 4, 4).sum(axis=(1, 3))
        assert set(np.unique(cells)) <= {0, 16}


def test_centred_support3_reduces_to_2d():
    assert np.array_equal(W.centred_support3(16, 16, 1)[0], W.centred_support(16, 16))
    s = W.centred_support3(16, 16, 4)
    lost = [(s[t] == 0).any() for t in range(4)]
    assert lost == [False, True, True, False]


def test_gaussian_atoms_unit_norm_and_seeded():
    d = W.gaussian_dictionary(64, 8, 8, 3)
    assert d.shape == (64, 8, 8)
    np.testing.assert_allclose(np.sqrt((d.reshape(64, -1) ** 2).sum(axis=1)), 1.0, rtol=1e-14)
    assert np.array_equal(d, W.gaussian_dictionary(64, 8, 8, 3))


def test_batch_shapes():
    w1 = W.config1()
    assert (w1.B, w1.M, w1.N, w1.K, w1.iterations) == (1, 32, 32, 2048, 100)
    w2 = W.config2(64)
    assert w2.samples.shape == (64, 32, 32) and w2.support.shape == (32, 32)
    # the blocks are the image's 32x32 areas at the stated corners
    img = W.tiled_image(512, 512, 2)
    t, l = w2.meta["corners"][5]
    assert np.array_equal(w2.samples[5], img[t:t + 32, l:l + 32])
    mixed = W.config4(30)
    assert [w.M for w in mixed] == [16, 32, 64] and sum(w.B for w in mixed) == 30
    for w in mixed:
        assert w.support.shape == (w.B, w.M, w.N) and w.K == 2 * w.M * w.N
        assert w.iters_per_block.min() >= 50 and w.iters_per_block.max() <= 500
