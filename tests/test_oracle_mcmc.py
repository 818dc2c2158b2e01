"""Pins of the MCMC relocation reference (Sec. 4.5 primitive management):
the opacity rule against the composited density it preserves, the sampling
distribution, and hand-built cases."""
import numpy as np
import pytest

from oracle import mcmc64 as M


@pytest.mark.parametrize("N", [1, 2, 3, 7, 40])
def test_cloned_opacity_composes_back_to_the_source(N):
    """N stacked copies of alpha o' let through (1 - o')^N = 1 - o."""
    o = np.array([0.006, 0.1, 0.5, 0.9, 0.999])
    op = 1.0 - (1.0 - o) ** (1.0 / N)
    np.testing.assert_allclose(1.0 - (1.0 - op) ** N, o, rtol=1e-12)


def _scene(P, K=5, seed=0, dead_frac=0.2):
    rng = np.random.default_rng(seed)
    act = rng.standard_normal((K, P))
    o = 1.0 / (1.0 + np.exp(-rng.standard_normal(P)))
    o[rng.random(P) < dead_frac] = rng.uniform(0.0, 0.005, size=None)
    act[2] = o.astype(np.float32)
    raw = act.copy()
    raw[2] = np.log(act[2] / (1 - act[2]))
    m = rng.standard_normal((K, P))
    v = rng.random((K, P))
    rand = rng.integers(0, 2 ** 63, size=P, dtype=np.uint64) * np.uint64(2) + rng.integers(0, 2, size=P,
                                                                                            dtype=np.uint64)
    return act, raw, m, v, rand


def test_hand_built_draws():
    o = np.array([0.5, 0.001, 0.25, 0.0, 0.25, 0.003], dtype=np.float32)
    act = np.stack([np.arange(6, dtype=np.float64), o.astype(np.float64)])
    raw = act.copy()
    m = np.ones((2, 6))
    v = np.ones((2, 6))
    # weights 2^23, 0, 2^22, 0, 2^22, 0: inclusive cumulative 2^23, 2^23, 3*2^22, 3*2^22, 2^24, 2^24
    rand = np.array([0, 0, 0, 2 ** 23, 0, 2 ** 24 - 1 + 5 * 2 ** 24], dtype=np.uint64)
    a, r, mm, vv, src = M.relocate(act, raw, m, v, 1, rand)
    assert src.tolist() == [-1, 0, -1, 2, -1, 4]
    want = [1 - 0.5 ** 0.5, 1 - 0.75 ** 0.5]
    np.testing.assert_allclose(a[1, [0, 1]], want[0], rtol=1e-6)  # source 0 and its copy
    np.testing.assert_allclose(a[1, [2, 3, 4, 5]], want[1], rtol=1e-6)
    assert a[0].tolist() == [0, 0, 2, 2, 4, 4]  # other rows copied from the source
    assert (mm == 0).all() and (vv == 0).all()  # every slot is a source or a copy here
    np.testing.assert_allclose(1 / (1 + np.exp(-r[1])), a[1], rtol=1e-12)


def test_sources_follow_the_weights_and_are_alive():
    rng = np.random.default_rng(1)
    P = 20000
    o = np.zeros(P, dtype=np.float32)
    live = np.array([0, 1, 2, 3, 4])
    o[live] = np.array([0.9, 0.5, 0.25, 0.05, 0.006], dtype=np.float32)
    act = np.stack([o.astype(np.float64)])
    rand = rng.integers(0, 2 ** 63, size=P, dtype=np.uint64)
    _, _, _, _, src = M.relocate(act, act.copy(), np.zeros_like(act), np.zeros_like(act), 0, rand)
    assert (src[live] == -1).all()
    drawn = src[src >= 0]
    assert set(np.unique(drawn)) <= set(live.tolist())
    counts = np.bincount(drawn, minlength=5)[:5]
    w = np.floor(o[live] * 2 ** 24)
    expect = w / w.sum() * drawn.size
    chi2 = ((counts - expect) ** 2 / expect).sum()
    assert chi2 < 25.0  # 4 degrees of freedom: p ~ 5e-5


def test_group_density_is_conserved():
    act, raw, m, v, rand = _scene(3000, seed=2)
    a, r, mm, vv, src = M.relocate(act, raw, m, v, 2, rand)
    for s in np.unique(src[src >= 0]):
        group = np.concatenate([[s], np.flatnonzero(src == s)])
        assert 1 - np.prod(1 - a[2, group]) == pytest.approx(act[2, s], rel=1e-10)
        assert (mm[:, group] == 0).all()
    untouched = (src < 0) & (np.bincount(src[src >= 0], minlength=act.shape[1]) == 0)
    assert np.array_equal(a[:, untouched], act[:, untouched])
    assert np.array_equal(mm[:, untouched], m[:, untouched])


def test_nothing_to_do():
    act, raw, m, v, rand = _scene(100, seed=3, dead_frac=0.0)
    act[2] = np.maximum(act[2], 0.01)
    a, r, mm, vv, src = M.relocate(act, raw, m, v, 2, rand)
    assert (src == -1).all() and np.array_equal(a, act)
    act[2] = 0.001  # nothing alive: no source to draw from
    a, r, mm, vv, src = M.relocate(act, raw, m, v, 2, rand)
    assert (src == -1).all() and np.array_equal(a, act)
