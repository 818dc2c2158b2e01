"""Property tests of the workspace layout arithmetic (host code of the
C-ABI, no GPU): over random problems the size is positive, a multiple of
256, never below the bytes the per-record, per-instance and per-pixel
arrays need, and non-decreasing in the instance capacity, the primitive
count and the image size; every invalid field gives 0."""
import pytest

hyp = pytest.importorskip("hypothesis")
st = pytest.importorskip("hypothesis.strategies")

from paper_2510_03312_gb300 import build as B  # noqa: E402
from paper_2510_03312_gb300 import scenes as S  # noqa: E402
from paper_2510_03312_gb300 import ubs as U  # noqa: E402

TILES = [(8, 8), (16, 16), (16, 32), (32, 32)]
FAKE = 0x10000  # plane pointers are never dereferenced by the size query


@pytest.fixture(scope="module", autouse=True)
def lib():
    B.build()
    return U.load()


def problem(Ns, Ps, sizes, tile, cap):
    scs = (U.ubs_scene * len(Ns))()
    for i, (N, P) in enumerate(zip(Ns, Ps)):
        scs[i].N, scs[i].rot_mode, scs[i].P = N, 0, P
        for name in S.PLANE_ORDER:
            setattr(scs[i], name, FAKE)
    vs = (U.ubs_view * len(sizes))()
    for i, (w, h, sid) in enumerate(sizes):
        vs[i].fx = vs[i].fy = 500.0
        vs[i].width, vs[i].height, vs[i].scene_id = w, h, sid % len(Ns)
    pr = U.ubs_problem()
    pr.scenes, pr.n_scenes, pr.views, pr.n_views = scs, len(Ns), vs, len(sizes)
    pr.cfg.tile_w, pr.cfg.tile_h = tile
    pr.cfg.alpha_min, pr.cfg.alpha_max, pr.cfg.T_min = 1 / 255, 0.99, 1e-4
    pr.cfg.eps2d, pr.cfg.near_plane, pr.cfg.jac_clip = 0.3, 0.2, 1.3
    pr.instance_capacity = cap
    return pr, (scs, vs)


scenes_st = st.lists(st.tuples(st.sampled_from([3, 4, 6, 7]), st.integers(1, 3_000_000)), min_size=1, max_size=4)
views_st = st.lists(st.tuples(st.integers(1, 4096), st.integers(1, 4096), st.integers(0, 3)), min_size=1, max_size=6)
SETTINGS = dict(max_examples=60, deadline=None)


@hyp.settings(**SETTINGS)
@hyp.given(scenes=scenes_st, views=views_st, tile=st.sampled_from(TILES), cap=st.integers(0, 50_000_000))
def test_size_bounds_and_alignment(scenes, views, tile, cap):
    Ns, Ps = [n for n, _ in scenes], [p for _, p in scenes]
    pr, keep = problem(Ns, Ps, views, tile, cap)
    n = U.ubs_workspace_size(pr)
    assert n > 0 and n % 256 == 0
    R = sum(Ps[sid % len(Ns)] for _, _, sid in views)
    npix = sum(w * h for w, h, _ in views)
    # records (48 B) and their screen gradients (48 B), four u32 instance
    # arrays of the capacity, three u32 pixel arrays
    assert n >= 96 * R + 16 * max(cap, 1) + 12 * npix


@hyp.settings(**SETTINGS)
@hyp.given(N=st.sampled_from([3, 4, 6, 7]), P=st.integers(1, 2_000_000), dP=st.integers(0, 100_000),
           w=st.integers(1, 2048), h=st.integers(1, 2048), dw=st.integers(0, 512),
           tile=st.sampled_from(TILES), cap=st.integers(0, 10_000_000), dcap=st.integers(0, 10_000_000))
def test_size_is_monotone(N, P, dP, w, h, dw, tile, cap, dcap):
    def size(P_, w_, cap_):
        pr, keep = problem([N], [P_], [(w_, h, 0)], tile, cap_)
        return U.ubs_workspace_size(pr)
    base = size(P, w, cap)
    assert size(P, w, cap + dcap) >= base
    assert size(P + dP, w, cap) >= base
    assert size(P, min(w + dw, 16384), cap) >= base


@hyp.settings(**SETTINGS)
@hyp.given(field=st.sampled_from(["N", "P", "tile", "width", "height", "fx", "scene_id", "cap", "alpha_max", "views"]),
           bad=st.integers(0, 3))
def test_invalid_fields_give_zero(field, bad):
    pr, (scs, vs) = problem([6], [1000], [(100, 80, 0)], (16, 16), 5000)
    if field == "N":
        scs[0].N = [0, 2, 5, 8][bad]
    elif field == "P":
        scs[0].P = [-1, -1000, -(1 << 40), -7][bad]
    elif field == "tile":
        pr.cfg.tile_w, pr.cfg.tile_h = [(12, 12), (16, 8), (64, 64), (0, 0)][bad]
    elif field == "width":
        vs[0].width = [0, -1, 16385, 1 << 20][bad]
    elif field == "height":
        vs[0].height = [0, -5, 16385, 1 << 30][bad]
    elif field == "fx":
        vs[0].fx = [0.0, -1.0, float("nan"), -float("inf")][bad]
    elif field == "scene_id":
        vs[0].scene_id = [1, -1, 64, 1000][bad]
    elif field == "cap":
        pr.instance_capacity = [-1, 1 << 31, 1 << 40, -(1 << 33)][bad]
    elif field == "alpha_max":
        pr.cfg.alpha_max = [0.0, -0.5, 1.5, float("nan")][bad]
    elif field == "views":
        pr.n_views = [0, -1, 257, 1000][bad]
    assert U.ubs_workspace_size(pr) == 0
