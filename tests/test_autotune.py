"""Host logic of the tile/schedule autotuner (no GPU): schedules partition
the views, the fastest candidate wins, plans are cached by shape."""
import numpy as np
import pytest

from paper_2510_03312_gb300 import autotune as A
from paper_2510_03312_gb300 import scenes as S


def _batch(n_views=40, seed=0):
    rng = np.random.default_rng(seed)
    scenes = [S.make_scene(10 + k, N, P) for k, (N, P) in enumerate([(3, 50), (6, 20), (7, 30)])]
    views = []
    for j in range(n_views):
        R, t = S.look_at(8.0 * np.array([0.0, 0.0, -1.0]))
        views.append(S.make_view(R, t, int(rng.integers(16, 300)), int(rng.integers(16, 200)),
                                 scene_id=int(rng.integers(0, 3))))
    return scenes, views, S.RasterConfig()


@pytest.mark.parametrize("name", list(A.SCHEDULES))
def test_schedules_partition_the_views(name):
    scenes, views, _ = _batch()
    groups = A.SCHEDULES[name](scenes, views)
    flat = sorted(i for g in groups for i in g)
    assert flat == list(range(len(views)))
    assert all(0 < len(g) <= A.MAX_VIEWS for g in groups)


def test_one_launch_chunks_at_the_view_limit():
    scenes, views, _ = _batch(n_views=600)
    groups = A.one_launch(scenes, views)
    assert [len(g) for g in groups] == [256, 256, 88]


def test_per_scene_groups_hold_one_scene():
    scenes, views, _ = _batch()
    for g in A.per_scene(scenes, views):
        assert len({views[i].scene_id for i in g}) == 1


def test_heavy_first_orders_by_expected_work():
    scenes, views, _ = _batch()
    (g,) = A.one_launch_heavy_first(scenes, views)
    cost = [views[i].width * views[i].height * np.log2(2 + scenes[views[i].scene_id].P) for i in g]
    assert all(a >= b for a, b in zip(cost, cost[1:]))


def test_tune_picks_the_fastest_and_records_every_candidate():
    scenes, views, cfg = _batch()
    calls = []

    def fake(tile, groups, form):
        calls.append((tile, len(groups), form))
        # fastest: 16x32 tiles in one persistent launch
        return 1.0 + 0.1 * len(groups) + (0.0 if tile == (16, 32) else 0.5) + (0.0 if form == "persistent" else 0.05)

    plan = A.tune(scenes, views, cfg, fake)
    assert plan.tile == (16, 32) and plan.schedule == "one_launch" and plan.form == "persistent"
    assert len(plan.table) == len(A.TILES) * len(A.SCHEDULES) * len(A.FORMS) == len(calls)
    assert plan.ms == min(plan.table.values())
    assert {"16x32/one_launch/persistent", "16x32/one_launch/grid", "16x32/one_launch/split"} <= set(plan.table)
    c = plan.config(cfg)
    assert (c.tile_w, c.tile_h, c.persistent, c.split_lists) == (16, 32, True, False)


def test_tune_ties_go_to_the_first_candidate():
    scenes, views, cfg = _batch()
    plan = A.tune(scenes, views, cfg, lambda tile, groups, form: 2.0)
    assert plan.tile == A.TILES[0] and plan.schedule == next(iter(A.SCHEDULES))
    assert plan.form == A.FORMS[0]


def test_plan_cache_hits_skip_measurement_and_persist(tmp_path):
    scenes, views, cfg = _batch()
    path = str(tmp_path / "plans.json")
    cache = A.PlanCache(path)
    p1 = A.tune(scenes, views, cfg, lambda t, g, f: float(t[0] * t[1]) + len(g) - 0.5 * (f == "split"), cache=cache)

    def boom(tile, groups, form):
        raise AssertionError("measured despite a cached plan")

    p2 = A.tune(scenes, views, cfg, boom, cache=A.PlanCache(path))
    assert (p2.tile, p2.schedule, p2.groups, p2.form) == (p1.tile, p1.schedule, p1.groups, p1.form)
    assert p2.form == "split"


def test_signature_follows_shapes_only():
    scenes, views, cfg = _batch()
    k = A.signature(scenes, views, cfg, A.TILES, A.SCHEDULES)
    assert k == A.signature(scenes, list(views), cfg, A.TILES, A.SCHEDULES)
    v2 = list(views)
    v2[0] = S.make_view(views[0].R, views[0].t, views[0].width + 1, views[0].height, scene_id=views[0].scene_id)
    assert k != A.signature(scenes, v2, cfg, A.TILES, A.SCHEDULES)
    s2 = [scenes[0].subset(np.arange(10))] + scenes[1:]
    assert k != A.signature(s2, views, cfg, A.TILES, A.SCHEDULES)
