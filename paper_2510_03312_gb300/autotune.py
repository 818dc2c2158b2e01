"""Tile shape and batch schedule selection for a batch of render jobs.

A plan is a tile shape for the blend (one of the shapes the kernels are
built for), a launch form of the blend kernels (one CTA per tile or 8x8
block, a persistent grid that takes them from a counter, or the grid with
long lists split into segments) and a schedule: a partition of the views into launches, each launch one problem
over the scenes its views use.  Candidates are timed on
the device by replaying a captured CUDA graph of the whole forward+backward
step, and the fastest is kept, cached under a signature of the batch's
shapes.

None of these choices changes the method's arithmetic: every pixel composites the
same records in the same (depth, index) order under any tile shape, and a
scene's gradient is the sum over all of its views whichever launch renders
them (Batch accumulates into one buffer per scene).  Only the float
summation order of gradients differs.
"""
from __future__ import annotations

import hashlib
import json
import math
import os
from dataclasses import dataclass, field

TILES = ((8, 8), (16, 16), (16, 32), (32, 32))
FORMS = ("grid", "persistent", "split")  # launch forms of the blend kernels
MAX_VIEWS = 256  # views per problem accepted by the C-ABI


def _chunks(idx, n=MAX_VIEWS):
    return [idx[i:i + n] for i in range(0, len(idx), n)] or [[]]


def one_launch(scenes, views):
    """All views in one problem, in the given order."""
    return _chunks(list(range(len(views))))


def one_launch_heavy_first(scenes, views):
    """All views in one problem, largest expected work first, so that the
    tiles of the heaviest views are dispatched first (shorter tail)."""
    cost = [v.width * v.height * math.log2(2 + scenes[v.scene_id].P) for v in views]
    order = sorted(range(len(views)), key=lambda i: (-cost[i], i))
    return _chunks(order)


def per_scene(scenes, views):
    """One problem per scene (its views in order)."""
    out = []
    for s in range(len(scenes)):
        g = [i for i, v in enumerate(views) if v.scene_id == s]
        out.extend(_chunks(g) if g else [])
    return out


def per_view(scenes, views):
    """One problem per view: the plain one-view-per-launch form."""
    return [[i] for i in range(len(views))]


SCHEDULES = {
    "one_launch": one_launch,
    "one_launch_heavy_first": one_launch_heavy_first,
    "per_scene": per_scene,
    "per_view": per_view,
}


def signature(scenes, views, cfg, tiles, schedules, forms=FORMS) -> str:
    """Key of a batch's shapes: scene (N, rotation mode, P), view (W, H,
    scene), the config constants that change the work, and the candidates."""
    d = {
        "scenes": [(int(s.N), int(s.rot_mode), int(s.P)) for s in scenes],
        "views": [(int(v.width), int(v.height), int(v.scene_id)) for v in views],
        "cfg": [float(cfg.alpha_min), float(cfg.alpha_max), float(cfg.T_min), float(cfg.eps2d),
                float(cfg.near), bool(cfg.tight_cut)],
        "tiles": [list(t) for t in tiles],
        "schedules": sorted(schedules),
        "forms": [str(f) for f in forms],
    }
    return hashlib.sha256(json.dumps(d, sort_keys=True).encode()).hexdigest()[:24]


@dataclass
class Plan:
    tile: tuple
    schedule: str
    groups: list
    ms: float
    table: dict = field(default_factory=dict)  # "WxH/schedule/form" -> ms
    form: str = "grid"

    def config(self, cfg):
        """``cfg`` with this plan's tile shape and launch form."""
        from dataclasses import replace
        return replace(cfg, tile_w=int(self.tile[0]), tile_h=int(self.tile[1]), **form_fields(self.form))

    def to_json(self):
        return {"tile": list(self.tile), "schedule": self.schedule, "groups": self.groups, "ms": self.ms,
                "table": self.table, "form": self.form}

    @classmethod
    def from_json(cls, d):
        return cls(tuple(d["tile"]), d["schedule"], [list(g) for g in d["groups"]], float(d["ms"]),
                   dict(d.get("table", {})), str(d.get("form", "grid")))


def form_fields(form: str) -> dict:
    """RasterConfig fields of a launch form."""
    if form not in FORMS:
        raise ValueError(f"unknown launch form {form!r}")
    return {"persistent": form == "persistent", "split_lists": form == "split"}


class PlanCache:
    """Plans by signature, optionally persisted as a JSON file."""

    def __init__(self, path: str | None = None):
        self.path = path
        self.plans = {}
        if path and os.path.exists(path):
            with open(path) as f:
                self.plans = {k: Plan.from_json(v) for k, v in json.load(f).items()}

    def get(self, key):
        return self.plans.get(key)

    def put(self, key, plan):
        self.plans[key] = plan
        if self.path:
            tmp = self.path + ".tmp"
            with open(tmp, "w") as f:
                json.dump({k: p.to_json() for k, p in self.plans.items()}, f)
            os.replace(tmp, self.path)


def tune(scenes, views, cfg, measure, tiles=TILES, schedules=None, cache: PlanCache | None = None,
         forms=FORMS) -> Plan:
    """Times every (tile, schedule, launch form) candidate with
    ``measure(tile, groups, form)`` (milliseconds per forward+backward step)
    and returns the fastest plan.  ``scenes`` need ``N``,
    ``rot_mode`` and ``P``; ``views`` need ``width``, ``height`` and
    ``scene_id``.  Ties go to the earlier candidate."""
    schedules = SCHEDULES if schedules is None else schedules
    key = signature(scenes, views, cfg, tiles, schedules, forms)
    if cache is not None:
        hit = cache.get(key)
        if hit is not None:
            return hit
    best, table = None, {}
    for tile in tiles:
        for name, make in schedules.items():
            groups = make(scenes, views)
            for form in forms:
                ms = float(measure(tuple(tile), groups, form))
                table[f"{tile[0]}x{tile[1]}/{name}/{form}"] = round(ms, 4)
                if best is None or ms < best.ms:
                    best = Plan(tuple(tile), name, groups, ms, form=form)
    if best is None:
        raise ValueError("no candidates")
    best.table = table
    if cache is not None:
        cache.put(key, best)
    return best


def device_measure(scenes, views, cfg, device="cuda", steps=3, warmup=1):
    """A ``measure`` for ``tune``: builds the schedule's Batch with the tile
    shape, sizes its capacities, captures the step in a CUDA graph and times
    ``steps`` replays with CUDA events (after ``warmup``).  ``scenes`` are
    DeviceScenes.  dL/dimage is a constant (its value does not change the
    work)."""
    from dataclasses import replace

    import torch

    from .raster import Batch

    def measure(tile, groups, form="grid"):
        c = replace(cfg, tile_w=int(tile[0]), tile_h=int(tile[1]), **form_fields(form))
        b = Batch(scenes, views, c, groups, device=device)
        b.size()
        dls = b.dL_like(1e-6)
        g = b.capture(dls)
        for _ in range(warmup):
            g.replay()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(steps):
            g.replay()
        e1.record()
        torch.cuda.synchronize()
        bad = [st.status for st in b.status() if st.status != 0]
        if bad:
            raise RuntimeError(f"device status {bad} while tuning")
        ms = e0.elapsed_time(e1) / steps
        del g, b
        torch.cuda.empty_cache()
        return ms

    return measure
