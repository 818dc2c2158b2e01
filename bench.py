"""Benchmark of the UBS differentiable rasterizer on GB300.

Workload (one step = one pass of the whole path over one batch): the static
N=3 scene of 1,000,000 primitives (64-cluster Gaussian mixture in [-5,5]^3)
seen by one 1600x1060 camera on a radius-8 sphere: preprocess -> bin_sort ->
render_fwd -> render_bwd (blend backward + parameter backward), dL/dimage of
an L1 loss against a uniform-random target precomputed once.  Metric:
forward+backward megapixels per second (and views per second).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Under torchrun (N > 1) every rank renders its own camera of the same scene
(weak scaling, no collective on the data path); the elapsed time is the
maximum over ranks.  ``--impl reference`` times the CPU oracle (float64
reference renderer) on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "fwd+bwd megapixels/sec and views/sec at 1 GB300, batched vs per-view; % of roofline"
L2_BYTES = 129 * 2 ** 20

# per-pair algorithmic work of the blend kernels: FP32 lane operations and,
# separately, MUFU operations (exp, reciprocal), whose pipe is 8x narrower
FWD_FP32_PER_PAIR, FWD_MUFU_PER_PAIR = 16, 2
BWD_FP32_PER_PAIR, BWD_MUFU_PER_PAIR = 45, 3
# training step: the image loss reads the image and the target and writes
# dL/dimage (12 B per pixel and channel); its work is the two separable 11-tap
# passes of the five SSIM window statistics (110 FMA) and of the three partial
# derivatives (66 FMA) plus ~30 operations of the map and its derivatives.
# Adam reads raw, grad, m, v and writes raw, m, v and the activated value.
LOSS_BYTES_PER_PC, LOSS_FP32_PER_PC = 12, 206
ADAM_BYTES_PER_PARAM = 32


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--primitives", type=int, default=1_000_000)
    ap.add_argument("--no-batched", action="store_true", help="skip the batched vs per-view comparison")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(x, dist, device):
    """The maximum of a per-rank float over all ranks (x itself without a
    process group): the job's elapsed time is its slowest rank's."""
    if dist is None:
        return float(x)
    import torch

    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world, steps, units_per_rank_step, total_ms):
    """Whole-job throughput: the units every rank processed in ``steps``
    steps over the (max-over-ranks) elapsed milliseconds."""
    return world * steps * units_per_rank_step / (total_ms / 1e3)


def config_of(wl, world):
    """The workload-identifying keys of the bench line, shared by both arms."""
    v = wl.views[0]
    return {"workload": wl.name, "primitives": wl.scenes[0].P, "views": len(wl.views), "width": v.width,
            "height": v.height, "tile": f"{wl.cfg.tile_w}x{wl.cfg.tile_h}", "parallelism": f"replicas x{world}"}


def workload(rank, P):
    from paper_2510_03312_gb300 import scenes as S

    wl = S.workload_static_large(P=P)
    if rank > 0:  # weak scaling: another camera of the same scene per rank
        rng = np.random.default_rng(1000 + rank)
        wl.views = S.sphere_views(rng, 1, 8.0, 1600, 1060)
    return wl


# ----------------------------------------------------------------------------
# clocks during the timed region
# ----------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index, self.proc, self.lines = index, None, []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
            except ValueError:
                continue
        if not rows:
            return None
        sm = sorted(r[0] for r in rows)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i, v in enumerate(r[2]) if v.lower().startswith("active")})
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": max(r[1] for r in rows), "reasons": reasons,
                "samples": len(rows)}


# ----------------------------------------------------------------------------
# our implementation
# ----------------------------------------------------------------------------

def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def alu_peak_tops(n_sm, sm_mhz):
    """FP32 lane-operation peak (128 FP32 lanes per SM per clock).  The MUFU
    pipe (16 per SM per clock) allows 8 FP32 operations per MUFU operation;
    for the backward blend (45 FP32 : 3 MUFU) and the forward blend (16 : 2)
    the FP32 pipe is the binding one or tied, so the ALU peak is the FP32
    lane rate."""
    return n_sm * 128 * sm_mhz * 1e6 / 1e12


def source_sha(path):
    return hashlib.sha256(open(path, "rb").read()).hexdigest()[:16]


def traffic_record(kernel):
    """DRAM bytes per launch of ``kernel`` from a committed ncu summary: a
    line ``traffic: kernel=K source=F source_sha=S dram_bytes_per_launch=B``
    in a profiles/*.md file.  None when no summary has one, or when the
    kernel's source file changed since it was captured (sha mismatch)."""
    d = os.path.join(ROOT, "profiles")
    if not os.path.isdir(d):
        return None
    for name in sorted(os.listdir(d)):
        if not name.endswith(".md"):
            continue
        for line in open(os.path.join(d, name)):
            line = line.strip().strip("`")
            if not line.startswith("traffic:"):
                continue
            kv = dict(x.split("=", 1) for x in line[len("traffic:"):].split() if "=" in x)
            if kv.get("kernel") != kernel:
                continue
            src = os.path.join(ROOT, "paper_2510_03312_gb300", "csrc", kv.get("source", ""))
            if not os.path.exists(src) or source_sha(src) != kv.get("source_sha"):
                return None
            return int(kv["dram_bytes_per_launch"])
    return None


def kernels_per_step(r):
    """Kernels of this library launched by one step (memsets excluded)."""
    V, S = len(r.views), len(r.scenes)
    NT = sum(((v.width + r.cfg.tile_w - 1) // r.cfg.tile_w) * ((v.height + r.cfg.tile_h - 1) // r.cfg.tile_h)
             for v in r.views)
    upload = (V + 15) // 16
    pre = upload + S
    # the count, the scan (two kernels, three over more than 2048 x 1024
    # tiles; the second also makes the tile order), the scatter, the
    # per-tile sort and the merge of long lists
    R = sum(r.scenes[v.scene_id].P for v in r.views)
    sort = 0 if R == 0 else (1 + 2 + (1 if (NT + 1023) // 1024 > 2048 else 0) + 3)
    # forward blend; zeroing of the visible records' gradient sums, backward
    # blend; parameter backward per scene
    return pre + sort + 1 + 2 + S


def step_rooflines(stage_ms, names, params_bytes, R, instances, NT, pairs, pk, n_sm):
    """Every stage against its bound, with a fixed algorithmic work per
    unit: preprocess reads the parameters once and writes 44 B per record;
    the sort is charged the bytes of an LSD sort of (tile, depth) keys, a
    reference count the binning itself does not move (12 B per instance to
    emit the keys, 24 B per instance per pass, ceil((tile bits + 32) / 8)
    passes, and 8 B per instance for the ranges);
    the forward blend costs 16 FP32 + 2 MUFU operations per pair, the
    backward blend 45 FP32 + 3 MUFU; the parameter backward reads the
    parameters and 40 B of screen gradients per record and writes the
    parameter gradients.  t_roof is the time at the peak of the binding
    unit; the path fraction is sum(t_roof) / measured step time."""
    hbm = pk["hbm_gbs"] * 1e9
    mhz = pk.get("sm_max_mhz", 2070.0)
    fp32 = n_sm * 128 * mhz * 1e6
    mufu = n_sm * 16 * mhz * 1e6
    tile_bits = max(1, math.ceil(math.log2(max(NT, 2))))
    passes = math.ceil((tile_bits + 32) / 8)
    work = {
        "preprocess": ("hbm", params_bytes + 44 * R),
        "bin_sort": ("hbm", instances * (12 + 24 * passes + 8)),
        "render_fwd": ("alu", (16 * pairs, 2 * pairs)),
        "render_bwd_blend": ("alu", (45 * pairs, 3 * pairs)),
        "render_bwd_params": ("hbm", 2 * params_bytes + 40 * R),
    }
    out, t_roof = {}, 0.0
    for n, ms in zip(names, stage_ms):
        bound, w = work[n]
        t = ms * 1e-3
        if bound == "hbm":
            tr = w / hbm
            out[n] = {"bound": "hbm", "bytes": int(w), "achieved": round(w / t / 1e9, 1), "peak": pk["hbm_gbs"],
                      "unit": "GB/s", "frac": round(tr / t, 4)}
        else:
            tr = max(w[0] / fp32, w[1] / mufu)
            out[n] = {"bound": "alu", "fp32_ops": int(w[0]), "mufu_ops": int(w[1]),
                      "achieved": round(w[0] / t / 1e12, 3), "peak": round(fp32 / 1e12, 2), "unit": "T lane-op/s",
                      "frac": round(tr / t, 4)}
        out[n]["ms"] = round(float(ms), 4)
        t_roof += tr
    total = float(sum(stage_ms)) * 1e-3
    path = {"t_roof_ms": round(t_roof * 1e3, 4), "t_ms": round(total * 1e3, 4), "frac": round(t_roof / total, 4),
            "sort_passes_counted": passes}
    return out, path


def bench_ours(args, rank, world, local):
    import torch

    from paper_2510_03312_gb300 import build as B
    from paper_2510_03312_gb300 import raster
    from paper_2510_03312_gb300 import scenes as S

    B.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    wl = workload(rank, args.primitives)
    sc = wl.scenes[0]
    ds = raster.DeviceScene.from_scene(sc, device=dev)
    r = raster.Rasterizer([ds], wl.views, wl.cfg, device=dev)
    img = r.forward(check=True)  # sizes the instance capacity (one sync)
    st = r.status()
    # dL/dimage of mean |image - target|
    target = r.pack(S.l1_target(1, wl.views))
    dL = (torch.sign(img - target) / img.numel()).contiguous()
    torch.cuda.synchronize()
    # pair counts (diagnostic kernel variant, outside the timed region): pairs
    # with r < 1 met before each pixel terminates (tile-free), and the
    # entries the forward's warps evaluate
    cnt = raster.count_pairs([ds], wl.views, wl.cfg, device=dev)
    pairs = int(cnt["pairs"].sum().item())
    visited = int(cnt["visited"].sum().item())
    del cnt
    flush = torch.empty(2 * L2_BYTES, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()

    def ev():
        return torch.cuda.Event(enable_timing=True)

    names = ["preprocess", "bin_sort", "render_fwd", "render_bwd_blend", "render_bwd_params"]

    def step(evs):
        evs[0].record(stream)
        r.preprocess()
        evs[1].record(stream)
        r.bin_sort()
        evs[2].record(stream)
        r.render_fwd()
        evs[3].record(stream)
        r.render_bwd_blend(dL)
        evs[4].record(stream)
        r.render_bwd_params()
        evs[5].record(stream)

    for i in range(args.warmup):
        flush.fill_(i & 0xFF)
        step([ev() for _ in range(6)])
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    all_evs = []
    wall0 = time.perf_counter()
    for i in range(args.steps):
        flush.fill_((i + 7) & 0xFF)
        evs = [ev() for _ in range(6)]
        step(evs)
        all_evs.append(evs)
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clk = clocks.stop()
    stage = np.array([[e[k].elapsed_time(e[k + 1]) for k in range(5)] for e in all_evs])  # ms
    step_ms = stage.sum(1)
    total_ms = float(step_ms.sum())
    total_ms = max_over_ranks(total_ms, dist, dev)
    mp_per_view = wl.views[0].width * wl.views[0].height / 1e6
    value = job_throughput(world, args.steps, mp_per_view, total_ms)
    ms_per_step = total_ms / args.steps
    # roofline of the dominant kernel
    stage_mean = stage.mean(0)
    dom = int(np.argmax(stage_mean))
    pk, pk_src = peaks()
    sm_mhz = (clk or {}).get("sm_mhz") or pk.get("sm_max_mhz", 2070.0)
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    ops_per_pair = {"render_fwd": FWD_FP32_PER_PAIR, "render_bwd_blend": BWD_FP32_PER_PAIR}
    roof = {}
    if names[dom] in ops_per_pair:
        ach = ops_per_pair[names[dom]] * pairs / (stage_mean[dom] * 1e-3) / 1e12
        peak = alu_peak_tops(n_sm, pk.get("sm_max_mhz", 2070.0))
        kern = "render_bwd_blend" if names[dom] == "render_bwd_blend" else "render_fwd"
        roof = {"bound": "alu", "kernel": kern, "achieved": round(ach, 3), "peak": round(peak, 2),
                "unit": "T lane-op/s", "frac": round(ach / peak, 4), "traffic": traffic_record(kern),
                "work": f"{ops_per_pair[names[dom]]} FP32 lane-ops per pair x {pairs} pairs",
                "peak_source": f"{n_sm} SMs x 128 FP32 lanes x {pk.get('sm_max_mhz', 2070.0):.0f} MHz "
                               f"(clock of {pk_src} peaks file)"}
    else:
        nbytes = {"preprocess": 60 * sc.P + 44 * sc.P}.get(names[dom])
        if nbytes:
            ach = nbytes / (stage_mean[dom] * 1e-3) / 1e9
            roof = {"bound": "hbm", "kernel": names[dom], "achieved": round(ach, 1),
                    "peak": pk["hbm_gbs"], "unit": "GB/s", "frac": round(ach / pk["hbm_gbs"], 4),
                    "traffic": traffic_record(names[dom])}
    params_bytes = ds.params.numel() * 4
    steps_roof, path_roof = step_rooflines(stage_mean, names, params_bytes, sc.P * len(wl.views),
                                           int(st.instances), r.n_tiles(), pairs, pk, n_sm)
    # the same step replayed as one captured CUDA graph (L2 flushed between steps)
    graph = r.capture(dL)
    for _ in range(3):
        graph.replay()
    torch.cuda.synchronize()
    g_ms = []
    for i in range(args.steps):
        flush.fill_((i + 3) & 0xFF)
        e0, e1 = ev(), ev()
        e0.record(stream)
        graph.replay()
        e1.record(stream)
        g_ms.append((e0, e1))
    torch.cuda.synchronize()
    g_total = float(sum(a.elapsed_time(b) for a, b in g_ms))
    g_total = max_over_ranks(g_total, dist, dev)
    graph_out = {"ms_per_step": round(g_total / args.steps, 4),
                 "value": round(job_throughput(world, args.steps, mp_per_view, g_total), 2)}
    del graph
    # end to end through the public API with host buffers
    e2e = bench_e2e(r, ds, dL, args, dev, world, dist, mp_per_view)
    train = bench_train(r, ds, wl, args, dev, pk, n_sm, flush) if rank == 0 and world == 1 else None
    out = {
        "metric": METRIC, "value": round(value, 2), "unit": "MP/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms_per_step, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": config_of(wl, world),
        "l2": "flushed (2x L2 buffer written) between timed steps",
        "counts": {"instances": int(st.instances), "visible_records": int(st.visible_records),
                   "pairs": pairs, "visited_pairs": visited,
                   "pairs_definition": "pixels x records with r < 1 met before the pixel terminates, "
                                       "tile-free (lists without the tight cut); visited = entries the "
                                       "forward's warps evaluate x pixels of the warp"},
        "views_per_sec": round(job_throughput(world, args.steps, 1, total_ms), 2),
        "stage_ms": {n: round(float(m), 4) for n, m in zip(names, stage_mean)},
        "roofline": roof,
        "roofline_steps": steps_roof,
        "roofline_path": path_roof,
        "graph": graph_out,
        "e2e": e2e,
        "train_step": train,
        "gpu_launches": kernels_per_step(r) * args.steps,
        "clocks": clk,
        "wall_s_timed_loop": round(wall, 3),
    }
    if rank == 0 and not args.no_batched and world == 1:
        out["batched"] = bench_batched(dev, pk, n_sm)
        out["deep_tile"] = bench_deep_tile(dev)
        out["forward_only"] = bench_small_forward(dev)
    if dist:
        dist.destroy_process_group()
    return out


def bench_train(r, ds, wl, args, dev, pk, n_sm, flush):
    """One training iteration of Sec. 4.5/5.1 on the same view: render,
    image loss (L1 + 0.2 (1 - SSIM)) and its gradient, backward, Adam with
    the paper's learning rates and penalties, spatial noise drawn outside the
    timed region.  Per-stage CUDA events; L2 flushed between steps.  The
    scene's parameters change every step (the optimiser updates them)."""
    import torch

    from paper_2510_03312_gb300 import scenes as S
    from paper_2510_03312_gb300 import train as TR

    target = r.pack(S.l1_target(1, wl.views))
    loss_fn = TR.ImageLoss(wl.views, device=dev)
    params0 = ds.params.clone()
    opt = TR.Adam(wl.scenes[0], ds.params)
    noise = torch.randn(3, ds.P, device=dev) * 1e-4
    dL = torch.empty_like(target)
    stream = torch.cuda.current_stream()
    names = ["preprocess", "bin_sort", "render_fwd", "image_loss", "render_bwd_blend", "render_bwd_params", "adam"]
    img_holder = {}

    def step(evs):
        calls = [r.preprocess, r.bin_sort, lambda: img_holder.update(img=r.render_fwd()),
                 lambda: loss_fn(img_holder["img"], target, dL), lambda: r.render_bwd_blend(dL),
                 lambda: img_holder.update(g=r.render_bwd_params()), lambda: opt.step(img_holder["g"][0], noise)]
        evs[0].record(stream)
        for k, c in enumerate(calls):
            c()
            evs[k + 1].record(stream)

    def ev():
        return torch.cuda.Event(enable_timing=True)

    rows = []
    for i in range(args.warmup + args.steps):
        flush.fill_((i + 11) & 0xFF)
        evs = [ev() for _ in range(len(names) + 1)]
        step(evs)
        if i >= args.warmup:
            rows.append(evs)
    torch.cuda.synchronize()
    loss_last = float(loss_fn.loss[0])
    # MCMC relocation (Sec. 4.5) with 1% of the primitives made dead first
    reloc = TR.Relocator(opt)
    gen = torch.Generator(device=dev).manual_seed(5)
    orow = reloc.opacity_row
    dead = torch.rand(ds.P, device=dev, generator=gen) < 0.01
    rand = torch.randint(-2 ** 63, 2 ** 63 - 1, (ds.P,), device=dev, dtype=torch.int64, generator=gen)
    r_ms = []
    for i in range(4):
        with torch.no_grad():
            opt.act[orow][dead] = 0.001
        torch.cuda.synchronize()
        e0, e1 = ev(), ev()
        e0.record(stream)
        reloc(rand)
        e1.record(stream)
        torch.cuda.synchronize()
        if i > 0:
            r_ms.append(e0.elapsed_time(e1))
    n_moved = int(reloc.n_relocated.item())
    stage = np.array([[e[k].elapsed_time(e[k + 1]) for k in range(len(names))] for e in rows]).mean(0)
    with torch.no_grad():
        ds.params.copy_(params0)  # leave the scene as the other measurements found it
    step_ms = float(stage.sum())
    v = wl.views[0]
    pc = 3 * v.width * v.height
    n_par = ds.params.numel()
    alu_peak = alu_peak_tops(n_sm, pk.get("sm_max_mhz", 2070.0))
    t_loss = stage[names.index("image_loss")] * 1e-3
    t_adam = stage[names.index("adam")] * 1e-3
    loss_ops = LOSS_FP32_PER_PC * pc
    loss_bytes = LOSS_BYTES_PER_PC * pc
    adam_bytes = ADAM_BYTES_PER_PARAM * n_par
    return {
        "ms_per_step": round(step_ms, 4),
        "MP_per_s": round(v.width * v.height / 1e6 / (step_ms * 1e-3), 2),
        "stage_ms": {n: round(float(m), 4) for n, m in zip(names, stage)},
        "loss_after_steps": round(loss_last, 6),
        "mcmc_relocate": {"ms": round(float(np.median(r_ms)), 4), "relocated": n_moved, "primitives": ds.P},
        "roofline": {
            "image_loss": {"bound": "alu", "fp32_ops": loss_ops, "bytes": loss_bytes,
                           "achieved": round(loss_ops / t_loss / 1e12, 3), "peak": round(alu_peak, 2),
                           "unit": "T lane-op/s", "frac": round(loss_ops / t_loss / 1e12 / alu_peak, 4),
                           "hbm_frac": round(loss_bytes / t_loss / 1e9 / pk["hbm_gbs"], 4)},
            "adam": {"bound": "hbm", "bytes": adam_bytes, "achieved": round(adam_bytes / t_adam / 1e9, 1),
                     "peak": pk["hbm_gbs"], "unit": "GB/s", "frac": round(adam_bytes / t_adam / 1e9 / pk["hbm_gbs"], 4)},
        },
        "work": f"{pc} pixel-channels ({LOSS_FP32_PER_PC} FP32 ops, {LOSS_BYTES_PER_PC} B each); "
                f"{n_par} parameters x {ADAM_BYTES_PER_PARAM} B",
    }


def bench_e2e(r, ds, dL, args, dev, world, dist, mp_per_view):
    """Same metric through the public API (Rasterizer.forward/backward) with
    host buffers.  Every step copies the parameters and dL/dimage from pinned
    host memory and reads the image and the gradients back, as a training or
    serving loop does.  The copies are pipelined against the compute:

    - copy-in, compute and copy-out run on three streams, with two buffer sets;
    - step i+1's inputs go in while step i computes and step i-1's results
      come out;
    - the compute of consecutive steps stays serialised on one stream;
    - events keep every buffer from being overwritten before its reader has
      finished."""
    import torch

    from paper_2510_03312_gb300 import raster

    h_params = ds.params.cpu().pin_memory()
    h_dL = dL.cpu().pin_memory()
    sets = []
    for k in range(2):
        dsk = raster.DeviceScene(ds.N, ds.rot_mode, torch.empty_like(ds.params))
        dsk.params.copy_(ds.params)
        rk = raster.Rasterizer([dsk], r.views, r.cfg, capacity=r.capacity, device=dev)
        sets.append({"ds": dsk, "r": rk, "dL": torch.empty_like(dL),
                     "h_img": torch.empty_like(rk.image, device="cpu").pin_memory(),
                     "h_grad": torch.empty_like(dsk.params, device="cpu").pin_memory(),
                     "in": torch.cuda.Event(), "comp": torch.cuda.Event(), "out": torch.cuda.Event()})
    s_in, s_comp, s_out = (torch.cuda.Stream(device=dev) for _ in range(3))
    for k in range(2):  # every event recorded once, so that the first waits are satisfied
        for e in ("in", "comp", "out"):
            sets[k][e].record()

    def step(i):
        b = sets[i % 2]
        with torch.cuda.stream(s_in):
            s_in.wait_event(b["comp"])  # the previous compute on this set is done with its inputs
            b["ds"].params.copy_(h_params, non_blocking=True)
            b["dL"].copy_(h_dL, non_blocking=True)
            b["in"].record(s_in)
        with torch.cuda.stream(s_comp):
            s_comp.wait_event(b["in"])
            s_comp.wait_event(b["out"])  # the previous results of this set have been read back
            img = b["r"].forward(check=False)
            g = b["r"].backward(b["dL"])[0]
            b["comp"].record(s_comp)
        with torch.cuda.stream(s_out):
            s_out.wait_event(b["comp"])
            b["h_img"].copy_(img, non_blocking=True)
            b["h_grad"].copy_(g, non_blocking=True)
            b["out"].record(s_out)

    for i in range(max(3, args.warmup)):
        step(i)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for i in range(args.steps):
        step(i)
    cur = torch.cuda.current_stream()
    for st in (s_in, s_comp, s_out):
        cur.wait_stream(st)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    ms = max_over_ranks(ms, dist, dev)
    bi = h_params.numel() * 4 + h_dL.numel() * 4
    bo = sets[0]["h_grad"].numel() * 4 + sets[0]["h_img"].numel() * 4
    return {"value": round(job_throughput(world, args.steps, mp_per_view, ms), 2), "unit": "MP/s",
            "h2d_bytes_per_step": bi, "d2h_bytes_per_step": bo, "ms_per_step": round(ms / args.steps, 4),
            "pipelined": "copy-in, compute, copy-out on three streams, two buffer sets; compute serialised"}


def time_calls(fn, steps, warmup):
    """Milliseconds per call of fn() (CUDA events on the current stream)."""
    import torch

    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


def bench_small_forward(dev, steps=200, warmup=20):
    """The static N=3 4,096-primitive 128x128 view, forward only (preprocess
    -> bin_sort -> render_fwd), eagerly and replayed as one captured graph."""
    import torch

    from paper_2510_03312_gb300 import raster
    from paper_2510_03312_gb300 import scenes as S

    wl = S.workload_static_small()
    ds = raster.DeviceScene.from_scene(wl.scenes[0], device=dev)
    r = raster.Rasterizer([ds], wl.views, wl.cfg, device=dev)
    r.forward(check=True)
    mp = wl.views[0].width * wl.views[0].height / 1e6
    eager = time_calls(lambda: r.forward(check=False), steps, warmup)
    side = torch.cuda.Stream(device=dev)
    side.wait_stream(torch.cuda.current_stream(dev))
    with torch.cuda.stream(side):
        r.forward(check=False)
    torch.cuda.current_stream(dev).wait_stream(side)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        r.forward(check=False)
    graph = time_calls(g.replay, steps, warmup)
    out = {}
    for name, ms in (("eager", eager), ("graph", graph)):
        out[name] = {"ms_per_step": round(ms, 5), "MP_per_s": round(mp / (ms / 1e3), 2),
                     "views_per_s": round(1 / (ms / 1e3), 1)}
    return {wl.name: out}


def batched_rooflines(ds, wl, dev, pk, n_sm, steps, warmup):
    """Roofline of one batch: the whole batch as one problem (16x16 tiles),
    each stage timed with CUDA events, against the same per-unit work as the
    single view's stages (parameters read once per batch).  Also returns
    the parameter bytes of the batch and of the per-view form (which reads a
    scene's parameters once per view, in preprocess and twice in the
    parameter backward)."""
    import torch

    from paper_2510_03312_gb300 import raster

    cnt = raster.count_pairs(ds, wl.views, wl.cfg, device=dev)
    pairs = int(cnt["pairs"].sum().item())
    visited = int(cnt["visited"].sum().item())
    del cnt
    torch.cuda.empty_cache()
    r = raster.Rasterizer(ds, wl.views, wl.cfg, device=dev)
    img = r.forward(check=True)
    st = r.status()
    dL = torch.full_like(img, 1e-6)
    names = ["preprocess", "bin_sort", "render_fwd", "render_bwd_blend", "render_bwd_params"]
    stream = torch.cuda.current_stream()
    calls = [r.preprocess, r.bin_sort, r.render_fwd, lambda: r.render_bwd_blend(dL), r.render_bwd_params]
    rows = []
    for i in range(warmup + steps):
        evs = [torch.cuda.Event(enable_timing=True) for _ in range(6)]
        evs[0].record(stream)
        for k, c in enumerate(calls):
            c()
            evs[k + 1].record(stream)
        if i >= warmup:
            rows.append(evs)
    torch.cuda.synchronize()
    stage = np.array([[e[k].elapsed_time(e[k + 1]) for k in range(5)] for e in rows]).mean(0)
    batch_pb = sum(d.params.numel() * 4 for d in ds)
    view_pb = sum(ds[v.scene_id].params.numel() * 4 for v in wl.views)
    R = sum(ds[v.scene_id].P for v in wl.views)
    steps_roof, path = step_rooflines(stage, names, batch_pb, R, int(st.instances), r.n_tiles(), pairs, pk, n_sm)
    del r
    torch.cuda.empty_cache()
    return steps_roof, path, batch_pb, view_pb, pairs, visited


def bench_deep_tile(dev, steps=5, warmup=2):
    """The deep-tile workload (a dense cluster of 60K faint primitives inside
    a few tiles, in front of a 300K-primitive sparse view, 1600x1060): one
    fwd+bwd step with the tile lists blended whole (grid form) and split into
    segments of 2048 entries merged with the over operator (split form)."""
    import torch

    from dataclasses import replace

    from paper_2510_03312_gb300 import raster
    from paper_2510_03312_gb300 import scenes as S

    wl = S.workload_deep_tile()
    ds = [raster.DeviceScene.from_scene(sc, device=dev) for sc in wl.scenes]
    mp = sum(v.width * v.height for v in wl.views) / 1e6
    out = {"workload": wl.name, "primitives": wl.scenes[0].P}
    names = ["preprocess", "bin_sort", "render_fwd", "render_bwd_blend", "render_bwd_params"]
    stream = torch.cuda.current_stream()
    for form, cfg in (("grid", wl.cfg), ("split", replace(wl.cfg, split_lists=True))):
        r = raster.Rasterizer(ds, wl.views, cfg, device=dev)
        img = r.forward(check=True)
        if form == "grid":
            counts = r.export(5).cpu().numpy().view(np.uint32).astype(np.int64)
            out["longest_list"] = int(np.diff(counts).max())
        dL = torch.full_like(img, 1e-6)
        calls = [r.preprocess, r.bin_sort, r.render_fwd, lambda: r.render_bwd_blend(dL), r.render_bwd_params]
        rows = []
        for i in range(warmup + steps):
            evs = [torch.cuda.Event(enable_timing=True) for _ in range(6)]
            evs[0].record(stream)
            for k, c in enumerate(calls):
                c()
                evs[k + 1].record(stream)
            if i >= warmup:
                rows.append(evs)
        torch.cuda.synchronize()
        stage = np.array([[e[k].elapsed_time(e[k + 1]) for k in range(5)] for e in rows]).mean(0)
        ms = float(stage.sum())
        out[form] = {"ms_per_step": round(ms, 4), "MP_per_s": round(mp / (ms / 1e3), 2),
                     "stage_ms": {n: round(float(m), 4) for n, m in zip(names, stage)}}
        del r
        torch.cuda.empty_cache()
    out["speedup_split"] = round(out["grid"]["ms_per_step"] / out["split"]["ms_per_step"], 3)
    return out


def bench_batched(dev, pk, n_sm, steps=5, warmup=2):
    """Batches of views, forward+backward per step:
      view-dependent N=6, 500K primitives, 16 x 1280x720;
      dynamic N=7, 300K primitives, 8 (camera, time) x 1352x1014;
      uneven mix, 64 jobs over 8 scenes (N in {3,6,7}, 10K-2M primitives,
      256x256 to 1920x1080).
    Forms: per_view = one problem per view launched back to back (the plain
    form); batched_one_launch = all views in one problem, 16x16 tiles, eager;
    batched = the autotuned tile shape and schedule with the whole step
    replayed as one captured CUDA graph.  Gradients of each scene are summed
    over its views in every form.  Each form's roofline fraction is
    t_roof / t_step, t_roof the time of the form's algorithmic work at the
    peaks (batched_rooflines; the per-view form adds its extra parameter
    reads; the autotuned form is counted at 16x16 tiles)."""
    import torch

    from paper_2510_03312_gb300 import autotune as A
    from paper_2510_03312_gb300 import raster
    from paper_2510_03312_gb300 import scenes as S

    res = {}
    for make in (S.workload_view_dependent, S.workload_dynamic, S.workload_uneven_mix):
        wl = make()
        ds = [raster.DeviceScene.from_scene(sc, device=dev) for sc in wl.scenes]
        mp = sum(v.width * v.height for v in wl.views) / 1e6
        nv = len(wl.views)
        out = {"views": nv, "megapixels": round(mp, 3), "primitives": [sc.P for sc in wl.scenes]}

        def entry(ms):
            return {"ms_per_step": round(ms, 4), "MP_per_s": round(mp / (ms / 1e3), 2),
                    "views_per_s": round(nv / (ms / 1e3), 2)}

        for name, groups in (("per_view", A.per_view(wl.scenes, wl.views)),
                             ("batched_one_launch", A.one_launch(wl.scenes, wl.views))):
            b = raster.Batch(ds, wl.views, wl.cfg, groups, device=dev)
            b.size()
            dls = b.dL_like(1e-6)
            out[name] = entry(time_calls(lambda: b.step(dls), steps, warmup))
            del b, dls
            torch.cuda.empty_cache()
        t0 = time.perf_counter()
        plan = A.tune(wl.scenes, wl.views, wl.cfg, A.device_measure(ds, wl.views, wl.cfg, device=dev))
        t_tune = time.perf_counter() - t0
        from dataclasses import replace
        cfg = plan.config(wl.cfg)
        b = raster.Batch(ds, wl.views, cfg, plan.groups, device=dev)
        b.size()
        dls = b.dL_like(1e-6)
        g = b.capture(dls)
        out["batched"] = entry(time_calls(g.replay, steps, warmup))
        out["batched"].update({"tile": f"{plan.tile[0]}x{plan.tile[1]}", "schedule": plan.schedule,
                               "blend_launch": plan.form,
                               "launches": len(plan.groups), "captured_graph": True})
        out["autotune"] = {"seconds": round(t_tune, 1), "candidates_ms": plan.table}
        out["speedup_batched"] = round(out["per_view"]["ms_per_step"] / out["batched"]["ms_per_step"], 3)
        del b, dls, g
        torch.cuda.empty_cache()
        steps_roof, path, batch_pb, view_pb, pairs, visited = batched_rooflines(ds, wl, dev, pk, n_sm, steps,
                                                                                warmup)
        t_roof = path["t_roof_ms"]
        t_roof_pv = t_roof + 3 * (view_pb - batch_pb) / (pk["hbm_gbs"] * 1e9) * 1e3
        out["pairs"] = pairs
        out["visited_pairs"] = visited
        out["roofline_steps"] = steps_roof
        out["roofline_path"] = path
        for form, tr in (("per_view", t_roof_pv), ("batched_one_launch", t_roof), ("batched", t_roof)):
            out[form]["roofline_frac"] = round(tr / out[form]["ms_per_step"], 4)
        res[wl.name] = out
        del ds
        torch.cuda.empty_cache()
    return res


# ----------------------------------------------------------------------------
# CPU oracle (baseline and reference arm)
# ----------------------------------------------------------------------------

def oracle_sample(P, n_tiles=24, seed=0):
    """Times the float64 oracle on a bounded sample of the workload: every
    primitive's float32 decision stage and float64 conditioning/projection
    (forward and autograd backward), plus the compositing forward+backward of
    n_tiles tiles; the tile part is scaled to the whole image."""
    import torch

    from oracle import render64 as R64

    wl = workload(0, P)
    t0 = time.perf_counter()
    orc = R64.Oracle(wl.scenes, wl.views, wl.cfg)
    counts = np.diff(orc.bins["ranges"], axis=1)[:, 0]
    rng = np.random.default_rng(seed)
    tiles = sorted(rng.choice(counts.size, n_tiles, replace=False).tolist())
    t1 = time.perf_counter()
    leaves = orc.leaves(True)
    recs = orc.records(leaves)
    t2 = time.perf_counter()
    out = orc.render(leaves=leaves, tiles=tiles, recs=recs)
    img = out["image"][0]
    m = ~torch.isnan(img)
    loss = torch.where(m, img, torch.zeros_like(img)).abs().sum()
    t3 = time.perf_counter()
    loss.backward()
    t4 = time.perf_counter()
    n_total = counts.size
    # backward time splits between records and tiles; attribute it by tile share
    t_prim = (t1 - t0) + (t2 - t1)
    t_tiles = (t3 - t2) + (t4 - t3)
    full = t_prim + t_tiles * n_total / n_tiles
    mp = wl.views[0].width * wl.views[0].height / 1e6
    return {"value": round(mp / full, 5), "unit": "MP/s", "cores": torch.get_num_threads(), "kind": "oracle",
            "sample": f"all {wl.scenes[0].P} primitives (float32 stage + float64 conditioning/projection) and "
                      f"forward+backward compositing of {n_tiles} of {n_total} tiles, tile time scaled to the "
                      f"whole 1600x1060 view",
            "seconds": round(t4 - t0, 2), "extrapolated_s_per_step": round(full, 2)}


def bench_reference(args, rank, world):
    if rank != 0:
        return None
    steps = []
    for i in range(args.warmup):
        oracle_sample(args.primitives, n_tiles=4, seed=100 + i)
    t0 = time.perf_counter()
    for i in range(args.steps):
        steps.append(oracle_sample(args.primitives, n_tiles=24, seed=i))
    timed_s = time.perf_counter() - t0
    v = float(np.mean([s["value"] for s in steps]))
    s0 = steps[0]
    # every step is a bounded sample; its measured seconds are the timed
    # region, the whole-view seconds it stands for are extrapolated
    return {"impl": "reference", "metric": METRIC, "value": round(v, 5), "unit": "MP/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(1e3 * timed_s / args.steps, 1),
            "extrapolated_ms_per_full_step": round(1e3 * float(np.mean([s["extrapolated_s_per_step"]
                                                                          for s in steps])), 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config_of(workload(0, args.primitives), world),
            "cpu_baseline": {"value": round(v, 5), "unit": "MP/s", "cores": s0["cores"], "kind": "oracle",
                             "sample": s0["sample"]},
            "e2e": {"value": round(v, 5), "unit": "MP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        out = bench_reference(args, rank, world)
        if out is not None:
            print(json.dumps(out), flush=True)
        return
    # the CPU baseline runs first, in this process before any CUDA work
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = oracle_sample(args.primitives, n_tiles=1200)
    out = bench_ours(args, rank, world, local)
    if rank == 0:
        out["cpu_baseline"] = cpu
        print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
