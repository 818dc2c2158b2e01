"""Host logic of the training step: the optimiser's per-plane table (Sec. 5.1
learning rates, Sec. 4.5 penalties and noise) and the inverse activations."""
import numpy as np
import pytest
import torch

from paper_2510_03312_gb300 import scenes as S
from paper_2510_03312_gb300 import train as TR
from paper_2510_03312_gb300 import ubs as U


@pytest.mark.parametrize("N,rot", [(3, S.ROT_QUAT), (3, S.ROT_SKEW1), (4, S.ROT_QUAT), (6, S.ROT_QUAT),
                                   (7, S.ROT_SKEW1)])
def test_plane_table(N, rot):
    tc = TR.TrainConfig()
    t = TR.plane_table(N, rot, tc)
    rows = S.plane_rows(N, rot)
    assert len(t) == S.params_per_primitive(N, rot)
    off = 0
    offs = {}
    for name in S.PLANE_ORDER:
        offs[name] = (off, rows[name])
        off += rows[name]
    C = N - 3
    o, n = offs["mean_x"]
    assert [t[o + i] for i in range(3)] == [(tc.lr_position, U.UBS_ACT_IDENTITY, 0.0, i) for i in range(3)]
    o, n = offs["scale_x"]
    assert all(t[o + i] == (tc.lr_scale, U.UBS_ACT_EXP, tc.lambda_sigma, -1) for i in range(3))
    o, n = offs["opacity"]
    assert t[o] == (tc.lr_opacity, U.UBS_ACT_SIGMOID, tc.lambda_o, -1)
    o, n = offs["L_q"]
    diag = [i * (i + 1) // 2 + i for i in range(C)]
    for r in range(n):
        want = (tc.lr_scale, U.UBS_ACT_EXP, 0.0, -1) if r in diag else (tc.lr_other, U.UBS_ACT_IDENTITY, 0.0, -1)
        assert t[o + r] == want
    # only the spatial mean takes noise; only opacity and spatial scales are penalised
    assert sorted(x[3] for x in t if x[3] >= 0) == [0, 1, 2]
    assert sum(1 for x in t if x[2] > 0) == 4
    assert sum(1 for x in t if x[1] == U.UBS_ACT_EXP) == 3 + C


def test_raw_from_activated_inverts_the_activations():
    sc = S.make_scene(3, 6, 50)
    t = TR.plane_table(6, sc.rot_mode, TR.TrainConfig())
    act = torch.tensor(sc.params, dtype=torch.float64)
    raw = TR.raw_from_activated(act, t)
    back = raw.clone()
    for k, (_, a, _, _) in enumerate(t):
        if a == U.UBS_ACT_SIGMOID:
            back[k] = torch.sigmoid(raw[k])
        elif a == U.UBS_ACT_EXP:
            back[k] = torch.exp(raw[k])
    assert torch.allclose(back, act, rtol=1e-12, atol=1e-12)


def test_checkpoint_round_trip(tmp_path):
    sc = S.make_scene(9, 7, 40)
    act = torch.tensor(sc.params)
    a = TR.Adam(sc, act.clone())
    a.m.normal_()
    a.v.uniform_()
    a.raw.add_(0.5)
    a.step_count = 17
    path = str(tmp_path / "ckpt.npz")
    TR.save_checkpoint(path, [a], iteration=123)
    b = TR.Adam(sc, act.clone())
    assert TR.load_checkpoint(path, [b]) == 123
    for name in ("raw", "act", "m", "v"):
        assert torch.equal(getattr(a, name), getattr(b, name)), name
    assert b.step_count == 17
    other = TR.Adam(S.make_scene(9, 3, 40), torch.tensor(S.make_scene(9, 3, 40).params))
    with pytest.raises(ValueError):
        TR.load_checkpoint(path, [other])
