"""The Python binding checks every tensor before its pointer reaches the
C-ABI (which takes bare pointers it cannot check against an allocation):
device, dtype, contiguity, shape or element count, and aliasing.  These run
on the CPU; no call below gets as far as the library."""
import numpy as np
import pytest
import torch

from paper_2510_03312_gb300 import raster
from paper_2510_03312_gb300 import scenes as S
from paper_2510_03312_gb300 import train as TR

CPU = torch.device("cpu")
CUDA0 = torch.device("cuda", 0)


def test_check_tensor_accepts_a_matching_tensor():
    t = torch.zeros(3, 5)
    assert raster.check_tensor(t, "t", CPU, shape=(3, 5)) is t
    assert raster.check_tensor(t, "t", CPU, numel=15) is t


@pytest.mark.parametrize("bad,kw,msg", [
    (torch.zeros(4), dict(device=CUDA0), "is on cpu"),
    (torch.zeros(4, dtype=torch.float64), dict(device=CPU), "dtype"),
    (torch.zeros(4, 4).t(), dict(device=CPU), "contiguous"),
    (torch.zeros(4, 3), dict(device=CPU, shape=(3, 4)), "shape"),
    (torch.zeros(11), dict(device=CPU, numel=12), "elements"),
    (torch.zeros(4, dtype=torch.int32), dict(device=CPU, dtype=torch.int64), "dtype"),
])
def test_check_tensor_rejects(bad, kw, msg):
    device = kw.pop("device")
    with pytest.raises(ValueError, match=msg):
        raster.check_tensor(bad, "x", device, **kw)


def test_check_tensor_rejects_non_tensors():
    with pytest.raises(TypeError):
        raster.check_tensor(np.zeros(4, np.float32), "x", CPU)


def test_overlaps():
    buf = torch.zeros(100)
    assert raster.overlaps(buf[:50], buf[49:])
    assert not raster.overlaps(buf[:50], buf[50:])
    assert raster.overlaps(buf, buf)
    assert not raster.overlaps(buf, torch.zeros(100))


def test_device_objects_refuse_the_host():
    sc = S.make_scene(1, 3, 64)
    with pytest.raises(ValueError):
        raster.DeviceScene(3, sc.rot_mode, torch.tensor(sc.params))  # a host tensor
    with pytest.raises(ValueError, match="CUDA"):
        TR.ImageLoss([S.View(np.eye(3), np.zeros(3), 10.0, 10.0, 4.0, 4.0, 8, 8)], device="cpu")


def test_optimiser_on_the_host_refuses_to_step():
    """A CPU optimiser (checkpoint handling works there) never hands its host
    pointers to the library."""
    sc = S.make_scene(2, 3, 40)
    opt = TR.Adam(sc, torch.tensor(sc.params))
    with pytest.raises(ValueError, match="CUDA"):
        opt.step(torch.zeros_like(opt.act))
    reloc = TR.Relocator(opt)
    with pytest.raises(ValueError, match="CUDA"):
        reloc(torch.zeros(opt.P, dtype=torch.int64))
    assert opt.step_count == 0


def test_optimiser_rejects_a_parameter_block_of_the_wrong_layout():
    sc = S.make_scene(2, 3, 40)
    with pytest.raises(ValueError):
        TR.Adam(sc, torch.tensor(sc.params)[:-1].contiguous())
    with pytest.raises(ValueError):
        TR.Adam(sc, torch.tensor(sc.params, dtype=torch.float64))
    with pytest.raises(ValueError):
        TR.Adam(sc, torch.tensor(sc.params).reshape(-1))
