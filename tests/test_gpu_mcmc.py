"""GPU parity of MCMC relocation (ubs_mcmc_relocate) against the reference:
the drawn sources bit for bit, copied parameters bit for bit, the cloned
opacities within float32 rounding, and the reset moments."""
import numpy as np
import pytest
import torch

from oracle import mcmc64 as M
from paper_2510_03312_gb300 import scenes as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_03312_gb300 import build as B
    B.build()
    return torch.device("cuda", 0)


def _case(P, seed, dead_frac):
    rng = np.random.default_rng(seed)
    sc = S.make_scene(seed, 6, P)
    act = sc.params.copy()
    orow = sc.offsets()["opacity"][0]
    o = act[orow]
    dead = rng.random(P) < dead_frac
    o[dead] = rng.uniform(0.0, 0.005, dead.sum()).astype(np.float32)
    raw = act.copy()
    raw[orow] = np.log(o / (1 - o))
    m = rng.standard_normal(act.shape).astype(np.float32)
    v = rng.random(act.shape).astype(np.float32)
    rand = rng.integers(0, 2 ** 63, size=P, dtype=np.uint64) * np.uint64(2) + rng.integers(0, 2, size=P,
                                                                                            dtype=np.uint64)
    return act, raw, m, v, rand, orow


@pytest.mark.parametrize("P,seed,dead_frac", [(3000, 1, 0.1), (5000, 2, 0.6), (1024, 3, 0.05), (1, 4, 0.0),
                                              (200_000, 5, 0.02), (777, 6, 1.0)])
def test_relocation_matches_reference(dev, P, seed, dead_frac):
    from paper_2510_03312_gb300 import ubs as U
    import ctypes
    act, raw, m, v, rand, orow = _case(P, seed, dead_frac)
    K = act.shape[0]
    t = {k: torch.tensor(a, device=dev).contiguous() for k, a in dict(act=act, raw=raw, m=m, v=v).items()}
    rnd = torch.tensor(rand.view(np.int64), device=dev)
    src = torch.empty(P, dtype=torch.int32, device=dev)
    nrel = torch.zeros(1, dtype=torch.int64, device=dev)
    n = U.ubs_mcmc_workspace_size(P)
    ws = torch.empty(n + 256, dtype=torch.uint8, device=dev)
    wp = (ws.data_ptr() + 255) // 256 * 256
    st = U.ubs_mcmc_relocate(K, P, orow, 0.005, t["act"].data_ptr(), t["raw"].data_ptr(), t["m"].data_ptr(),
                             t["v"].data_ptr(), rnd.data_ptr(), src.data_ptr(), nrel.data_ptr(), wp, n,
                             ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == U.UBS_OK
    a_r, r_r, m_r, v_r, src_r = M.relocate(act, raw, m, v, orow, rand)
    s_g = src.cpu().numpy()
    assert np.array_equal(s_g, src_r)
    assert int(nrel.item()) == int((src_r >= 0).sum())
    ag, rg = t["act"].cpu().numpy(), t["raw"].cpu().numpy()
    other = [k for k in range(K) if k != orow]
    assert np.array_equal(ag[other], a_r[other].astype(np.float32))
    assert np.array_equal(rg[other], r_r[other].astype(np.float32))
    np.testing.assert_allclose(ag[orow], a_r[orow], rtol=2e-6, atol=1e-9)
    touched = (src_r >= 0) | (np.bincount(src_r[src_r >= 0], minlength=P) > 0)
    np.testing.assert_allclose(rg[orow][touched], r_r[orow][touched], rtol=2e-5, atol=2e-5)
    assert np.array_equal(rg[orow][~touched], raw[orow][~touched])
    assert np.array_equal(t["m"].cpu().numpy(), m_r.astype(np.float32))
    assert np.array_equal(t["v"].cpu().numpy(), v_r.astype(np.float32))
