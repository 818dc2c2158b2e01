"""Reference of MCMC relocation (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU legs of ``bench.py``
may use this module; the CUDA path never imports it.

Sec. 4.5 (optimisation and implementation): primitive management follows
the kernel-agnostic MCMC scheme of Deformable Beta Splatting; a primitive
cloned into N copies takes the opacity o' = 1 - (1 - o)^(1/N), which keeps
the composited density of the N stacked copies equal to the original's.

Readings (the paper states the opacity rule, not the procedure):

* A primitive is dead when its opacity is at most a threshold (0.005, the
  value of 3DGS-MCMC, on which the DBS scheme builds).
* Each dead primitive is moved onto a live source drawn with probability
  proportional to the source's opacity.  The draw is made exact: the weight
  of a live primitive is the integer floor(o * 2^24) (o in float32; the
  product is exact), the cumulative weights are integers, and each dead slot
  j brings its own 64-bit random number rand[j] (drawn by the caller): its
  source is the first primitive whose inclusive cumulative weight exceeds
  rand[j] mod (total weight).  Nothing is relocated when no primitive lives.
* A source drawn n times and its n new copies (N = n + 1 primitives) take
  o' = 1 - (1 - o)^(1/N); every other parameter of a copy is the source's.
  "Kernel-agnostic": no scale or Beta parameter is adjusted.
* The optimiser state (Adam moments) of the sources and the relocated slots
  is reset to zero.

Parity: pinned (tests/test_oracle_mcmc.py): the opacity rule composes back to
the source's alpha for every N; the sampled sources follow the weights
(chi-square on many draws) and are never dead; hand-built cases with known
draws; conservation of the total composited opacity of each source group.
"""
from __future__ import annotations

import numpy as np

DEAD_THRESHOLD = 0.005
WEIGHT_SCALE = 2 ** 24


def weights(opacity: np.ndarray, threshold: float = DEAD_THRESHOLD):
    """(dead mask, integer weights) from float32 opacities."""
    o = np.asarray(opacity, dtype=np.float32)
    dead = o <= np.float32(threshold)
    w = np.floor(o * np.float32(WEIGHT_SCALE)).astype(np.int64)
    w[dead] = 0
    return dead, w


def relocate(act, raw, m, v, opacity_row: int, rand, threshold: float = DEAD_THRESHOLD):
    """Relocate the dead primitives of one scene.

    act, raw, m, v: [K, P] arrays (the rasterizer's activated parameters, the
    optimiser's raw parameters and its moments); row ``opacity_row`` of act is
    the opacity (raw = logit of it).  rand: [P] uint64.  Returns
    (act', raw', m', v', sources) with sources[j] the source of dead slot j
    (-1 for live slots)."""
    act = np.array(act, dtype=np.float64)
    raw = np.array(raw, dtype=np.float64)
    m = np.array(m, dtype=np.float64)
    v = np.array(v, dtype=np.float64)
    K, P = act.shape
    dead, w = weights(act[opacity_row].astype(np.float32), threshold)
    src = np.full(P, -1, dtype=np.int64)
    total = int(w.sum())
    if total == 0 or not dead.any():
        return act, raw, m, v, src
    cdf = np.cumsum(w)  # inclusive
    rnd = np.asarray(rand, dtype=np.uint64)
    for j in np.flatnonzero(dead):
        r = int(rnd[j]) % total
        src[j] = int(np.searchsorted(cdf, r, side="right"))
    counts = np.bincount(src[src >= 0], minlength=P)
    o_src = act[opacity_row].copy()
    N = counts + 1
    new_o = 1.0 - (1.0 - o_src) ** (1.0 / N)
    for j in np.flatnonzero(dead):
        s = src[j]
        act[:, j] = act[:, s]
        raw[:, j] = raw[:, s]
        act[opacity_row, j] = new_o[s]
        raw[opacity_row, j] = np.log(new_o[s] / (1.0 - new_o[s]))
        m[:, j] = 0.0
        v[:, j] = 0.0
    for s in np.flatnonzero(counts):
        act[opacity_row, s] = new_o[s]
        raw[opacity_row, s] = np.log(new_o[s] / (1.0 - new_o[s]))
        m[:, s] = 0.0
        v[:, s] = 0.0
    return act, raw, m, v, src
