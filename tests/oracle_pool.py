"""The FP64 oracle's per-sample radiance in one spawned process per host core, for the parity tests
at full size (test infrastructure: it runs the oracle as it stands, only on several cores).

Spawned, not forked, so that no CUDA state of the test process is inherited. Every process gets the
scene once (pickled at start-up) and reads the parameter texture from one shared-memory block, so a
2048^2 x 5 texture is not copied per task. A perturbed evaluation (one texel channel moved by h, for
finite differences) works on a private copy that each process makes once, the texel restored
exactly after the evaluation.
"""
from __future__ import annotations

import multiprocessing as mp
import os
from multiprocessing import shared_memory

import numpy as np

_W: dict = {}


def _init(scene, shm_name, shape):
    from oracle import orc
    _W["orc"] = orc
    _W["sc"] = orc.Scene(scene)
    _W["shm"] = shared_memory.SharedMemory(name=shm_name)
    _W["tex"] = np.ndarray(shape, np.float64, buffer=_W["shm"].buf)


def _render(pixels, samples, iteration, stream, pert):
    orc, sc = _W["orc"], _W["sc"]
    if pert is None:
        return orc.render_samples(sc, _W["tex"], pixels, samples, iteration, stream)
    if "own" not in _W:                     # this process's private copy, made once
        _W["own"] = _W["tex"].copy()
    tex = _W["own"]
    y, x, c, d = pert
    keep = tex[y, x, c]
    tex[y, x, c] = keep + d
    try:
        return orc.render_samples(sc, tex, pixels, samples, iteration, stream)
    finally:
        tex[y, x, c] = keep                 # restored exactly


class OraclePool:
    """with OraclePool(scene, tex) as op: op.render_samples(pixels, samples, iteration, stream)"""

    def __init__(self, scene: dict, tex, workers: int | None = None):
        t = np.ascontiguousarray(np.asarray(tex, np.float64))
        self.shape = t.shape
        self.shm = shared_memory.SharedMemory(create=True, size=max(t.nbytes, 8))
        np.ndarray(t.shape, np.float64, buffer=self.shm.buf)[...] = t
        self.workers = workers or os.cpu_count() or 1
        self.pool = mp.get_context("spawn").Pool(self.workers, initializer=_init,
                                                  initargs=(scene, self.shm.name, self.shape))

    def render_samples(self, pixels, samples, iteration, stream, pert=None):
        """Radiance of the paths (pixels[k], samples[k]) as orc.render_samples computes it, the
        paths dealt round-robin to the processes and returned in the caller's order."""
        pixels = np.ascontiguousarray(pixels, np.uint32)
        samples = np.ascontiguousarray(samples, np.uint32)
        n = len(pixels)
        parts = min(self.workers * 4, max(n, 1))
        idx = [np.arange(k, n, parts) for k in range(parts)]
        res = self.pool.starmap(_render, [(pixels[i], samples[i], iteration, stream, pert) for i in idx])
        out = np.zeros((n, 3), np.float64)
        for i, r in zip(idx, res):
            out[i] = r
        return out

    def close(self):
        if self.pool is not None:
            self.pool.close()
            self.pool.join()
            self.pool = None
        if self.shm is not None:
            self.shm.close()
            self.shm.unlink()
            self.shm = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
