"""The FP64 oracle's P and P^T evaluated on all host cores (test infrastructure).

TEST INFRASTRUCTURE ONLY: used by the benchmark's CPU baseline and reference arm to time
the oracle on every host core, and by the test suite.  It shares no code with the CUDA
path.  The rays of the scan are split into contiguous view ranges, one per worker process
(spawned, so that it is safe after CUDA has been initialised); each worker runs the
oracle's own plain-C Siddon routines (siddon.c) on its rays:
  P f      -- every ray's line integral is computed exactly as in Operator.project, so the
              result is bit-identical to the single-process oracle;
  P^T y    -- each worker scatters its rays into a partial image, and the partial images
              are added in worker order (the same FP64 terms as Operator.backproject, summed
              in a different, fixed order).
f, y and the partial images travel through shared memory; only view ranges are sent.
Everything else of the oracle (CGLS, (P2), the clamp) is unchanged and single-threaded:
ShardedOperator is a drop-in replacement for Operator in eptv_oracle.cgls / reconstruct.
"""
from __future__ import annotations

import multiprocessing as mp
import os
from multiprocessing import shared_memory

import numpy as np

from . import eptv_oracle as O

_W = {}


def _init(geom, names, n_workers):
    g = geom
    _W["g"] = g
    _W["rays"] = O.rays(g)
    _W["shm"] = [shared_memory.SharedMemory(name=n) for n in names]
    _W["f"] = np.ndarray((g.n_pix,), dtype=np.float64, buffer=_W["shm"][0].buf)
    _W["y"] = np.ndarray((g.n_rays,), dtype=np.float64, buffer=_W["shm"][1].buf)
    _W["parts"] = np.ndarray((n_workers, g.n_pix), dtype=np.float64, buffer=_W["shm"][2].buf)


def _project(task):
    w, r0, r1 = task
    g = _W["g"]
    sx, sy, ux, uy = (a[r0:r1] for a in _W["rays"])
    _W["y"][r0:r1] = O.project_rays(g.nx, g.ny, g.dx, g.dy, sx, sy, ux, uy, _W["f"])
    return w


def _backproject(task):
    w, r0, r1 = task
    g = _W["g"]
    sx, sy, ux, uy = (a[r0:r1] for a in _W["rays"])
    _W["parts"][w] = O.backproject_rays(g.nx, g.ny, g.dx, g.dy, sx, sy, ux, uy, _W["y"][r0:r1])
    return w


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


class ShardedOperator:
    """P and P^T of one geometry on n_workers processes (default: every host core)."""

    def __init__(self, g, n_workers: int | None = None):
        self.g = g
        n = max(1, min(n_workers or host_cores(), g.n_views))
        self.n_workers = n
        bounds = np.linspace(0, g.n_views, n + 1).round().astype(int)
        self.tasks = [(w, int(bounds[w]) * g.n_bins, int(bounds[w + 1]) * g.n_bins) for w in range(n)]
        sizes = [8 * g.n_pix, 8 * g.n_rays, 8 * n * g.n_pix]
        self._shm = [shared_memory.SharedMemory(create=True, size=s) for s in sizes]
        self._f = np.ndarray((g.n_pix,), dtype=np.float64, buffer=self._shm[0].buf)
        self._y = np.ndarray((g.n_rays,), dtype=np.float64, buffer=self._shm[1].buf)
        self._parts = np.ndarray((n, g.n_pix), dtype=np.float64, buffer=self._shm[2].buf)
        O.build()
        self._pool = mp.get_context("spawn").Pool(n, initializer=_init,
                                                  initargs=(g, [m.name for m in self._shm], n))

    def project(self, f):
        g = self.g
        self._f[:] = np.asarray(f, dtype=np.float64).reshape(-1)
        self._pool.map(_project, self.tasks)
        return self._y.copy().reshape(g.n_views, g.n_bins)

    def backproject(self, y):
        g = self.g
        self._y[:] = np.asarray(y, dtype=np.float64).reshape(-1)
        self._pool.map(_backproject, self.tasks)
        out = np.zeros(g.n_pix)
        for w in range(self.n_workers):       # fixed order
            out += self._parts[w]
        return out.reshape(g.ny, g.nx)

    def close(self):
        if self._pool is not None:
            self._pool.close()
            self._pool.join()
            self._pool = None
        for m in self._shm:
            m.close()
            m.unlink()
        self._shm = []

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
