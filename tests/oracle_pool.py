"""The FP64 oracle's preprocessing of a large scene on all host cores (test
infrastructure): the oracle's own ``preprocess`` on ranges of Gaussians in
worker processes started with ``spawn`` (the test process holds a CUDA
context), the projected records gathered in shared memory.  Nothing of the
oracle's arithmetic is changed: each Gaussian is projected by the same
routine, independently of the others."""
from __future__ import annotations

import multiprocessing as mp
import os
from multiprocessing import shared_memory

import numpy as np

_S = {}


def _init(attrs_name, shape, dtype, g_name, cam, mlp, use_mlp):
    import oracle
    oracle.build()
    a = shared_memory.SharedMemory(name=attrs_name)
    g = shared_memory.SharedMemory(name=g_name)
    _S.update(oracle=oracle, a_shm=a, g_shm=g, shape=shape, dtype=dtype, cam=cam, mlp=mlp,
              use_mlp=use_mlp)


def _part(rng):
    lo, hi = rng
    oracle = _S["oracle"]
    attrs = np.ndarray(_S["shape"], _S["dtype"], buffer=_S["a_shm"].buf)
    out = oracle.preprocess(attrs[lo:hi], _S["cam"], _S["mlp"], use_mlp=_S["use_mlp"])
    view = np.ndarray((_S["shape"][0],), oracle.GAUSS_DTYPE, buffer=_S["g_shm"].buf)
    view[lo:hi] = out
    del attrs, view
    return hi - lo


def preprocess(attrs: np.ndarray, cam, mlp=None, use_mlp: bool = False, procs: int | None = None):
    """oracle.preprocess(attrs, cam, mlp, use_mlp), split over processes."""
    import oracle
    oracle.build()
    attrs = np.ascontiguousarray(attrs)
    n = attrs.shape[0]
    procs = procs or os.cpu_count() or 1
    a_shm = shared_memory.SharedMemory(create=True, size=max(attrs.nbytes, 1))
    g_shm = shared_memory.SharedMemory(create=True, size=max(n * oracle.GAUSS_DTYPE.itemsize, 1))
    try:
        av = np.ndarray(attrs.shape, attrs.dtype, buffer=a_shm.buf)
        av[:] = attrs
        del av
        parts = 4 * procs
        bounds = [n * k // parts for k in range(parts + 1)]
        ctx = mp.get_context("spawn")
        with ctx.Pool(procs, initializer=_init,
                      initargs=(a_shm.name, attrs.shape, attrs.dtype, g_shm.name, cam, mlp,
                                use_mlp)) as pool:
            pool.map(_part, [(bounds[k], bounds[k + 1]) for k in range(parts)], chunksize=1)
        gv = np.ndarray((n,), oracle.GAUSS_DTYPE, buffer=g_shm.buf)
        g = gv.copy()
        del gv
        return g
    finally:
        for m in (a_shm, g_shm):
            m.close()
            m.unlink()
