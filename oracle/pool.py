"""Worker processes for the oracle's independent per-slice work.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

In Algorithm 1 the fine sweeps of Step A, the restriction and coarse
evaluations of Step B, the interpolation of Step D and the fine evaluations
that end the predictor are independent across time slices (each slice runs on
its own processor in the paper); only Step C and the rounds of the predictor
are ordered.  ``SlicePool`` runs such independent calls of one level's methods
in worker processes so that the oracle uses every host core at the sizes of
the benchmark.  It changes no arithmetic: every call is the same
``SDCLevel`` method on the same arrays, in a process of its own, and the
results come back in slice order.  The processes are started with the
``spawn`` method (never forked), so they are safe to create after a GPU
context exists in the parent.
"""
from __future__ import annotations

import multiprocessing as mp
import os

_LEVELS: dict = {}


def _init(specs: dict) -> None:
    os.environ.setdefault("OPENBLAS_NUM_THREADS", "1")
    from .sdc import SDCLevel
    for name, args in specs.items():
        _LEVELS[name] = SDCLevel(*args)


def _call(task):
    name, method, args = task
    return getattr(_LEVELS[name], method)(*args)


def _ping(_):
    return len(_LEVELS)


class SlicePool:
    """``specs`` maps a level name to the ``SDCLevel`` constructor arguments
    (T, nlat, nlon, num_nodes, dt, params); every worker builds each level
    once.  ``run(name, method, arg_tuples)`` returns
    ``[getattr(level, method)(*a) for a in arg_tuples]``."""

    # a worker that cannot start (an import error) would be restarted forever
    # by multiprocessing.Pool: every wait below is bounded instead
    START_TIMEOUT_S, CALL_TIMEOUT_S = 600, 7200

    def __init__(self, specs: dict, workers: int | None = None):
        self.workers = max(1, workers or (os.cpu_count() or 1))
        self._pool = mp.get_context("spawn").Pool(self.workers, initializer=_init, initargs=(specs,))
        try:
            self._pool.map_async(_ping, range(self.workers), chunksize=1).get(self.START_TIMEOUT_S)
        except BaseException:
            self.close()
            raise

    def run(self, name: str, method: str, arg_tuples: list) -> list:
        tasks = [(name, method, tuple(a)) for a in arg_tuples]
        return self._pool.map_async(_call, tasks, chunksize=1).get(self.CALL_TIMEOUT_S)

    def pids(self) -> list[int]:
        """Process ids of the workers (to account for the CPU time they use)."""
        return [p.pid for p in self._pool._pool] if self._pool is not None else []

    def close(self) -> None:
        if self._pool is not None:
            self._pool.terminate()
            self._pool.join()
            self._pool = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
