"""Oracle work items for process pools in the GPU tests.

Module-level functions, so that a pool started with the spawn method can
pickle them; this module imports only numpy and the oracle (no GPU code), so
spawned workers never touch the device.
"""
import concurrent.futures as cf
import multiprocessing as mp
import os

import oracle


def spawn_pool(workers=None):
    """A process pool started with spawn (safe after the parent used the GPU)."""
    n = workers or min(16, os.cpu_count() or 1)
    return cf.ProcessPoolExecutor(max_workers=n, mp_context=mp.get_context("spawn"))


def full_solve(args):
    """oracle.solve on one mesh: (rho, N, dx0, method, interp) -> potentials."""
    rho, N, dx0, method, interp = args
    return oracle.solve(rho, N, dx0, method=method, interp=interp)


def cells(args):
    """The direct-sum route at sampled cells: (rho, N, dx0, samples) -> values."""
    rho, N, dx0, samples = args
    return oracle.nested_potential_at(rho, N, dx0, samples)
