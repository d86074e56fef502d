"""Shared helpers of the GPU parity tests (systems, contexts, oracle states)."""
import functools

import numpy as np
import pytest

torch = pytest.importorskip("torch")


@functools.lru_cache(maxsize=None)
def system(name):
    from workloads import make_system
    return make_system(name)


@functools.lru_cache(maxsize=None)
def oracle_state(name):
    from oracle import groundstate
    return groundstate.solve(system(name))


@functools.lru_cache(maxsize=None)
def context(name):
    import __graft_entry__
    __graft_entry__.build()
    from paper_2505_02319_gb300 import groundstate
    return groundstate.context_for(system(name))


def dev(a):
    return torch.tensor(np.ascontiguousarray(a).ravel(), dtype=torch.float64, device="cuda")


def rel(a, b):
    a = np.asarray(a).ravel()
    b = np.asarray(b).ravel()
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))
