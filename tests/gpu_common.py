"""Shared fixtures for the GPU parity tests: the same seeded inputs feed the
oracle and the CUDA path."""
import numpy as np

import inputs


def have_gpu():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


def sorted_sets(sets):
    return [np.sort(np.asarray(s)) for s in sets]


def c1_edges():
    # configuration 1: directed R-MAT, 2^14 nodes, 2^17 draws, (0.57, 0.19, 0.19, 0.05)
    return inputs.rmat(14, 1 << 17, seed=1)
