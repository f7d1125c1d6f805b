"""Walkers of uneven N stepped together: one handle per size class, a walker
group (qmcdu_group_*) that forks the classes' persistent sweeps onto their own
streams, gives each a share of the SMs in proportion to its flush work, and can
replay the whole step from one CUDA graph. Thin wrapper: every step runs in the
library's kernels."""
from __future__ import annotations

import numpy as np

from . import inputs
from .qmcdu import Walkers, qmcdu_group_create, qmcdu_group_destroy, qmcdu_group_step


class SizeClass:
    """`batch` walkers of N electrons with delay K on their own CUDA stream."""

    def __init__(self, N, K, batch, precision="fp64", base_seed=0, stream=None):
        import torch
        self.N, self.K, self.batch, self.base_seed = N, K, batch, base_seed
        self.stream = stream if stream is not None else torch.cuda.Stream()
        self.walkers = Walkers(N, K, precision, batch, stream=self.stream)

    def initial_matrices(self):
        return np.stack([inputs.initial_matrix(inputs.walker_seed(self.base_seed, b), self.N)
                         for b in range(self.batch)])

    def load(self, A=None):
        self.walkers.set_matrix(self.initial_matrices() if A is None else A)

    def results(self, nsweeps):
        acc = np.zeros((nsweeps, self.batch, self.N), dtype=np.uint8)
        rat = np.zeros((nsweeps, self.batch, self.N))
        self.walkers.step_results(nsweeps, acc, rat)
        return acc, rat

    def close(self):
        self.walkers.close()


class WalkerGroup:
    """Size classes stepped as one (optionally graph-captured) launch sequence."""

    def __init__(self, classes):
        self.classes = list(classes)
        self.g = qmcdu_group_create([c.walkers.h for c in self.classes])

    def step(self, first_sweep, nsweeps, sigma, recompute=True, use_graph=True):
        seeds = [c.base_seed for c in self.classes]
        qmcdu_group_step(self.g, seeds, first_sweep, nsweeps, sigma, recompute, use_graph)

    def synchronize(self):
        for c in self.classes:
            c.stream.synchronize()

    def close(self):
        if self.g:
            self.synchronize()
            qmcdu_group_destroy(self.g)
            self.g = None
