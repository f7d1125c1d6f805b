"""Spin-resolved walkers: two Slater determinants per walker, one for the N_up
and one for the N_down electrons (the paper's solid-state sizing counts both
spins, Sec. III). The wavefunction is det(A_up) det(A_down); moving an up
electron changes only A_up, so its Metropolis ratio is the up determinant's
ratio alone, and likewise for down electrons. A sweep moves the up electrons,
then the down electrons, each spin's determinant through its own handle of
the library (its own delay queue, flushes and recomputes); log|det| and sign
of the walker are the sum and the product of the two (qmcdu_logdet_product,
on the device).

Thin orchestration over two handles: every step runs in the library's kernels.
The spin-down walkers draw from keys offset by `down_key_offset` so that the
two determinants never share random numbers.
"""
from __future__ import annotations

import numpy as np

from .qmcdu import Walkers, qmcdu_logdet_product


class SpinWalkers:
    def __init__(self, n_up, n_down, K, precision="fp64", batch=1, stream=None,
                 down_key_offset=1 << 40):
        self.n_up, self.n_down, self.batch = int(n_up), int(n_down), int(batch)
        self.off = int(down_key_offset)
        self.up = Walkers(n_up, min(K, n_up), precision, batch, stream=stream)
        self.down = Walkers(n_down, min(K, n_down), precision, batch, stream=stream)

    def load(self, seeds):
        """Draw each walker's two matrices on the device from its key."""
        seeds = [int(s) for s in seeds]
        self.up.load_walkers(0, self.batch, seeds=seeds)
        self.down.load_walkers(0, self.batch, seeds=[s + self.off for s in seeds])

    def sweep(self, seeds, sweep_index, sigma, accepted_up=None, accepted_down=None,
              ratios_up=None, ratios_down=None):
        """One sweep of every walker: its up electrons, then its down electrons."""
        seeds = [int(s) for s in seeds]
        walkers = list(range(self.batch))
        self.up.sweep_walkers(walkers, seeds, [sweep_index] * self.batch, sigma,
                              accepted_out=accepted_up, ratios_out=ratios_up)
        self.down.sweep_walkers(walkers, [s + self.off for s in seeds],
                                [sweep_index] * self.batch, sigma,
                                accepted_out=accepted_down, ratios_out=ratios_down)

    def logdet(self):
        """(log|det A_up| + log|det A_down|, sign(det A_up) sign(det A_down)) per walker."""
        la = np.zeros(self.batch)
        sg = np.zeros(self.batch, dtype=np.int32)
        qmcdu_logdet_product(self.up.h, self.down.h, la, sg, self.batch)
        return la, sg

    def close(self):
        self.up.close()
        self.down.close()
