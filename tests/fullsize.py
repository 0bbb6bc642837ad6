"""Which walkers of a full-size batch the oracle recomputes one by one.

A sample of at least ``n`` walkers: the 8 lightest and the 8 heaviest (the shortest and
the longest mode bands), up to 16 whose band (by the oracle's own band rule) starts at
the first or ends at the last grid bin, then seeded random picks.  Not a test module."""
import numpy as np


def sample_walkers(orc, th, t0, modes, grid, n=128, seed=0):
    B = th.shape[0]
    m = th[:, 0]
    pick = list(np.argsort(m)[:8]) + list(np.argsort(m)[-8:])
    edge = []
    for b in range(B):
        if len(edge) >= 16:
            break
        for (l, mm) in modes:
            r = orc.band(th[b], t0, l, mm, grid.f0, grid.df, grid.n_bins)
            if r is not None and (r[2] == 0 or r[3] == grid.n_bins - 1):
                edge.append(b)
                break
    pick += edge
    rest = np.setdiff1d(np.arange(B), pick)
    rng = np.random.default_rng(seed)
    need = max(n - len(set(pick)), 0)
    pick += list(rng.choice(rest, size=min(need, rest.size), replace=False))
    return np.unique(np.array(pick, dtype=np.int64)), len(set(edge))
