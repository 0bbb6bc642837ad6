"""Plain numpy reference of the relative-binning (heterodyned) likelihood
(TEST INFRASTRUCTURE ONLY; shares no code with the CUDA path).

The paper leaves faster approximations of its likelihood as future work (Sec. II.A);
this is one from the literature: relative binning (Zackay, Dai & Venumadhav 2018),
the heterodyning of Cornish (2010) with a fiducial waveform h0 near the posterior.
Written out here, mode by mode and channel by channel:

* Coarse bins: n_rb + 1 edges log-spaced in frequency across the union [lo, hi] of the
  fiducial's mode bands, each snapped to the nearest grid bin, together with every
  mode's band start j_lo and end j_hi + 1 (sorted, duplicates dropped; the last edge is
  hi + 1); bin b holds the grid bins e_b <= j < e_{b+1}.
* Summary data per mode lm, channel c, bin b (w = 4 df / S_c, Eq. (3)):
      A0 = sum_j w d h0_lm*,        A1 = sum_j w d h0_lm* (f_j - f_b),
      B0 = sum_j w h0_lm h0_l'm'*,  B1 = sum_j w h0_lm h0_l'm'* (f_j - f_b)
  for every pair of modes, with f_b the frequency of edge e_b.
* For parameters theta, the ratio r_lm,c(f) = h_lm,c(f; theta) / h0_lm,c(f) at the edges,
  linear inside each bin: r0 = r(f_b), r1 = (r(f_{b+1}) - r(f_b)) / (f_{b+1} - f_b); where
  h0 vanishes at one edge of a bin (a band ends there), r is the other edge's value
  across the bin (r1 = 0); where it vanishes at both, r0 = r1 = 0.  Then
      <d|h> = Re sum (A0 conj(r0) + A1 conj(r1)),
      <h|h> = Re sum_{lm, l'm'} (B0 r0_lm conj(r0_l'm') + B1 (r0_lm conj(r1_l'm') + r1_lm conj(r0_l'm'))),
  summed over channels and bins, and ln L = <d|h> - <h|h>/2 - <d|d>/2 (Eq. (2)).
The templates are the direct model (waveform and response evaluated at each frequency).
"""
from __future__ import annotations

import numpy as np

import oracle as O


def edges(th_fid, t0, modes, grid, n_rb):
    """Grid indices of the bin edges (sorted, unique, last = hi + 1)."""
    lo, hi, marks = None, None, []
    for (l, m) in modes:
        b = O.band(th_fid, t0, l, m, grid.f0, grid.df, grid.n_bins)
        if b is None:
            continue
        lo = b[2] if lo is None else min(lo, b[2])
        hi = b[3] if hi is None else max(hi, b[3])
        marks += [b[2], b[3] + 1]
    if lo is None:
        raise ValueError("the fiducial has no active mode on this grid")
    f_lo, f_hi = grid.f0 + lo * grid.df, grid.f0 + (hi + 1) * grid.df
    f = np.exp(np.linspace(np.log(f_lo), np.log(f_hi), n_rb + 1))
    j = np.clip(np.rint((f - grid.f0) / grid.df).astype(np.int64), lo, hi + 1)
    return np.unique(np.concatenate([j, marks, [lo, hi + 1]]))


def summary(th_fid, t0, modes, grid, e, d, psd, chunk=200000):
    """A0, A1 [L, 3, nb] and B0, B1 [L, L, 3, nb] (complex) and <d|d>."""
    L, nb = len(modes), len(e) - 1
    A0 = np.zeros((L, 3, nb), complex)
    A1 = np.zeros_like(A0)
    B0 = np.zeros((L, L, 3, nb), complex)
    B1 = np.zeros_like(B0)
    jlo, jend = int(e[0]), int(e[-1])
    for s in range(jlo, jend, chunk):
        j = np.arange(s, min(s + chunk, jend))
        f = grid.f0 + j * grid.df
        b = np.clip(np.searchsorted(e, j, side="right") - 1, 0, nb - 1)
        fb = grid.f0 + e[b] * grid.df
        w = 4.0 * grid.df / psd[:, j]
        h0 = np.array([O.mode_response(th_fid, t0, l, m, grid.f0, grid.df, grid.n_bins, f)
                       for (l, m) in modes])                     # [L, 3, n]
        dd = d[:, j]
        for a in range(L):
            x = w * dd * np.conj(h0[a])
            for c in range(3):
                A0[a, c] += np.bincount(b, x[c].real, nb) + 1j * np.bincount(b, x[c].imag, nb)
                y = x[c] * (f - fb)
                A1[a, c] += np.bincount(b, y.real, nb) + 1j * np.bincount(b, y.imag, nb)
            for a2 in range(L):
                x = w * h0[a] * np.conj(h0[a2])
                for c in range(3):
                    B0[a, a2, c] += np.bincount(b, x[c].real, nb) + 1j * np.bincount(b, x[c].imag, nb)
                    y = x[c] * (f - fb)
                    B1[a, a2, c] += np.bincount(b, y.real, nb) + 1j * np.bincount(b, y.imag, nb)
    return A0, A1, B0, B1


def bin_ratios(th, th_fid, t0, modes, grid, e):
    """r0, r1 [L, 3, nb] by the edge rule above."""
    f = grid.f0 + e * grid.df
    R0, R1 = [], []
    for (l, m) in modes:
        h = O.mode_response(th, t0, l, m, grid.f0, grid.df, grid.n_bins, f)
        h0 = O.mode_response(th_fid, t0, l, m, grid.f0, grid.df, grid.n_bins, f)
        ok = h0 != 0
        r = np.where(ok, h / np.where(ok, h0, 1.0), 0.0)
        okL, okR = ok[:, :-1], ok[:, 1:]
        rL, rR = r[:, :-1], r[:, 1:]
        both = okL & okR
        R0.append(np.where(okL, rL, np.where(okR, rR, 0.0)))
        R1.append(np.where(both, (rR - rL) / (f[1:] - f[:-1]), 0.0))
    return np.array(R0), np.array(R1)


def loglike(th, th_fid, t0, modes, grid, e, summ, dd):
    """ln L, <d|h>, <h|h> of one parameter vector by relative binning."""
    A0, A1, B0, B1 = summ
    r0, r1 = bin_ratios(th, th_fid, t0, modes, grid, e)
    dh = np.sum(A0 * np.conj(r0) + A1 * np.conj(r1)).real
    hh = 0.0
    L = len(modes)
    for a in range(L):
        for a2 in range(L):
            hh += np.sum(B0[a, a2] * r0[a] * np.conj(r0[a2])
                         + B1[a, a2] * (r0[a] * np.conj(r1[a2]) + r1[a] * np.conj(r0[a2]))).real
    return dh - 0.5 * hh - 0.5 * dd, dh, hh
