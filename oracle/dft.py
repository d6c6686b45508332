"""Running discrete Fourier transform of Hz probe samples, FP64 oracle.

Test infrastructure: only the tests, the smoke check and the benchmark's CPU
baseline use this package.

The paper reports its results as frequency responses (Sec. VI: the cavity
and waveguide responses and the reflected power of the rod test), i.e.
spectra of probe fields.  A probe sample o^n = Hz^{n+1/2} belongs to the
half-step time t^{n+1/2} = (n + 1/2) dt (Eq. (5)), so the transform of the
samples n = n0 .. n0 + N - 1 at frequency f is the plain sum

    X(f) = sum_n o^n exp(-i 2 pi f t^{n+1/2}) dt .
"""
from __future__ import annotations

import numpy as np


def dft(samples, dt: float, freqs, n0: int = 0) -> np.ndarray:
    """samples [nsteps, nprobe] (step n0 first) -> X [nprobe, nfreq], complex."""
    o = np.asarray(samples, dtype=np.float64)
    if o.ndim == 1:
        o = o[:, None]
    f = np.asarray(freqs, dtype=np.float64)
    t = (n0 + np.arange(o.shape[0]) + 0.5) * dt
    X = np.zeros((o.shape[1], f.size), dtype=np.complex128)
    for k in range(f.size):
        X[:, k] = (np.exp(-2j * np.pi * f[k] * t) @ o) * dt
    return X
