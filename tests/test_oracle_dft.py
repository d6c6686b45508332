"""Pins for the oracle's running DFT of probe samples: an FFT library routine
at the bin frequencies, the closed form of a sampled cosine, and the Yee
dispersion relation (the spectral peak of a cavity mode lies within one bin
of its discrete angular frequency)."""
import numpy as np
import pytest

from oracle import dft, scheme, yee
from oracle.yee import C0

rng = np.random.default_rng(1609071)


@pytest.mark.parametrize("n0", [0, 37])
def test_bins_equal_fft(n0):
    """At f_k = k / (N dt): X(f_k) = dt exp(-i pi k (2 n0 + 1) / N) FFT(o)[k]."""
    N, dt = 256, 1.3e-12
    o = rng.standard_normal((N, 3))
    k = np.arange(0, 40)
    X = dft.dft(o, dt, k / (N * dt), n0=n0)
    F = np.fft.fft(o, axis=0)[k, :].T
    ref = dt * np.exp(-1j * np.pi * k * (2 * n0 + 1) / N)[None, :] * F
    assert np.abs(X - ref).max() < 1e-12 * np.abs(ref).max()


def test_sampled_cosine_closed_form():
    """o^n = cos(2 pi f0 t_n): each exponential sums as a geometric series,
    sum_{n<N} exp(i a (n + 1/2)) = exp(i a / 2)(1 - exp(i a N)) / (1 - exp(i a))."""
    N, dt, f0 = 500, 1e-12, 37e9
    t = (np.arange(N) + 0.5) * dt
    o = np.cos(2 * np.pi * f0 * t)
    f = np.linspace(1e9, 80e9, 23)

    def geo(a):
        return np.exp(0.5j * a) * (1 - np.exp(1j * a * N)) / (1 - np.exp(1j * a))

    ref = 0.5 * dt * (geo(2 * np.pi * (f0 - f) * dt) + geo(-2 * np.pi * (f0 + f) * dt))
    X = dft.dft(o, dt, f)[0]
    assert np.abs(X - ref).max() < 1e-10 * np.abs(ref).max()


def test_cavity_mode_peak_at_discrete_frequency():
    """P2: a lossless PEC-cavity mode (m, n) run through the oracle's time
    loop; |X(f)| of a probe peaks within one bin of
    w_mn = (2/dt) asin(c dt sqrt(sin^2(m pi/2nx)/dx^2 + sin^2(n pi/2ny)/dy^2))."""
    nx, ny, dx, dy, m, n = 20, 14, 1e-3, 1e-3, 7, 5
    dt = 0.9 * yee.cfl_limit(dx, dy)
    grid = yee.CoarseGrid(nx, ny, dx, dy, dt, np.ones((ny, nx)), np.zeros((ny, nx)))
    st = scheme.State(*grid.zeros())
    ii, jj = np.meshgrid(np.arange(nx), np.arange(ny))
    st.Hz = np.cos(m * np.pi * (ii + 0.5) / nx) * np.cos(n * np.pi * (jj + 0.5) / ny)
    N = 4000
    out = np.zeros((N, 1))
    for s in range(N):
        scheme.step(grid, st, [], (), s, [(0, 0)], out)
    w = (2 / dt) * np.arcsin(C0 * dt * np.sqrt(np.sin(m * np.pi / (2 * nx)) ** 2 / dx**2
                                               + np.sin(n * np.pi / (2 * ny)) ** 2 / dy**2))
    df = 1.0 / (N * dt)
    f = np.arange(0.25, 0.5 / dt * 0.999 / df) * df     # quarter-bin offset grid up to Nyquist
    X = np.abs(dft.dft(out, dt, f)[0])
    assert abs(f[np.argmax(X)] - w / (2 * np.pi)) <= df
    # the continuous-space cavity frequency is a different number at this mesh
    f_cont = C0 / 2 * np.sqrt((m / (nx * dx)) ** 2 + (n / (ny * dy)) ** 2)
    assert abs(f_cont - w / (2 * np.pi)) > 3 * df


def test_planted_whole_step_time_is_caught(monkeypatch):
    """Sampling at t^n instead of t^{n+1/2} (a plausible slip) fails the FFT pin."""
    N, dt = 64, 1e-12
    o = rng.standard_normal((N, 1))
    k = np.arange(1, 9)
    F = np.fft.fft(o, axis=0)[k, :].T
    ref = dt * np.exp(-1j * np.pi * k / N)[None, :] * F
    X = dft.dft(o, dt, k / (N * dt), n0=0)
    assert np.abs(X - ref).max() < 1e-12 * np.abs(ref).max()
    Xbad = dft.dft(o, dt, k / (N * dt), n0=0) * np.exp(1j * np.pi * k / N)[None, :]  # t^n sampling
    assert np.abs(Xbad - ref).max() > 1e-3 * np.abs(ref).max()
