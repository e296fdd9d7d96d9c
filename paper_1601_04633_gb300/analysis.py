"""Analysis of the mean hot-wall Nusselt number history Nu(t) (host side).

The paper reports, for each case of Table 1 (Sec. 4), whether the mean Nusselt
number reaches a steady value or oscillates, and for oscillating cases the
mean, amplitude and period, with time measured by the Fourier number
Fo = alpha t / H^2 (Eq. 20). This module computes those statistics from a
per-step series. The period is that of the dominant spectral peak; a second
estimate is the mean spacing of upward crossings, located by linear
interpolation between steps: first of the window mean (or, if the record
drifts too much for that, of its linear trend), then, to separate the
oscillation from any slow wave or drift, of the moving average over one such
period. The amplitude is half the peak-to-peak range of the oscillation about
that moving average; the drift is the mean of the last fifth of the window
minus that of the first fifth.
"""
from __future__ import annotations

from dataclasses import dataclass, asdict

import numpy as np


def dominant_period(f, x, min_samples=5, max_fraction=1.0 / 3.0):
    """Period (in the units of f) of the largest spectral peak of x(f): linear trend
    removed, Hann window, zero-padded 8x FFT, parabolic interpolation of the
    log-magnitude around the peak. Periods shorter than ``min_samples`` samples
    or longer than ``max_fraction`` of the record are ignored. None if no peak."""
    x = np.asarray(x, dtype=np.float64)
    n = len(x)
    if n < 16:
        return None
    dt = float(f[1] - f[0])
    t = np.arange(n)
    x = x - np.polyval(np.polyfit(t, x, 1), t)
    X = np.abs(np.fft.rfft(x * np.hanning(n), n=8 * n))
    fr = np.fft.rfftfreq(8 * n, d=dt)
    ok = (fr > 1.0 / (max_fraction * n * dt)) & (fr < 1.0 / (min_samples * dt))
    if not ok.any() or X[ok].max() <= 0:
        return None
    k = int(np.nonzero(ok)[0][np.argmax(X[ok])])
    if 0 < k < len(X) - 1 and X[k - 1] > 0 and X[k + 1] > 0:
        a, b, c = np.log(X[k - 1]), np.log(X[k]), np.log(X[k + 1])
        shift = 0.5 * (a - c) / (a - 2 * b + c) if (a - 2 * b + c) != 0 else 0.0
    else:
        shift = 0.0
    freq = fr[k] + shift * (fr[1] - fr[0])
    return float(1.0 / freq) if freq > 0 else None


@dataclass
class NuStats:
    steady: bool
    mean: float
    amplitude: float          # half the peak-to-peak range of the oscillation
    peak_to_peak: float
    period_fo: float | None   # dominant spectral period in Fo; None when steady
    crossing_period_fo: float | None  # mean spacing of upward crossings (see above)
    cycles: int               # complete cycles seen in the window
    window_fo: tuple          # (start, end) of the analysed window in Fo
    drift: float              # mean of the last fifth of the window minus the first fifth

    def as_dict(self):
        return asdict(self)


def fourier_number(steps, alpha: float, H: float):
    """Fo = alpha t / H^2 (Eq. 20) for step counts t (lattice units, dt = 1)."""
    return alpha * np.asarray(steps, dtype=np.float64) / (H * H)


def _crossing_period(f, d):
    """Mean spacing of upward zero crossings of d(f), and the number of complete cycles."""
    up = np.nonzero((d[:-1] < 0) & (d[1:] >= 0))[0]
    if len(up) < 2:
        return None, 0
    t = f[up] + (f[up + 1] - f[up]) * (-d[up]) / (d[up + 1] - d[up])
    return float((t[-1] - t[0]) / (len(t) - 1)), len(t) - 1


def nu_statistics(series, fo_per_step: float, window_fo: float | None = None,
                  steady_tol: float = 1e-3) -> NuStats:
    """Statistics of Nu over the last ``window_fo`` Fourier units of ``series``.

    series[k] is the mean Nu after step k + 1. The record counts as steady when the
    peak-to-peak range of its residual about a cubic fit over the window is below
    ``steady_tol`` times the mean (a settled or monotonically settling record).
    """
    nu = np.asarray(series, dtype=np.float64)
    n = len(nu)
    if n < 4:
        raise ValueError("need at least 4 samples")
    fo = (np.arange(n) + 1) * fo_per_step
    if window_fo is None:
        start = n // 2
    else:
        start = max(0, n - int(round(window_fo / fo_per_step)))
    w = nu[start:]
    f = fo[start:]
    mean = float(w.mean())
    p2p = float(w.max() - w.min())
    tt = (f - f[0]) / max(f[-1] - f[0], 1e-300)
    resid = w - np.polyval(np.polyfit(tt, w, 3), tt)
    # steady, or converging without oscillating: the record leaves only a tiny
    # residual about a smooth (cubic) trend over the window
    steady = float(resid.max() - resid.min()) <= steady_tol * abs(mean)
    fifth = max(1, len(w) // 5)
    drift = float(w[-fifth:].mean() - w[:fifth].mean())
    period, cycles, amplitude = None, 0, 0.5 * p2p
    if not steady:
        period, cycles = _crossing_period(f, w - mean)
        if period is None or cycles < 2:
            trend = np.polyval(np.polyfit(f - f[0], w, 1), f - f[0])
            period, cycles = _crossing_period(f, w - trend)
        if period is not None:
            L = int(round(period / fo_per_step))
            if 2 <= L < len(w) // 2:
                # centred moving average over one period (valid part only)
                c = np.cumsum(np.concatenate([[0.0], w]))
                ma = (c[L:] - c[:-L]) / L
                off = L // 2
                seg = w[off:off + len(ma)]
                fseg = f[off:off + len(ma)]
                p2, c2 = _crossing_period(fseg, seg - ma)
                if p2 is not None:
                    period, cycles = p2, c2
                    amplitude = 0.5 * float((seg - ma).max() - (seg - ma).min())
    spectral = None if steady else dominant_period(f, w)
    return NuStats(steady=bool(steady), mean=mean, amplitude=amplitude if not steady else 0.0,
                   peak_to_peak=p2p, period_fo=spectral, crossing_period_fo=period if not steady else None,
                   cycles=cycles if not steady else 0, window_fo=(float(f[0]), float(f[-1])), drift=drift)


# The four cases of the paper's Table 1 (Sec. 4): (Ra, Pr).
PAPER_CASES = {1: (1e4, 0.01), 2: (5e4, 0.01), 3: (5e4, 0.005), 4: (1e5, 0.01)}


def run_case(case: int, n: int, alpha: float, fo_end: float = 4.0, window_fo: float = 2.0, seed=None,
             device="cuda"):
    """One of the paper's cases on the GPU: an n x n cavity at lattice thermal
    diffusivity alpha (which sets the Mach number, Ma = sqrt(3) alpha
    sqrt(Ra Pr) / n, through Eqs. 9 and 21), run to Fourier number fo_end; the
    statistics of its mean-Nu history over the last window_fo."""
    from . import dmrt as D
    from . import inputs

    Ra, Pr = PAPER_CASES[case]
    steps = int(round(fo_end * n * n / alpha))
    cav = inputs.Cavity(n, n, Ra, Pr, alpha=alpha, seed=10 + case if seed is None else seed)
    sim = D.Cavity2D.from_inputs(cav, nu_capacity=steps, device=device)
    sim.step(steps)
    sim.check()
    series = sim.nusselt(steps)[2]
    ma = sim.consts.Ma
    sim.close()
    s = nu_statistics(series, alpha / (n * n), window_fo=window_fo)
    out = {"case": case, "Ra": Ra, "Pr": Pr, "n": n, "alpha": alpha, "Ma": ma, "steps": steps}
    out.update(s.as_dict())
    return out


def main():
    import argparse
    import json

    ap = argparse.ArgumentParser(description="Statistics of the paper's cases (Table 1) on the GPU, "
                                             "over grids and lattice diffusivities (Mach numbers).")
    ap.add_argument("--cases", type=int, nargs="+", default=[2, 3, 4])
    ap.add_argument("--n", type=int, nargs="+", default=[128])
    ap.add_argument("--alpha", type=float, nargs="+", default=[0.05, 0.1, 0.14])
    ap.add_argument("--fo", type=float, default=4.0, help="Fourier number to run to")
    ap.add_argument("--window", type=float, default=2.0, help="analysis window (Fo) at the end of the run")
    args = ap.parse_args()
    for n in args.n:
        for alpha in args.alpha:
            for case in args.cases:
                print(json.dumps(run_case(case, n, alpha, args.fo, args.window)), flush=True)


if __name__ == "__main__":
    main()
