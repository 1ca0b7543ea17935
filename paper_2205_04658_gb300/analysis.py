"""Long-run statistics of a stirred run (Part I, "Results"; appendix "Minimum Simulation
Time"): time-averaged energy spectra sampled at a decorrelation interval after the
spectrum has settled, their statistical error, the filtered (inertial-range) velocity,
and the power-law slope compared with Kolmogorov's -5/3.

The spectra and band energies come from the library (rlbm_spectrum, rlbm_band_energy);
this module only schedules the samples and reduces them on the host.

Readings:
  * samples every N = 18 steps (t = 0.9 at dt = 0.05), the decorrelation interval the
    paper settles on, from t = 32 (step 640), when its spectra have become stable;
  * the error of a time-averaged bin is the standard error of the mean over the M
    samples, sqrt((<E^2> - <E>^2) / M) (the printed formula, a mean of square roots of
    differences of squares, is garbled);
  * the velocity filter keeps the wave vectors below the stirring shell, |k|^2 < kmin^2,
    the range the paper calls inertial.
"""
import numpy as np

DECORRELATION_STEPS = 18   # N = t / dt with t = 0.9
SETTLE_STEP = 640          # t = 32 at dt = 0.05


def time_average(samples):
    """Mean and standard error of the mean of spectra samples (M x nbins)."""
    a = np.asarray(samples, dtype=np.float64)
    m = a.shape[0]
    mean = a.mean(axis=0)
    var = np.maximum((a * a).mean(axis=0) - mean * mean, 0.0)
    return mean, np.sqrt(var / m)


def power_law_slope(k, E):
    """Least-squares slope of log E against log k (bins with E > 0)."""
    k = np.asarray(k, dtype=np.float64)
    E = np.asarray(E, dtype=np.float64)
    sel = (k > 0) & (E > 0)
    if sel.sum() < 2:
        raise ValueError("need at least two positive bins")
    slope, _ = np.polyfit(np.log(k[sel]), np.log(E[sel]), 1)
    return float(slope)


def compensated(k, E, power=5.0 / 3.0):
    """E(k) k^power: flat where the spectrum follows k^-power."""
    return np.asarray(E, dtype=np.float64) * np.asarray(k, dtype=np.float64) ** power


def sample_run(lattice, nsamples, nbins, kf, every=DECORRELATION_STEPS, start=SETTLE_STEP):
    """Advance `lattice` (an rlbm.Lattice) to step `start`, then take `nsamples` samples
    `every` steps apart of its spectrum (nbins bins) and of its rms velocity filtered to
    |k| < kf.  Returns dict(steps, spectra (nsamples x nbins), filtered_velocity)."""
    if lattice.current_step < start:
        lattice.step(start - lattice.current_step)
    steps, spectra, vel = [], [], []
    for i in range(nsamples):
        if i:
            lattice.step(every)
        steps.append(lattice.current_step)
        spectra.append(lattice.spectrum(nbins))
        vel.append(lattice.filtered_velocity(kf))
    return dict(steps=np.array(steps), spectra=np.array(spectra), filtered_velocity=np.array(vel))


def current_density_run(lattice, nsteps, every=1, region=None):
    """Part II's current density: advance an open-channel `lattice` by `nsteps` steps,
    recording j_x at the outflow column every `every` steps (j(t)) and, at the end, j_x
    across the columns of `region` (slice; default: the downstream half) (j(x)).
    Returns dict(t_steps, j_t, j_x)."""
    steps, jt = [], []
    for i in range(0, nsteps, every):
        lattice.step(min(every, nsteps - i))
        jx, _ = lattice.column_means()
        steps.append(lattice.current_step)
        jt.append(jx[-1])
    jx, _ = lattice.column_means()
    if region is None:
        region = slice(lattice.nx // 2, lattice.nx)
    return dict(t_steps=np.array(steps), j_t=np.array(jt), j_x=jx[region])


def fluctuation_spectrum(signal):
    """|FFT|^2 of a signal's fluctuation about its mean, for the non-negative frequencies
    (j(omega) from j(t), j(k_x) from j(x))."""
    s = np.asarray(signal, dtype=np.float64)
    return np.abs(np.fft.rfft(s - s.mean())) ** 2
