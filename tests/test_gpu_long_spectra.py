"""Long-run statistics of the 16-bit storage forms: the time-averaged energy spectrum of
the stirred 1024 x 1024 run (shell 8 <= |k| <= 10, amplitude 1e-4, seed 2, eta/s 0.05)
over 20 000 steps, sampled every 500 steps after t = 32 (step 640), in the inverse-cascade
range 2 <= n < 8, against the FP32 run of the same workload (whose parity with the FP64
oracle is checked pointwise at 200 steps elsewhere; a 20 000-step oracle run of this
size would take hours on the host).  Bar: within 2 % in every bin.  FP16 (11-bit mantissa,
stochastic rounding) meets it; BF16 (8-bit mantissa) does not: the per-step forcing
increments of this workload sit below its resolution and the time-averaged spectrum
comes out tens of percent low.  Its value is asserted against a sanity bound only, so
that it stays reported."""
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

N, STEPS, EVERY, START = 1024, 20000, 500, 640


@pytest.fixture(scope="module")
def R():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2205_04658_gb300 import build as B
    from paper_2205_04658_gb300 import rlbm
    if not os.path.exists(rlbm.LIB_PATH):
        B.build()
    return rlbm


def _mean_spectrum(R, precision):
    lat = R.Lattice(N, N, precision=precision, eta_over_s=0.05, kmin=8, kmax=10, force_amp=1e-4, seed=2)
    acc = np.zeros(12)
    count = 0
    done = 0
    for target in range(START, STEPS + 1, EVERY):
        lat.step(target - done)
        done = target
        acc += lat.spectrum(12)
        count += 1
    lat.close()
    return acc / count


@pytest.fixture(scope="module")
def ref(R):
    return _mean_spectrum(R, "f32")


BF16_MISS = pytest.mark.xfail(strict=True, raises=AssertionError,
                              reason="BF16 deviation storage misses the 2 % bar on the time-averaged spectrum")


@pytest.mark.parametrize("precision", ["f16", pytest.param("bf16", marks=BF16_MISS)])
def test_time_averaged_inertial_spectrum_within_2_percent(R, ref, precision):
    got = _mean_spectrum(R, precision)
    rel = np.abs(got[2:8] / ref[2:8] - 1.0)
    print("%s: mean E(n), n = 2..7, relative to FP32: %s" % (precision, np.array2string(rel, precision=4)))
    assert np.all(ref[2:8] > 0.0)
    assert rel.max() <= 0.02


def test_long_run_analysis_pipeline(R):
    """The analysis of a long stirred run: spectra and filtered velocities sampled every
    18 steps from t = 32 on, time-averaged with their standard errors, and the slope of the
    averaged spectrum below the stirring shell (reported: the paper's -5/3 is qualitative,
    and this small forcing gives a weak cascade)."""
    from paper_2205_04658_gb300 import analysis as A
    lat = R.Lattice(N, N, precision="f32", eta_over_s=0.05, kmin=8, kmax=10, force_amp=1e-4, seed=2)
    out = A.sample_run(lat, nsamples=400, nbins=12, kf=8)
    lat.close()
    assert out["steps"][0] == A.SETTLE_STEP and np.all(np.diff(out["steps"]) == A.DECORRELATION_STEPS)
    mean, err = A.time_average(out["spectra"])
    assert np.all(np.isfinite(err)) and np.all(err[2:8] < mean[2:8])
    v = out["filtered_velocity"]
    assert np.all(v > 0.0)
    # the filter keeps every bin below the shell: its energy is at least that of bins 0..6
    # (round(|k|) <= 6 implies |k| < 8) at every sample
    assert np.all(0.5 * v ** 2 >= out["spectra"][:, :7].sum(axis=1) * (1 - 1e-12))
    slope = A.power_law_slope(np.arange(2, 8), mean[2:8])
    print("filtered velocity %.3e (first half %.3e, second half %.3e); slope of <E(n)>, n = 2..7: %.2f"
          % (np.sqrt(np.mean(v ** 2)), np.sqrt(np.mean(v[:200] ** 2)), np.sqrt(np.mean(v[200:] ** 2)), slope))
    assert np.isfinite(slope)
