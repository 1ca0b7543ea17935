"""FP16 storage holds 2^8 h: the round trip through rlbm_set_state / rlbm_get_state gives
exactly the FP16 numbers of 256 h divided by 256 (round to nearest even), so deviations far
below FP16's unscaled normal range (2^-14) keep FP16's relative precision; a value beyond the
stored range (|h| > 255.9) is stored as infinity and the next step reports it."""
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


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


def _scaled_fp16(h):
    """What FP16 storage of 256 h returns, in h: FP32 first (as the host packing does), then
    FP16 by round to nearest even."""
    return (np.asarray(h, np.float64) * 256.0).astype(np.float32).astype(np.float16).astype(np.float64) / 256.0


def test_state_round_trip_is_the_scaled_fp16_grid(R):
    nx, ny = 40, 24
    lat = R.Lattice(nx, ny, precision="f16", eta_over_s=0.05)
    q = R.rlbm_num_planes(lat.ctx)
    rng = np.random.default_rng(11)
    scales = np.array([3e-9, 1e-7, 4e-6, 1e-4, 3e-2, 2.0, 30.0])
    h = rng.normal(size=(q, ny, nx)) * scales[rng.integers(0, scales.size, size=(q, ny, nx))]
    lat.set_state(h, 5)
    got, step = lat.get_state()
    lat.close()
    assert step == 5
    assert np.array_equal(got, _scaled_fp16(h))
    # below 2^-14 unscaled FP16 would keep only multiples of 2^-24; the scaled form keeps
    # FP16's relative precision (2^-11) down to |h| = 2^-22
    small = (np.abs(h) >= 2.0 ** -22) & (np.abs(h) < 2.0 ** -14)
    assert small.sum() > 100
    rel = np.abs(got[small] - h[small]) / np.abs(h[small])
    assert rel.max() <= 2.0 ** -11
    unscaled = h[small].astype(np.float32).astype(np.float16).astype(np.float64)
    assert (np.abs(unscaled - h[small]) / np.abs(h[small])).max() > 2.0 ** -9


def test_value_beyond_the_stored_range_is_reported(R):
    lat = R.Lattice(32, 32, precision="f16", eta_over_s=0.1, rounding=1)
    h, step = lat.get_state()
    h[4, 10, 12] = 300.0  # 256 h = 76800 > 65504: stored as infinity
    lat.set_state(h, step)
    got, _ = lat.get_state()
    assert np.isinf(got[4, 10, 12])
    lat.step(2)
    with pytest.raises(R.RlbmError) as e:
        lat.sync()
    assert e.value.status == R.RLBM_E_UNSTABLE
    lat.close()
