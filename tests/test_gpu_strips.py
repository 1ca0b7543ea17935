"""Strip contexts of the library (a lattice decomposed into strips of rows, halos moved by
rlbm_halo_pack / rlbm_halo_unpack between steps) against the same lattice as one context:
bit-identical fields and states in FP64, FP32 and FP16 (whose stochastic rounding is keyed
on the lattice's own rows), periodic in y and between walls with discs across strip edges,
strips of uneven heights (partial tile rows).  Misuse is refused."""
import os

import numpy as np
import pytest

from paper_2205_04658_gb300 import inputs

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


def _config(nx, ny, walls):
    e, ux, uy = inputs.smooth_random_fields(nx, ny, seed=nx + ny, eps_amp=0.02, u_amp=0.04, kmax=4)
    kw = dict(eta_over_s=0.05, kmin=2, kmax=5, force_amp=1e-3, seed=23, init_eps=e, init_ux=ux, init_uy=uy)
    if walls:
        mask = np.zeros((ny, nx), np.uint8)
        Y, X = np.mgrid[0:ny, 0:nx]
        for cx, cy in ((10, 33), (40, 66), (70, 20)):  # discs across the strip edges at rows 33 and 66
            mask[(X - cx) ** 2 + (Y - cy) ** 2 <= 9] = 1
        kw.update(walls_y=1, solid=mask, body_force=(2e-4, 0.0))
    return kw


@pytest.mark.parametrize("precision", ["f64", "f32", "f16"])
@pytest.mark.parametrize("walls", [0, 1])
def test_strips_equal_one_context(R, precision, walls):
    import torch
    from paper_2205_04658_gb300 import strips
    nx, ny, n = 96, 100, 30
    kw = _config(nx, ny, walls)
    stream = torch.cuda.Stream()
    one = R.Lattice(nx, ny, stream=stream, precision=precision, **kw)
    one.step(n)
    ref = one.moments()
    ref_state = one.get_state()[0]
    one.close()
    for nstrips in (3, 1):  # 33 / 33 / 34 rows, and one strip that is its own neighbour
        if walls and nstrips == 1:
            continue
        S = strips.StripSet(nx, ny, nstrips, stream=stream, precision=precision, **kw)
        S.step(n)
        assert S.current_step == n
        got = S.moments()
        for k in range(3):
            assert np.array_equal(got[k], ref[k]), (nstrips, k)
        assert np.abs(got[3] - ref[3]).max() <= 1e-12 * abs(ref[3][0])
        assert np.array_equal(S.get_state()[0], ref_state)
        S.close()


def test_strip_misuse_is_refused(R):
    import torch
    stream = torch.cuda.Stream()
    whole = R.Lattice(32, 32, stream=stream, precision="f32", eta_over_s=0.05)
    buf = torch.zeros(1 << 16, dtype=torch.uint8, device="cuda")  # a zero ghost row is the rest state
    with pytest.raises(R.RlbmError) as e:
        R.rlbm_halo_pack(whole.ctx, 0, buf.data_ptr())
    assert e.value.status == R.RLBM_E_INVAL and "whole lattice" in str(e.value)
    assert R.rlbm_halo_bytes(whole.ctx) == 0
    whole.close()
    # the bottom strip of a lattice between walls: face 0 is a wall
    s = R.Lattice(32, 16, stream=stream, precision="f32", eta_over_s=0.05, walls_y=1, strip_y0=0, strip_ny_total=48)
    # 6 crossing planes, one padded FP32 row each: 32 cells + 128-byte margin + ghost, in 128-byte lines
    assert R.rlbm_halo_bytes(s.ctx) == 6 * 96 * 4
    with pytest.raises(R.RlbmError) as e:
        R.rlbm_halo_unpack(s.ctx, 0, buf.data_ptr())
    assert e.value.status == R.RLBM_E_INVAL and "wall" in str(e.value)
    with pytest.raises(R.RlbmError) as e:  # the face above is not unpacked yet
        s.step(1)
    assert e.value.status == R.RLBM_E_STATE
    with pytest.raises(R.RlbmError) as e:
        R.rlbm_halo_unpack(s.ctx, 1, buf.data_ptr() + 8)  # misaligned
    assert e.value.status == R.RLBM_E_INVAL
    R.rlbm_halo_unpack(s.ctx, 1, buf.data_ptr())
    with pytest.raises(R.RlbmError) as e:
        s.step(2)
    assert e.value.status == R.RLBM_E_INVAL
    s.step(1)
    with pytest.raises(R.RlbmError) as e:  # the moments read the ghost rows of the current state
        s.moments()
    assert e.value.status == R.RLBM_E_STATE
    with pytest.raises(R.RlbmError) as e:
        s.spectrum(8)
    assert e.value.status == R.RLBM_E_INVAL
    s.close()
