"""The allocation-free spectrum entry point (rlbm_spectrum_noalloc) against the
context-based one (rlbm_spectrum).

rlbm_spectrum_noalloc serves callers that cannot call cudaMalloc (all device memory
owned by their own allocator or a fixed budget, or loops where cudaMalloc's implicit
device-wide synchronisation is unacceptable): its FFT work buffers live in a fixed
array inside the library.  This file is collected last on purpose, so that a run that
stops at its first failure has already run every other test."""
import os

import numpy as np
import pytest

from paper_2205_04658_gb300 import inputs


@pytest.fixture(scope="module")
def R():
    from paper_2205_04658_gb300 import build as B
    from paper_2205_04658_gb300 import rlbm
    if not os.path.exists(rlbm.LIB_PATH):
        B.build()
    return rlbm


def test_rejects_sizes_beyond_its_limit(R):
    """Checked before any CUDA call: works without a GPU."""
    with pytest.raises(R.RlbmError) as e:
        R.rlbm_spectrum_noalloc(0x1000, 0x2000, 1024, 1024, 16, 0x3000, 0)
    assert e.value.status == R.RLBM_E_INVAL and "131072" in str(e.value)
    with pytest.raises(R.RlbmError) as e:
        R.rlbm_spectrum_noalloc(0x1000, 0x2000, 64, 64, 9000, 0x3000, 0)
    assert e.value.status == R.RLBM_E_INVAL and "nbins" in str(e.value)


@pytest.mark.gpu
def test_matches_the_context_spectrum_on_two_calls_in_a_row(R):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    nbins = 70
    stream = torch.cuda.current_stream()
    for call, (nx, ny, seed) in enumerate(((96, 80, 1), (120, 64, 2))):
        e, ux, uy = inputs.smooth_random_fields(nx, ny, seed=seed, u_amp=0.05, kmax=6)
        lat = R.Lattice(nx, ny, precision="f64", eta_over_s=0.05, kmin=3, kmax=6, force_amp=1e-3, seed=seed,
                        init_eps=e, init_ux=ux, init_uy=uy)
        lat.step(10)
        _, UX, UY, _ = lat.moments()
        ref = lat.spectrum(nbins)
        lat.close()
        d_ux = torch.from_numpy(UX).cuda()
        d_uy = torch.from_numpy(UY).cuda()
        d_E = torch.full((nbins,), -1.0, dtype=torch.float64, device="cuda")
        R.rlbm_spectrum_noalloc(d_ux.data_ptr(), d_uy.data_ptr(), nx, ny, nbins, d_E.data_ptr(), stream.cuda_stream)
        torch.cuda.synchronize()
        got = d_E.cpu().numpy()
        assert np.abs(got - ref).max() <= 1e-10 * ref.max(), call


@pytest.mark.gpu
@pytest.mark.parametrize("nx,ny,nbins", [(512, 256, 400), (16384, 8, 8200), (16381, 8, 8200)])
def test_matches_the_context_spectrum_at_its_limits(R, nx, ny, nbins):
    """The edges of what the entry point accepts: all 2^17 cells (512 x 256), a row of 16384
    with every bin up to the top one (|k| = 8192 lands in bin 8192 of 8200), and a prime row
    length (16381: its transform is one stage of direct sums shared by a block's threads).
    Each against rlbm_spectrum of a context of the same shape holding the same fields."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    e, ux, uy = inputs.smooth_random_fields(nx, ny, seed=nx + ny, u_amp=0.05, kmax=3)
    rng = np.random.default_rng(nx)
    ux = ux + 1e-3 * rng.standard_normal((ny, nx))  # energy in every bin, the top one included
    uy = uy + 1e-3 * rng.standard_normal((ny, nx))
    lat = R.Lattice(nx, ny, precision="f64", eta_over_s=0.05, init_eps=e, init_ux=ux, init_uy=uy)
    _, UX, UY, _ = lat.moments()
    ref = lat.spectrum(nbins)
    lat.close()
    d_ux = torch.from_numpy(UX).cuda()
    d_uy = torch.from_numpy(UY).cuda()
    d_E = torch.full((nbins,), -1.0, dtype=torch.float64, device="cuda")
    for _ in range(2):
        R.rlbm_spectrum_noalloc(d_ux.data_ptr(), d_uy.data_ptr(), nx, ny, nbins, d_E.data_ptr(),
                                torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        got = d_E.cpu().numpy()
        assert np.abs(got - ref).max() <= 1e-10 * ref.max()
    top = int(round(np.hypot(nx // 2, ny // 2)))
    assert ref[top] > 0.0 and np.all(ref[top + 1:] == 0.0)
