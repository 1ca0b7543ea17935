"""ctypes binding of librlbm.so (include/rlbm.h), the GB300 relativistic lattice
Boltzmann library.  Argument marshalling only: every step of the update runs in
the library's CUDA kernels.  PyTorch provides the device workspace and the stream.

The functions keep the C names (rlbm_init, rlbm_step, rlbm_moments, ...); the
``Lattice`` class bundles a workspace, a stream and a context.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "librlbm.so")

RLBM_OK, RLBM_E_INVAL, RLBM_E_NOMEM, RLBM_E_CUDA = 0, 1, 2, 3
RLBM_E_UNSTABLE, RLBM_E_UNPHYSICAL, RLBM_E_TIMEOUT, RLBM_E_STATE = 4, 5, 6, 7
PRECISION = {"f64": 0, "f32": 1, "f16": 2, "bf16": 3}
STORE_BYTES = {"f64": 8, "f32": 4, "f16": 2, "bf16": 2}


class RlbmError(RuntimeError):
    def __init__(self, status, message):
        super().__init__("rlbm status %d: %s" % (status, message))
        self.status = status


class rlbm_config(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("walls_y", ctypes.c_int32),
        ("vset", ctypes.c_int32), ("precision", ctypes.c_int32), ("rounding", ctypes.c_int32),
        ("a", ctypes.c_double), ("dt", ctypes.c_double), ("eta_over_s", ctypes.c_double),
        ("eps0", ctypes.c_double), ("body_force", ctypes.c_double * 2),
        ("kmin", ctypes.c_int32), ("kmax", ctypes.c_int32), ("force_amp", ctypes.c_double),
        ("seed", ctypes.c_uint64), ("solid", ctypes.POINTER(ctypes.c_uint8)),
        ("init_eps", ctypes.POINTER(ctypes.c_double)), ("init_ux", ctypes.POINTER(ctypes.c_double)),
        ("init_uy", ctypes.POINTER(ctypes.c_double)), ("fp64_landau_vmax", ctypes.c_double),
        ("open_x", ctypes.c_int32), ("inflow_ux", ctypes.c_double),
        ("strip_y0", ctypes.c_int32), ("strip_ny_total", ctypes.c_int32),
        ("strip_solid_halo", ctypes.POINTER(ctypes.c_uint8)),
    ]


_lib = None


def lib():
    """The loaded library; raises if it has not been built (there is no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("librlbm.so is not built (%s); run paper_2205_04658_gb300.build.build()" % LIB_PATH)
        L = ctypes.CDLL(LIB_PATH)
        P, c_i32, c_i64, c_sz = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_size_t
        dp = ctypes.POINTER(ctypes.c_double)
        sig = {
            "rlbm_query_workspace": (c_i32, [ctypes.POINTER(rlbm_config), ctypes.POINTER(c_sz)]),
            "rlbm_init": (c_i32, [ctypes.POINTER(rlbm_config), P, c_sz, P, ctypes.POINTER(P)]),
            "rlbm_step": (c_i32, [P, c_i64]),
            "rlbm_moments": (c_i32, [P, dp, dp, dp, dp]),
            "rlbm_spectrum": (c_i32, [P, c_i32, dp]),
            "rlbm_band_energy": (c_i32, [P, c_i64, c_i64, dp]),
            "rlbm_column_means": (c_i32, [P, dp, dp]),
            "rlbm_get_state": (c_i32, [P, dp, ctypes.POINTER(c_i64)]),
            "rlbm_set_state": (c_i32, [P, dp, c_i64]),
            "rlbm_num_planes": (c_i32, [P]),
            "rlbm_set_launch": (c_i32, [P, c_i32, c_i32, c_i32]),
            "rlbm_autotune": (c_i32, [P, c_i32, dp]),
            "rlbm_velocity_classes": (c_i32, [c_i32, dp]),
            "rlbm_batch_query_workspace": (c_i32, [c_i32, ctypes.POINTER(c_sz)]),
            "rlbm_batch_init": (c_i32, [ctypes.POINTER(P), c_i32, P, c_sz, P, ctypes.POINTER(P)]),
            "rlbm_batch_set_launch": (c_i32, [P, c_i32, c_i32]),
            "rlbm_batch_step": (c_i32, [P, c_i64]),
            "rlbm_batch_autotune": (c_i32, [P, c_i32, dp]),
            "rlbm_batch_last_error": (ctypes.c_char_p, [P]),
            "rlbm_batch_free": (None, [P]),
            "rlbm_spectrum_noalloc": (c_i32, [P, P, c_i32, c_i32, c_i32, P, P]),
            "rlbm_halo_bytes": (c_i32, [P, ctypes.POINTER(c_sz)]),
            "rlbm_halo_pack": (c_i32, [P, c_i32, P]),
            "rlbm_halo_unpack": (c_i32, [P, c_i32, P]),
            "rlbm_num_modes": (c_i32, [P]),
            "rlbm_set_mode_scale": (c_i32, [P, dp, c_i32]),
            "rlbm_gradient_query_workspace": (c_i32, [P, c_i64, c_i32, ctypes.POINTER(c_sz)]),
            "rlbm_gradient": (c_i32, [P, c_i64, c_i32, P, c_sz, dp, dp, dp, dp]),
            "rlbm_sync": (c_i32, [P]),
            "rlbm_wait_selftest": (c_i32, [P, c_i64]),
            "rlbm_current_step": (c_i64, [P]),
            "rlbm_last_error": (ctypes.c_char_p, [P]),
            "rlbm_free": (None, [P]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _check(status, ctx=None):
    if status != RLBM_OK:
        raise RlbmError(status, lib().rlbm_last_error(ctx).decode())


def _dptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def make_config(nx, ny, precision="f32", walls_y=0, vset=3, a=0.1, dt=0.05, eta_over_s=0.1, eps0=1.0,
                body_force=(0.0, 0.0), kmin=0, kmax=0, force_amp=0.0, seed=0, solid=None,
                init_eps=None, init_ux=None, init_uy=None, fp64_landau_vmax=0.0, rounding="stochastic",
                open_x=0, inflow_ux=0.0, strip_y0=0, strip_ny_total=0, strip_solid_halo=None):
    """An rlbm_config and the host arrays it points to (keep both alive until rlbm_init
    returns)."""
    keep = {}

    def arr(x, dtype, name, rows=ny):
        if x is None:
            return None
        a_ = np.ascontiguousarray(np.asarray(x, dtype=dtype).reshape(rows, nx))
        keep[name] = a_
        return a_.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8 if dtype == np.uint8 else ctypes.c_double))

    c = rlbm_config()
    c.nx, c.ny, c.walls_y, c.vset = nx, ny, int(walls_y), int(vset)
    c.precision = PRECISION[precision] if isinstance(precision, str) else int(precision)
    c.rounding = {"stochastic": 0, "nearest": 1}[rounding] if isinstance(rounding, str) else int(rounding)
    c.a, c.dt, c.eta_over_s, c.eps0 = a, dt, eta_over_s, eps0
    c.body_force[0], c.body_force[1] = body_force
    c.kmin, c.kmax, c.force_amp, c.seed = int(kmin), int(kmax), float(force_amp), int(seed)
    c.solid = arr(solid, np.uint8, "solid")
    c.init_eps = arr(init_eps, np.float64, "eps")
    c.init_ux = arr(init_ux, np.float64, "ux")
    c.init_uy = arr(init_uy, np.float64, "uy")
    c.fp64_landau_vmax = fp64_landau_vmax
    c.open_x, c.inflow_ux = int(open_x), float(inflow_ux)
    c.strip_y0, c.strip_ny_total = int(strip_y0), int(strip_ny_total)
    c.strip_solid_halo = arr(strip_solid_halo, np.uint8, "solid_halo", rows=2)
    return c, keep


# ----- C names ---------------------------------------------------------------
def rlbm_query_workspace(cfg):
    n = ctypes.c_size_t(0)
    _check(lib().rlbm_query_workspace(ctypes.byref(cfg), ctypes.byref(n)))
    return n.value


def rlbm_init(cfg, dev_workspace, nbytes, cuda_stream):
    ctx = ctypes.c_void_p()
    _check(lib().rlbm_init(ctypes.byref(cfg), ctypes.c_void_p(dev_workspace), nbytes,
                           ctypes.c_void_p(cuda_stream), ctypes.byref(ctx)))
    return ctx


def rlbm_step(ctx, nsteps):
    _check(lib().rlbm_step(ctx, int(nsteps)), ctx)


def rlbm_moments(ctx, eps=None, ux=None, uy=None, totals=None):
    _check(lib().rlbm_moments(ctx, _dptr(eps), _dptr(ux), _dptr(uy), _dptr(totals)), ctx)


def rlbm_spectrum(ctx, nbins, E):
    _check(lib().rlbm_spectrum(ctx, int(nbins), _dptr(E)), ctx)


def rlbm_band_energy(ctx, k2lo, k2hi):
    E = np.zeros(1)
    _check(lib().rlbm_band_energy(ctx, int(k2lo), int(k2hi), _dptr(E)), ctx)
    return E[0]


def rlbm_column_means(ctx, jx=None, jy=None):
    _check(lib().rlbm_column_means(ctx, _dptr(jx), _dptr(jy)), ctx)


def rlbm_get_state(ctx, host):
    step = ctypes.c_int64(0)
    _check(lib().rlbm_get_state(ctx, _dptr(host), ctypes.byref(step)), ctx)
    return step.value


def rlbm_set_state(ctx, host, step):
    _check(lib().rlbm_set_state(ctx, _dptr(host), int(step)), ctx)


def rlbm_num_planes(ctx):
    return lib().rlbm_num_planes(ctx)


def rlbm_set_launch(ctx, ctas, stages=0, stir_rows=0):
    _check(lib().rlbm_set_launch(ctx, int(ctas), int(stages), int(stir_rows)), ctx)


def rlbm_autotune(ctx, reps=10):
    ms = ctypes.c_double(0.0)
    _check(lib().rlbm_autotune(ctx, int(reps), ctypes.byref(ms)), ctx)
    return ms.value


def rlbm_spectrum_noalloc(d_ux, d_uy, nx, ny, nbins, d_E, cuda_stream):
    """Spectrum of device velocity fields (device pointers as integers), allocating nothing."""
    _check(lib().rlbm_spectrum_noalloc(ctypes.c_void_p(d_ux), ctypes.c_void_p(d_uy), int(nx), int(ny), int(nbins),
                                       ctypes.c_void_p(d_E), ctypes.c_void_p(cuda_stream)))


def rlbm_halo_bytes(ctx):
    n = ctypes.c_size_t(0)
    _check(lib().rlbm_halo_bytes(ctx, ctypes.byref(n)), ctx)
    return n.value


def rlbm_halo_pack(ctx, face, dev_out):
    _check(lib().rlbm_halo_pack(ctx, int(face), ctypes.c_void_p(dev_out)), ctx)


def rlbm_halo_unpack(ctx, face, dev_in):
    _check(lib().rlbm_halo_unpack(ctx, int(face), ctypes.c_void_p(dev_in)), ctx)


def rlbm_velocity_classes(vset=3):
    """(Q, 4) array of (v_x, v_y, v_z^2, w) of the folded classes (plane order of get/set_state)."""
    q = lib().rlbm_velocity_classes(int(vset), None)
    out = np.empty(4 * q)
    lib().rlbm_velocity_classes(int(vset), _dptr(out))
    return out.reshape(q, 4)


def rlbm_num_modes(ctx):
    return lib().rlbm_num_modes(ctx)


def rlbm_set_mode_scale(ctx, sigma):
    s_ = np.ascontiguousarray(sigma, dtype=np.float64).ravel()
    _check(lib().rlbm_set_mode_scale(ctx, _dptr(s_), int(s_.size)), ctx)


def rlbm_gradient_query_workspace(ctx, nsteps, segment=0):
    n = ctypes.c_size_t(0)
    st = lib().rlbm_gradient_query_workspace(ctx, int(nsteps), int(segment), ctypes.byref(n))
    if st != RLBM_OK:
        raise RlbmError(st, lib().rlbm_last_error(None).decode())
    return n.value


def rlbm_gradient(ctx, nsteps, segment, dev_workspace, nbytes):
    """(J, dJ/dsigma (nmodes,), dJ/d(eta/s), dJ/dF_body (2,))."""
    J = np.zeros(1)
    gs = np.zeros(max(1, rlbm_num_modes(ctx)))
    ge = np.zeros(1)
    gb = np.zeros(2)
    _check(lib().rlbm_gradient(ctx, int(nsteps), int(segment), ctypes.c_void_p(dev_workspace), nbytes,
                               _dptr(J), _dptr(gs), _dptr(ge), _dptr(gb)), ctx)
    return J[0], gs[:rlbm_num_modes(ctx)], ge[0], gb


def rlbm_sync(ctx):
    _check(lib().rlbm_sync(ctx), ctx)


def rlbm_wait_selftest(ctx, max_cycles):
    """Queue the bounded-wait self-test: the next syncing call raises RLBM_E_TIMEOUT."""
    _check(lib().rlbm_wait_selftest(ctx, int(max_cycles)), ctx)


def rlbm_current_step(ctx):
    return lib().rlbm_current_step(ctx)


def rlbm_last_error(ctx=None):
    return lib().rlbm_last_error(ctx).decode()


def rlbm_free(ctx):
    lib().rlbm_free(ctx)


# ----- convenience -----------------------------------------------------------
class Lattice:
    """A lattice on the current CUDA device: a torch-allocated workspace, a stream
    (torch's current stream unless one is given) and a library context."""

    def __init__(self, nx, ny, stream=None, **kw):
        import torch
        self.nx, self.ny = nx, ny
        cfg, keep = make_config(nx, ny, **kw)
        self.nbytes = rlbm_query_workspace(cfg)
        self._ws = torch.empty(self.nbytes + 256, dtype=torch.uint8, device="cuda")
        base = self._ws.data_ptr()
        self.ptr = (base + 255) // 256 * 256
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.ctx = rlbm_init(cfg, self.ptr, self.nbytes, self.stream.cuda_stream)
        del keep

    def step(self, n=1):
        rlbm_step(self.ctx, n)

    def moments(self):
        e = np.empty((self.ny, self.nx))
        ux = np.empty_like(e)
        uy = np.empty_like(e)
        tot = np.empty(4)
        rlbm_moments(self.ctx, e, ux, uy, tot)
        return e, ux, uy, tot

    def totals(self):
        tot = np.empty(4)
        rlbm_moments(self.ctx, None, None, None, tot)
        return tot

    def spectrum(self, nbins):
        E = np.empty(nbins)
        rlbm_spectrum(self.ctx, nbins, E)
        return E

    def band_energy(self, k2lo, k2hi=0):
        """(1/2) sum of |v^(k)|^2 / (nx ny)^2 over k2lo <= |k|^2 < k2hi (k2hi <= 0: unbounded)."""
        return rlbm_band_energy(self.ctx, k2lo, k2hi)

    def column_means(self):
        """(j_x, j_y): column means of v = u / u^0, nx values each."""
        jx = np.empty(self.nx)
        jy = np.empty(self.nx)
        rlbm_column_means(self.ctx, jx, jy)
        return jx, jy

    def filtered_velocity(self, kf):
        """rms velocity of the field filtered to |k| < kf (the range below a stirring shell)."""
        return float(np.sqrt(2.0 * self.band_energy(0, kf * kf)))

    def get_state(self):
        q = rlbm_num_planes(self.ctx)
        h = np.empty((q, self.ny, self.nx))
        step = rlbm_get_state(self.ctx, h)
        return h, step

    def set_state(self, h, step):
        rlbm_set_state(self.ctx, np.ascontiguousarray(h, dtype=np.float64), step)

    @property
    def current_step(self):
        return rlbm_current_step(self.ctx)

    def set_launch(self, ctas, stages=0, stir_rows=0):
        rlbm_set_launch(self.ctx, ctas, stages, stir_rows)

    def autotune(self, reps=10):
        return rlbm_autotune(self.ctx, reps)

    @property
    def num_modes(self):
        return rlbm_num_modes(self.ctx)

    def set_mode_scale(self, sigma):
        rlbm_set_mode_scale(self.ctx, sigma)

    def gradient(self, nsteps, segment=0):
        """Runs nsteps steps and the adjoint: (J, dJ/dsigma, dJ/d(eta/s), dJ/dF_body).
        The checkpoint workspace is allocated by torch for the call."""
        import torch
        nbytes = rlbm_gradient_query_workspace(self.ctx, nsteps, segment)
        ws = torch.empty(nbytes + 256, dtype=torch.uint8, device="cuda")
        ptr = (ws.data_ptr() + 255) // 256 * 256
        with torch.cuda.stream(self.stream):
            out = rlbm_gradient(self.ctx, nsteps, segment, ptr, nbytes)
        del ws
        return out

    def sync(self):
        rlbm_sync(self.ctx)

    def close(self):
        if getattr(self, "ctx", None) is not None:
            rlbm_free(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ----- batches -----------------------------------------------------------------
def _bcheck(status, b=None):
    if status != RLBM_OK:
        raise RlbmError(status, lib().rlbm_batch_last_error(b).decode())


def rlbm_batch_query_workspace(nmembers):
    n = ctypes.c_size_t(0)
    _bcheck(lib().rlbm_batch_query_workspace(int(nmembers), ctypes.byref(n)))
    return n.value


def rlbm_batch_init(ctxs, dev_workspace, nbytes, cuda_stream):
    arr = (ctypes.c_void_p * len(ctxs))(*[c.value for c in ctxs])
    b = ctypes.c_void_p()
    _bcheck(lib().rlbm_batch_init(arr, len(ctxs), ctypes.c_void_p(dev_workspace), nbytes,
                                  ctypes.c_void_p(cuda_stream), ctypes.byref(b)))
    return b


def rlbm_batch_set_launch(b, ctas, stages=0):
    _bcheck(lib().rlbm_batch_set_launch(b, int(ctas), int(stages)), b)


def rlbm_batch_step(b, nsteps):
    _bcheck(lib().rlbm_batch_step(b, int(nsteps)), b)


def rlbm_batch_autotune(b, reps=5):
    ms = ctypes.c_double(0.0)
    _bcheck(lib().rlbm_batch_autotune(b, int(reps), ctypes.byref(ms)), b)
    return ms.value


def rlbm_batch_free(b):
    lib().rlbm_batch_free(b)


class Batch:
    """Lattices advanced together, one persistent launch per step.  The lattices should
    live on the batch's stream (a non-default stream enables CUDA-graph replay)."""

    def __init__(self, lattices, stream=None):
        import torch
        self.lattices = list(lattices)
        self.stream = stream if stream is not None else self.lattices[0].stream
        self.nbytes = rlbm_batch_query_workspace(len(self.lattices))
        self._ws = torch.empty(self.nbytes + 256, dtype=torch.uint8, device="cuda")
        ptr = (self._ws.data_ptr() + 255) // 256 * 256
        self.b = rlbm_batch_init([l.ctx for l in self.lattices], ptr, self.nbytes, self.stream.cuda_stream)

    def step(self, n=1):
        rlbm_batch_step(self.b, n)

    def set_launch(self, ctas, stages=0):
        rlbm_batch_set_launch(self.b, ctas, stages)

    def autotune(self, reps=5):
        return rlbm_batch_autotune(self.b, reps)

    def close(self):
        if getattr(self, "b", None) is not None:
            rlbm_batch_free(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
