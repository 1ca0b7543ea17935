"""Host-side checks of the C ABI that need no GPU: the library loads, exports every
entry point that include/rlbm.h declares, and validates configurations and sizes."""
import ctypes
import os
import re

import pytest

from paper_2205_04658_gb300 import build as B
from paper_2205_04658_gb300 import rlbm as R

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built():
    if not os.path.exists(R.LIB_PATH):
        B.build()
    R.lib()


def declared_symbols():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            src = open(os.path.join(ROOT, "include", h)).read()
            names |= set(re.findall(r"RLBM_API\s+[\w\s\*]+?\b(rlbm_\w+)\s*\(", src))
    return names


def test_every_declared_symbol_is_exported():
    names = declared_symbols()
    assert {"rlbm_init", "rlbm_step", "rlbm_moments", "rlbm_spectrum", "rlbm_free"} <= names
    L = ctypes.CDLL(R.LIB_PATH)
    for n in sorted(names):
        assert hasattr(L, n), n


def test_no_internal_symbols_leak():
    out = os.popen("nm -D --defined-only %s" % R.LIB_PATH).read()
    exported = {line.split()[-1] for line in out.splitlines() if " T " in line}
    assert exported <= declared_symbols(), exported - declared_symbols()


def test_workspace_size_scales_with_precision_and_lattice():
    sizes = {}
    for p in ("f64", "f32", "f16", "bf16"):
        cfg, _ = R.make_config(1024, 1024, precision=p, kmin=8, kmax=10, force_amp=1e-4)
        sizes[p] = R.rlbm_query_workspace(cfg)
    pop = {p: 2 * 17 * 1024 * 1024 * R.STORE_BYTES[p] for p in sizes}
    for p in sizes:
        assert sizes[p] > pop[p]
    assert sizes["f64"] - sizes["f32"] > pop["f32"] * 0.99
    cfg, _ = R.make_config(1000, 77, precision="f32")
    assert R.rlbm_query_workspace(cfg) % 256 == 0


@pytest.mark.parametrize("bad,msg", [
    (dict(nx=4), "nx and ny"),
    (dict(dt=0.2, a=0.1), "dt / a"),
    (dict(eta_over_s=0.0), "eta_over_s"),
    (dict(precision=7), "precision"),
    (dict(kmin=8, kmax=40, force_amp=1e-4), "kmax"),
    (dict(vset=2, body_force=(1e-3, 0.0)), "vset 3"),
    (dict(walls_y=2), "walls_y"),
    (dict(fp64_landau_vmax=1.5), "fp64_landau_vmax"),
    (dict(eps0=-1.0), "eps0"),
    (dict(open_x=2), "open_x"),
    (dict(open_x=1, inflow_ux=1.5), "inflow_ux"),
])
def test_invalid_configs_are_rejected(bad, msg):
    kw = dict(nx=64, ny=64, precision="f32")
    kw.update(bad)
    cfg, _ = R.make_config(**kw)
    with pytest.raises(R.RlbmError) as e:
        R.rlbm_query_workspace(cfg)
    assert e.value.status == R.RLBM_E_INVAL and msg in str(e.value)


def test_init_rejects_bad_workspace_without_touching_the_gpu():
    cfg, _ = R.make_config(64, 64)
    n = R.rlbm_query_workspace(cfg)
    with pytest.raises(R.RlbmError) as e:
        R.rlbm_init(cfg, 0, n, 0)
    assert e.value.status == R.RLBM_E_INVAL
    with pytest.raises(R.RlbmError) as e:
        R.rlbm_init(cfg, 0x1000, n - 1, 0)
    assert e.value.status == R.RLBM_E_NOMEM
    with pytest.raises(R.RlbmError) as e:
        R.rlbm_init(cfg, 0x1001, n, 0)
    assert "aligned" in str(e.value)


def test_null_context_calls_fail_cleanly():
    L = R.lib()
    assert L.rlbm_step(None, 1) == R.RLBM_E_INVAL
    assert L.rlbm_wait_selftest(None, 1000) == R.RLBM_E_INVAL
    assert L.rlbm_current_step(None) == -1
    assert L.rlbm_num_planes(None) == -1
    L.rlbm_free(None)
    assert isinstance(R.rlbm_last_error(None), str)
