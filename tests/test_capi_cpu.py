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


def declared_prototypes():
    protos = {}
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            src = open(os.path.join(ROOT, "include", h)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            for name, args in re.findall(r"RLBM_API\s+[\w\s\*]+?\b(rlbm_\w+)\s*\(([^)]*)\)", src, flags=re.S):
                args = args.strip()
                protos[name] = 0 if args in ("", "void") else args.count(",") + 1
    return protos


def test_binding_signatures_match_the_header():
    """Every declared entry point has a ctypes signature with the header's argument count."""
    L = R.lib()
    for name, nargs in declared_prototypes().items():
        fn = getattr(L, name)
        assert fn.argtypes is not None, name
        assert len(fn.argtypes) == nargs, (name, len(fn.argtypes), nargs)


def test_config_struct_layout_matches_the_header(tmp_path):
    """rlbm_config as ctypes lays out exactly as the C compiler lays out the header's struct."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    fields = [f[0] for f in R.rlbm_config._fields_]
    prog = ["#include <stdio.h>", "#include <stddef.h>", '#include "rlbm.h"', "int main(void) {",
            '  printf("%zu\\n", sizeof(rlbm_config));']
    prog += ['  printf("%%zu\\n", offsetof(rlbm_config, %s));' % f for f in fields]
    prog += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(prog) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    vals = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    assert vals[0] == ctypes.sizeof(R.rlbm_config)
    for f, off in zip(fields, vals[1:]):
        assert getattr(R.rlbm_config, f).offset == off, f


@pytest.mark.parametrize("vset", [3, 2])
def test_velocity_classes_fold_the_oracle_set(vset):
    """The library's folded classes (built by the library on the host) equal the oracle's
    directions grouped by their in-plane part: summed weights and the common v_z^2."""
    import numpy as np
    from oracle import rlbm_oracle as O
    C = R.rlbm_velocity_classes(vset)
    v, w = O.velocity_set(vset)
    groups = {}
    for vi, wi in zip(v, w):
        key = (round(vi[0], 12), round(vi[1], 12))
        vz2 = vi[2] ** 2 if v.shape[1] == 3 else 0.0
        g = groups.setdefault(key, [0.0, vz2])
        g[0] += wi
        assert abs(g[1] - vz2) < 1e-15
    assert C.shape == (len(groups), 4)
    seen = set()
    for vx, vy, vz2, wq in C:
        key = (round(vx, 12), round(vy, 12))
        assert key in groups and key not in seen, key
        seen.add(key)
        assert abs(groups[key][0] - wq) < 1e-15 and abs(groups[key][1] - vz2) < 1e-15, key
    assert R.lib().rlbm_velocity_classes(5, None) == -1
