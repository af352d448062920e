"""CPU checks of the C ABI: libkerr builds, loads without a GPU, exports every
function include/kerr.h declares, and its structs have the layout the
Python binding assumes."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

from paper_1706_07062_gb300 import build as B
from paper_1706_07062_gb300 import kerr as K
from paper_1706_07062_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "kerr.h")


@pytest.fixture(scope="module")
def libpath():
    return B.build()


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\**\s*(kerr_[a-z_0-9]+)\s*\(",
                                 src, flags=re.M)))


def test_header_declares_the_boundary():
    fns = declared_functions()
    for name in ("kerr_init", "kerr_destroy", "kerr_trace_rays", "kerr_trace_camera",
                 "kerr_trace_particles", "kerr_last_error", "kerr_get_stats", "kerr_autotune"):
        assert name in fns


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\bT (kerr_[a-z_0-9]+)", out))
    missing = [f for f in declared_functions() if f not in exported]
    assert not missing, missing
    L = ctypes.CDLL(libpath)            # loads with no GPU present
    for f in declared_functions():
        assert hasattr(L, f)


def test_struct_layout_matches_binding(tmp_path):
    prog = tmp_path / "sz.c"
    prog.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "kerr.h"\n'
                    'int main(void){printf("%zu %zu %zu %zu %zu %zu %zu %zu\\n", sizeof(kerr_opts),'
                    ' sizeof(kerr_camera), sizeof(kerr_stats), offsetof(kerr_opts, budget_ns),'
                    ' offsetof(kerr_stats, kernel_ms), offsetof(kerr_camera, ny),'
                    ' sizeof(kerr_tuning), offsetof(kerr_stats, clip_rhs)); return 0;}\n')
    exe = tmp_path / "sz"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.dirname(HEADER), str(prog), "-o", str(exe)],
                   check=True)
    vals = list(map(int, subprocess.run([str(exe)], capture_output=True, text=True,
                                        check=True).stdout.split()))
    assert vals == [ctypes.sizeof(K.Opts), ctypes.sizeof(K.Camera), ctypes.sizeof(K.Stats),
                    K.Opts.budget_ns.offset, K.Stats.kernel_ms.offset, K.Camera.ny.offset,
                    ctypes.sizeof(K.Tuning), K.Stats.clip_rhs.offset]


def test_defaults_and_variants_without_gpu(libpath):
    o = K.default_opts()
    assert o.prec == K.FP32_KAHAN and o.tol == 1e-6 and o.h0 == 1.0
    assert o.max_steps == 1_000_000 and o.r_escape == 0.0 and np.isinf(o.t_end)
    assert o.fp64_zone == 1.5 and o.clip_maxit == 40 and o.variant == -1
    assert o.zone_quantum == 32 and o.zone_variant == -1
    n = K.kerr_num_variants()
    assert n >= 1
    rays = []
    for v in range(n):
        b, m = K.kerr_variant_info(v)
        assert b % 32 == 0 and m >= 1
        b2, m2, r, rm = K.kerr_variant_shape(v)
        assert (b2, m2) == (b, m) and r in (1, 2) and rm in (0, 1)
        assert r == 1 or rm == 1          # paired steps always call their right-hand side
        rays.append(r)
    assert 1 in rays and 2 in rays
    with pytest.raises(K.KerrError):
        K.kerr_variant_info(n)
    with pytest.raises(K.KerrError):
        K.kerr_variant_shape(-1)


def test_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    monkeypatch.setattr(K, "_lib", None)
    monkeypatch.setattr(K, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(K.KerrError):
        K.lib()


def test_workloads_are_seeded_and_shaped():
    a = W.camera_subset(W.CAMERA_1024)
    b = W.camera_subset(W.CAMERA_1024)
    assert np.array_equal(a, b) and a.size == 4096 and np.unique(a).size == 4096
    cams = W.camera_batch()
    assert len(cams) == 64
    assert all(c.nx in W.BATCH_SIDES and 0 <= c.a <= 0.998 for c in cams)
    ps = W.particles(n=4096)
    assert ps.x0.shape == (4, 4096) and ps.v0.shape == (3, 4096)
    assert np.all((ps.semi_major >= 10) & (ps.semi_major <= 1000))
    # Newtonian energy of the drawn state matches the drawn semi-major axis
    r = np.linalg.norm(ps.x0[1:], axis=0)
    v2 = np.sum(ps.v0 ** 2, axis=0)
    np.testing.assert_allclose(0.5 * v2 - 1 / r, -0.5 / ps.semi_major, rtol=1e-9)
    sub = W.particle_subset(ps, k=256)
    assert sub.size == 256
