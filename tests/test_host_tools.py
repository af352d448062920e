"""CPU checks of the library's host-only entry points: surrogate parameter
files, the autotuner's cache file and workload keys, and the argument checks
of the fault-injection hook.  None of these needs a GPU."""
import numpy as np
import pytest

from paper_1706_07062_gb300 import build as B
from paper_1706_07062_gb300 import kerr as K


@pytest.fixture(scope="module", autouse=True)
def built():
    B.build()
    K.lib()


def test_params_file_round_trip(tmp_path):
    n = K.kerr_surrogate_num_params()
    p = np.random.default_rng(7).standard_normal(n).astype(np.float32)
    f = tmp_path / "w.bin"
    K.kerr_params_write(str(f), p)
    raw = f.read_bytes()
    assert len(raw) == 96 + 4 * n and raw[:8] == b"KERRSURR"
    assert np.frombuffer(raw[8:12], np.uint32)[0] == 1
    assert np.frombuffer(raw[16:24], np.int64)[0] == n
    q = K.kerr_params_read(str(f))
    assert np.array_equal(p, q)
    # the payload is the FP32 vector as is, after the header
    assert np.array_equal(np.frombuffer(raw[96:], np.float32), p)


def test_params_file_is_validated(tmp_path):
    n = K.kerr_surrogate_num_params()
    p = np.arange(n, dtype=np.float32)
    f = tmp_path / "w.bin"
    K.kerr_params_write(str(f), p)
    raw = bytearray(f.read_bytes())
    bad = tmp_path / "bad.bin"
    # a flipped parameter byte fails the checksum
    b = bytearray(raw)
    b[96 + 17] ^= 0x40
    bad.write_bytes(bytes(b))
    with pytest.raises(K.KerrError, match="checksum"):
        K.kerr_params_read(str(bad))
    # another magic, another layer width, a truncated or padded file
    for mutate, what in ((lambda x: x.__setitem__(0, ord("X")), "parameter file"),
                         (lambda x: x.__setitem__(28, x[28] ^ 1), "parameter file")):
        b = bytearray(raw)
        mutate(b)
        bad.write_bytes(bytes(b))
        with pytest.raises(K.KerrError, match=what):
            K.kerr_params_read(str(bad))
    bad.write_bytes(bytes(raw[:-4]))
    with pytest.raises(K.KerrError, match="length"):
        K.kerr_params_read(str(bad))
    bad.write_bytes(bytes(raw) + b"\0")
    with pytest.raises(K.KerrError, match="length"):
        K.kerr_params_read(str(bad))
    with pytest.raises(K.KerrError):
        K.kerr_params_write(str(bad), p[:-1])           # wrong parameter count
    with pytest.raises(K.KerrError):
        K.kerr_params_read(str(tmp_path / "missing.bin"))


def test_tune_cache_store_and_lookup(tmp_path):
    path = str(tmp_path / "tune.txt")
    gpu, key = "NVIDIA GB300 (152 SMs)", K.kerr_tune_key_particles(1 << 20)
    assert K.kerr_tune_cache_lookup(path, gpu, key) is None          # no file yet
    t = K.Tuning(3, 5, 12.5, 0, 21)
    K.kerr_tune_cache_store(path, gpu, key, t)
    K.kerr_tune_cache_store(path, "other GPU (10 SMs)", key, K.Tuning(7, 1, 1.0, 0, 1))
    got = K.kerr_tune_cache_lookup(path, gpu, key)
    assert (got.variant, got.zone_variant, got.from_cache) == (3, 5, 1)
    assert abs(got.ms - 12.5) < 1e-6
    # a later line for the same pair wins
    K.kerr_tune_cache_store(path, gpu, key, K.Tuning(4, 6, 11.0, 0, 21))
    got = K.kerr_tune_cache_lookup(path, gpu, key)
    assert (got.variant, got.zone_variant) == (4, 6)
    assert K.kerr_tune_cache_lookup(path, gpu, key + "x") is None
    lines = open(path).read().splitlines()
    assert len(lines) == 3 and all(len(l.split("\t")) == 5 for l in lines)
    with pytest.raises(K.KerrError):
        K.kerr_tune_cache_store(path, "bad\tname", key, t)
    with open(path, "a") as fh:
        fh.write("garbage line\n")
    with pytest.raises(K.KerrError, match="malformed"):
        K.kerr_tune_cache_lookup(path, gpu, key)


def test_tune_keys_separate_workloads():
    o32 = K.default_opts()
    o64 = K.default_opts(prec=K.FP64)
    cam = K.camera(0.99, 0.3, 1000.0, 25.0, 1024, 1024)
    k32 = K.kerr_tune_key_cameras(cam, o32)
    assert k32 == K.kerr_tune_key_cameras(cam, o32)
    assert k32 != K.kerr_tune_key_cameras(cam, o64)                   # precision
    assert k32 != K.kerr_tune_key_cameras(K.camera(0.5, 0.3, 1000.0, 25.0, 1024, 1024), o32)
    assert k32 != K.kerr_tune_key_cameras(cam, K.default_opts(tol=1e-8))
    assert "rays=1048576" in k32
    kp = K.kerr_tune_key_particles(1 << 20, o32)
    assert kp != K.kerr_tune_key_particles(1 << 19, o32) and kp.startswith("particles:")
    with pytest.raises(K.KerrError):
        K.kerr_tune_key_particles(0, o32)


def test_fault_injection_hook_arguments():
    with pytest.raises(K.KerrError):
        K.kerr_debug_fail_alloc(-1)
    K.kerr_debug_fail_alloc(0)
