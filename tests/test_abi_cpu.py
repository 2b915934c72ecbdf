"""The C-ABI library loads and exports every symbol include/*.h declares, and its
argument checks answer without touching a GPU.  CPU only."""
import ctypes
import glob
import os
import re

import pytest

import paper_2305_05810_gb300 as stf
from paper_2305_05810_gb300 import build as stf_build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    stf_build.build()
    return stf.load()


def _declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
        names |= set(re.findall(r"\b(stf_\w+)\s*\(", text))
    return sorted(names)


def test_every_declared_symbol_is_exported(lib):
    names = _declared_functions()
    assert "stf_lookup_batch" in names and "stf_create_texture" in names
    for n in names:
        assert hasattr(lib, n), n


def test_version_and_struct_sizes(lib):
    assert stf.stf_version() == 10000
    assert ctypes.sizeof(stf.TextureDesc) == 72
    assert ctypes.sizeof(stf.LookupParams) == 40


def test_argument_errors_without_gpu(lib):
    h = ctypes.c_void_p()
    assert lib.stf_create_texture(None, None, ctypes.byref(h)) == 1
    assert "NULL" in stf.stf_last_error()
    desc = stf.TextureDesc(kind=9, format=0, channels=1, mip_levels=1)
    buf = (ctypes.c_float * 4)()
    desc.data = ctypes.addressof(buf)
    assert lib.stf_create_texture(ctypes.byref(desc), None, ctypes.byref(h)) == 1
    assert "kind" in stf.stf_last_error()
    desc.kind, desc.channels = 0, 3
    desc.dims[:] = [4, 4, 1]
    assert lib.stf_create_texture(ctypes.byref(desc), None, ctypes.byref(h)) == 1
    assert "channels" in stf.stf_last_error()
    desc.channels, desc.mip_levels = 4, 9
    assert lib.stf_create_texture(ctypes.byref(desc), None, ctypes.byref(h)) == 1
    assert "mip_levels" in stf.stf_last_error()
    p = stf.make_params()
    bogus = ctypes.c_void_p(0x1234)
    assert lib.stf_lookup_batch(bogus, ctypes.byref(p), None, None, 0, None, None, None) == 2
    assert lib.stf_lookup_batch_deterministic(None, ctypes.byref(p), None, None, 0, None, None) == 2
    assert lib.stf_destroy(bogus) == 2
    b = ctypes.c_int64()
    assert lib.stf_texture_bytes(bogus, ctypes.byref(b)) == 2
    with pytest.raises(stf.StfError) as e:
        stf.stf_destroy(0x1234)
    assert e.value.status == 2
    assert lib.stf_anisotropic_lod(bogus, None, 0, ctypes.c_float(8.0), None, None) == 2
    assert lib.stf_lookup_batch_ewa(bogus, ctypes.byref(p), None, None, 0, ctypes.c_float(8.0),
                                    None, None, None) == 2
    v = ctypes.c_int32(7)
    assert lib.stf_device_accessible(None, None) == 1            # NULL out
    assert lib.stf_device_accessible(None, ctypes.byref(v)) == 0 and v.value == 0   # NULL pointer


def test_ewa_weight_table_is_the_oracle_table(lib):
    """The library's EWA weight table (a host-side table, no GPU involved) holds the
    oracle's float64 values exp(-2 r) - exp(-2) at r = i / 127, rounded to float32."""
    import numpy as np
    from oracle import ewa
    assert np.array_equal(np.array(stf.stf_ewa_weight_table(), dtype=np.float32),
                          ewa.weight_lut().astype(np.float32))       # correctly rounded


def test_binding_raises_when_library_missing(monkeypatch, tmp_path):
    monkeypatch.setattr(stf, "_lib", None)
    monkeypatch.setattr(stf_build, "LIB", str(tmp_path / "missing.so"))
    with pytest.raises(OSError):
        stf.load(build_if_missing=False)
