"""The C-ABI library builds for sm_103a, loads without a GPU, and exports every function
``include/asx.h`` declares; argument checks that happen before any CUDA call work on a
CPU-only machine."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2406_14933_gb300 import build
    path = build.build()
    return C.CDLL(path)


def _declared(header):
    text = open(os.path.join(ROOT, "include", header)).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(asx_[a-z0-9_]+)\s*\(", text)))


def test_exports_every_declared_symbol(lib):
    names = _declared("asx.h")
    assert "asx_step" in names and "asx_run_until" in names and "asx_mass_ledger" in names
    for name in names:
        assert hasattr(lib, name), name


def test_binding_covers_header():
    from paper_2406_14933_gb300 import asx
    assert sorted(asx.exported_names()) == _declared("asx.h")


def test_host_side_argument_checks(lib):
    from paper_2406_14933_gb300 import asx
    asx.load()
    d = asx.asx_raster_desc()
    d.rows, d.cols, d.edge_m = 1, 10, 1.0            # rows < 2
    with pytest.raises(asx.AsxError) as e:
        asx.asx_create_raster(d)
    assert e.value.status == asx.ASX_EINVAL
    d.rows, d.cols, d.edge_m = 10, 10, -1.0          # edge <= 0
    with pytest.raises(asx.AsxError):
        asx.asx_create_raster(d)
    d.edge_m = 1.0
    d.bc[2] = 7                                      # unknown boundary type
    with pytest.raises(asx.AsxError):
        asx.asx_create_raster(d)
    d.bc[2] = 0
    d.n_classes = 99
    with pytest.raises(asx.AsxError):
        asx.asx_create_raster(d)
    assert asx.asx_last_error(None) == "null raster handle"
