"""CPU-side checks of the C ABI: the library builds, loads, exports every
symbol include/mpo.h declares, validates arguments, and refuses to run without
a GPU (there is no CPU fallback)."""
import ctypes
import os
import re

import pytest

from paper_2003_13163_gb300 import build as B
from paper_2003_13163_gb300 import mpo

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "mpo.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(mpo_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return mpo.load_library()


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert "mpo_init" in names and "mpo_apply_layer" in names and "mpo_entropy" in names and "mpo_free" in names
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) <= set(mpo.EXPORTS)


def test_version(lib):
    assert b"sm_103a" in lib.mpo_version()


def test_argument_validation_before_device(lib):
    h = ctypes.c_void_p()
    assert lib.mpo_init(ctypes.byref(h), 7, 16, 0, None, None) == -1      # odd n
    assert lib.mpo_init(ctypes.byref(h), 8, 0, 0, None, None) == -1      # chi_max
    assert lib.mpo_init(ctypes.byref(h), 8, 16, 5, None, None) == -1     # precision
    assert lib.mpo_init(None, 8, 16, 0, None, None) == -1
    assert lib.mpo_apply_layer(None, 0, None, None, 0) == -1
    n_i = (ctypes.c_int * 2)(8, 7)
    assert lib.mpo_init_batch(None, 2, n_i, 16, 0, None, None, 0) == -1
    assert lib.mpo_init_batch(ctypes.byref(h), 0, n_i, 16, 0, None, None, 0) == -1   # k
    assert lib.mpo_init_batch(ctypes.byref(h), 2, n_i, 16, 0, None, None, 0) == -1   # odd n_1
    assert lib.mpo_init_batch(ctypes.byref(h), 2, None, 16, 0, None, None, 0) == -1
    assert lib.mpo_apply_layer_batch(None, 1, None, None, None, None, None, None) == -1
    assert lib.mpo_batch_instance(None, 0, ctypes.byref(h)) == -1
    lib.mpo_free(None)                                                    # no-op


def test_no_cpu_fallback(lib):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    with pytest.raises(mpo.MPOError) as e:
        mpo.MPO(8, 16)
    assert e.value.code == -2
    with pytest.raises(mpo.MPOError) as e:
        mpo.MPOBatch([8, 6], 16)
    assert e.value.code == -2


def test_missing_library_fails_loudly(tmp_path):
    saved = mpo._lib
    try:
        mpo._lib = None
        with pytest.raises(RuntimeError):
            mpo.load_library(str(tmp_path / "absent.so"))
    finally:
        mpo._lib = saved
