"""The C ABI library loads and exports every function include/*.h declares, and the
binding's structures match the header's layout (no compute call: CPU only)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
LIB = os.path.join(ROOT, "paper_2212_10680_gb300", "libfmlbm.so")


def declared_functions():
    names = set()
    for hdr in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(hdr).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(fmlbm_[a-z0-9_]+)\s*\(", text):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(LIB):
        from paper_2212_10680_gb300 import build
        build.build()
    return ctypes.CDLL(LIB)


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 18
    missing = [n for n in sorted(names) if not hasattr(lib, n)]
    assert not missing, missing


def test_status_strings_and_version(lib):
    lib.fmlbm_status_str.restype = ctypes.c_char_p
    lib.fmlbm_version.restype = ctypes.c_char_p
    assert lib.fmlbm_status_str(0) == b"FMLBM_OK"
    assert lib.fmlbm_status_str(4) == b"FMLBM_E_NONPHYSICAL"
    assert b"sm_103a" in lib.fmlbm_version()


def test_struct_layout_matches_header():
    from paper_2212_10680_gb300 import fmlbm
    # 2 int32 + 2 double + 5 x 4 double + 16 double
    assert ctypes.sizeof(fmlbm.fmlbm_mixture) == 8 + 16 + 5 * 32 + 128
    assert ctypes.sizeof(fmlbm.fmlbm_lattice) == 8 + 8 + 16
    # 2 uint64 + 2 int32 + int64 + 4 double + 2 x 4 double
    assert ctypes.sizeof(fmlbm.fmlbm_result) == 16 + 8 + 8 + 32 + 64


def test_lattice_bytes_needs_no_gpu(lib):
    from paper_2212_10680_gb300 import fmlbm
    L = fmlbm.make_lattice(1024, 1024, 1.0, precision="fp32")
    n = fmlbm.fmlbm_lattice_bytes(2, L)
    # two FP32 distribution buffers of 2 x 9 planes dominate
    assert n >= 2 * 2 * 9 * 1024 * 1024 * 4
    L16 = fmlbm.make_lattice(1024, 1024, 1.0, precision="bf16dev")
    assert fmlbm.fmlbm_lattice_bytes(2, L16) < n


def test_buffer_sizes_need_no_gpu(lib):
    # the caller-provided buffers of fmlbm_create_with_buffers, per buffer: N x 9 planes of the
    # storage type (16-bit forms: N x 8 planes of 2 bytes plus N float planes for a = 0), and
    # the stored force, 2 planes of the storage arithmetic type
    from paper_2212_10680_gb300 import fmlbm
    nxy = 64 * 32
    cases = {"fp64": (2 * 9 * nxy * 8, 0, 2 * nxy * 8), "fp32": (2 * 9 * nxy * 4, 0, 2 * nxy * 4),
             "bf16dev": (2 * 8 * nxy * 2, 2 * nxy * 4, 2 * nxy * 4), "fp16dev": (2 * 8 * nxy * 2, 2 * nxy * 4, 2 * nxy * 4)}
    for prec, want in cases.items():
        assert fmlbm.fmlbm_buffer_sizes(2, fmlbm.make_lattice(64, 32, 1.0, precision=prec)) == want, prec
    for n, L in ((5, fmlbm.make_lattice(64, 32, 1.0)), (2, fmlbm.make_lattice(0, 32, 1.0))):
        with pytest.raises(fmlbm.FmlbmError) as ei:
            fmlbm.fmlbm_buffer_sizes(n, L)
        assert ei.value.status == 1
