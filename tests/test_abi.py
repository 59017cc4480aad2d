"""CPU-side checks of the C-ABI boundary: the header is plain C, the library
loads without a GPU, and it exports every entry point the header declares."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "wt.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*int\s+(wt_\w+)\s*\(", src, flags=re.M)))


def test_header_is_plain_c(tmp_path):
    c = tmp_path / "use.c"
    c.write_text('#include "wt.h"\nint main(void){ wt_tree *t = 0; wt_info_t i; (void)i;'
                 ' return wt_free(t); }\n')
    subprocess.check_call(["gcc", "-std=c99", "-Wall", "-Werror", "-fsyntax-only",
                           "-I", os.path.join(ROOT, "include"), str(c)])


@pytest.fixture(scope="module")
def lib():
    from paper_1407_8142_gb300 import build, wt
    build.build()
    return wt.load()


def test_library_exports_every_declared_symbol(lib):
    names = declared_functions()
    assert len(names) >= 14
    for name in names:
        assert hasattr(lib, name), f"{name} declared in wt.h but not exported"


def test_binding_covers_the_header():
    from paper_1407_8142_gb300 import wt
    assert sorted(wt.SIGNATURES) == declared_functions()


def test_host_side_argument_checks(lib):
    """Errors detected on the host return before any CUDA call that needs a GPU."""
    import ctypes
    from paper_1407_8142_gb300 import wt
    out = ctypes.c_void_p()
    # bad symbol size, sigma = 0, sigma beyond the storage type, too many levels, n >= 2^32
    for n, sigma, b in ((10, 4, 3), (10, 0, 1), (10, 257, 1), (10, 1 << 27, 4), (1 << 32, 4, 1)):
        assert lib.wt_create(n, sigma, b, None, ctypes.byref(out)) == wt.WT_ERR_ARG
    cfg = wt.Config(100, 0, 0, 0)  # tile_threads must be 128/256/512
    assert lib.wt_create(10, 4, 1, ctypes.byref(cfg), ctypes.byref(out)) == wt.WT_ERR_ARG
    cfg = wt.Config(0, 0, 0, 0, 5)  # at most 4 levels per pass
    assert lib.wt_create(10, 4, 1, ctypes.byref(cfg), ctypes.byref(out)) == wt.WT_ERR_ARG
    assert lib.wt_matrix_create(10, 4, 1, ctypes.byref(cfg), ctypes.byref(out)) == wt.WT_ERR_ARG
    assert lib.wt_build_host_async(None, None, None, None, None) == wt.WT_ERR_ARG
    assert lib.wt_rebuild(None, None, None) == wt.WT_ERR_ARG
    assert lib.wt_sync(None) == wt.WT_ERR_ARG
    assert lib.wt_free(None) == wt.WT_OK


def test_noalloc_size_checks_cannot_wrap(lib):
    """The allocation-free build rejects oversized problems on the host, before
    any CUDA call, also where n * symbol_bytes would wrap around 2^64."""
    from paper_1407_8142_gb300 import wt
    for n, b in (((1 << 21) + 1, 1), ((1 << 20) + 1, 2), ((1 << 19) + 1, 4),
                 (1 << 32, 1), (1 << 63, 2), ((1 << 62) + 1, 4), ((1 << 64) - 1, 1)):
        assert lib.wt_build_noalloc(None, n, 4, b, None, None, None, None, None, None) == wt.WT_ERR_ARG
    # sigma beyond 2^16 (17 levels) is beyond the fixed scratch
    assert lib.wt_build_noalloc(None, 10, (1 << 16) + 1, 4, None, None, None, None, None,
                                None) == wt.WT_ERR_ARG


def test_resize_checks_on_the_host(lib):
    """wt_resize rejects a NULL tree before touching the device."""
    from paper_1407_8142_gb300 import wt
    assert lib.wt_resize(None, 10) == wt.WT_ERR_ARG
