"""Host-side checks of the C ABI that need no GPU: the library builds for
sm_103a, loads, exports every entry point include/sft.h declares, and rejects
bad arguments before touching the device."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_entry_points():
    inc = os.path.join(ROOT, "include")
    src = "".join(open(os.path.join(inc, f)).read() for f in sorted(os.listdir(inc))
                  if f.endswith(".h"))
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(sft_[a-z_A-Z0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2210_06014_gb300 import build, sft
    build.build()
    return sft.load()


def test_header_declares_the_core_calls():
    names = declared_entry_points()
    for must in ["sft_init", "sft_refresh_C", "sft_update_factors", "sft_update_core", "sft_loss"]:
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    from paper_2210_06014_gb300 import sft
    for name in declared_entry_points():
        assert hasattr(lib, name), name
    assert sorted(sft.EXPORTED) == declared_entry_points()


def test_null_arguments_are_rejected_on_the_host(lib):
    from paper_2210_06014_gb300 import sft
    assert lib.sft_workspace_bytes(None, 4096) == 0
    ctx = ctypes.c_void_p()
    st = lib.sft_init(None, None, None, None, None, None, 0, ctypes.byref(ctx))
    assert st == sft.SFT_EINVAL and not ctx.value
    assert lib.sft_refresh_C(None, 0) == sft.SFT_EINVAL
    assert lib.sft_update_factors(None, 0, None, None, None, 0, 1, 0.0, 0.0) == sft.SFT_EINVAL
    assert lib.sft_update_core(None, 0, None, None, None, 0, 1, 0.0, 0.0) == sft.SFT_EINVAL
    assert lib.sft_sync(None, 0) == sft.SFT_EINVAL
    assert lib.sft_slices_expand_rows(None, 0, None, 1, None) == sft.SFT_EINVAL
    assert lib.sft_fibers_expand_coords(None, 0, None, 1, None, 1, None) == sft.SFT_EINVAL
    assert lib.sft_last_error(None) == b"null context"
    lib.sft_destroy(None)


@pytest.mark.parametrize("dims,J,R,prec,want", [
    ((10, 10), (8, 8), 8, 0, "ok"),
    ((10,), (8,), 8, 0, "EINVAL"),            # order 1
    ((10, 10), (8, 8), 12, 0, "ENOTSUP"),     # R not supported
    ((10, 10), (8, 6), 8, 0, "ENOTSUP"),      # J not supported
    ((10, 10), (4, 4), 32, 0, "ENOTSUP"),     # 4J < R
    ((10, 10), (8, 8), 8, 1, "ok"),           # bfloat16 cached products
    ((10, 10), (8, 8), 8, 7, "EINVAL"),       # unknown precision
    ((0, 10), (8, 8), 8, 0, "EINVAL"),        # empty mode
])
def test_config_validation(lib, dims, J, R, prec, want):
    """sft_init rejects unsupported shapes before it needs a device; a valid
    shape gets as far as asking for the device (which this host lacks).  The
    pointers are placeholders that are never dereferenced: every case here
    returns before any device work."""
    import torch
    from paper_2210_06014_gb300 import sft
    if want == "ok" and torch.cuda.is_available():
        pytest.skip("a valid config would reach the device; covered by the GPU tests")
    cfg = sft.make_config(dims, J, R, True, prec, stream=0)
    ctx = ctypes.c_void_p()
    fake = (ctypes.c_void_p * len(dims))(*([256] * len(dims)))
    st = lib.sft_init(ctypes.byref(cfg), fake, fake, fake, None, ctypes.c_void_p(256), 1 << 20,
                      ctypes.byref(ctx))
    if want == "ok":
        assert st == sft.SFT_ECUDA
    else:
        assert st == getattr(sft, "SFT_" + want)
    assert not ctx.value
