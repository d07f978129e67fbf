"""The C-ABI library builds, loads and exports every entry point that
include/hf.h declares; its error paths work without a GPU.  No GPU needed."""
import ctypes as C
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "hf.h")


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(hf_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2211_14346_gb300 import build, _lib
    build.build()
    return _lib.load()


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("hf_open", "hf_define_cuts", "hf_submit_chunk", "hf_poll", "hf_fetch_results",
              "hf_close", "hf_last_error", "hf_run_device"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    from paper_2211_14346_gb300 import _lib
    so = _lib.LIB_PATH
    out = subprocess.run(["nm", "-D", "--defined-only", so], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\sT\s(hf_\w+)", out))
    declared = set(_declared())
    assert declared <= exported, declared - exported
    assert set(_lib.declared_symbols()) == declared
    for n in declared:
        assert hasattr(lib, n)


def test_error_paths_without_gpu(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("exercises the no-device path")
    from paper_2211_14346_gb300 import _lib
    ctx = C.c_void_p()
    st = lib.hf_open(None, C.byref(ctx))
    assert st in (_lib.HF_ECUDA, _lib.HF_EINVAL)
    assert ctx.value is None
    assert lib.hf_last_error(None)  # a message, not NULL
    assert lib.hf_close(None) == _lib.HF_OK
    assert lib.hf_open(None, None) == _lib.HF_EINVAL
    # calls on a NULL context are rejected, not crashes
    t = C.c_uint64()
    assert lib.hf_submit_chunk(None, 1, None, 0, 0, 0, 1, C.byref(t)) == _lib.HF_EINVAL
    assert lib.hf_poll(None, 1, None) == _lib.HF_EINVAL
    assert lib.hf_fetch_results(None, 1, None, 0) == _lib.HF_EINVAL
    assert lib.hf_run_device(None, 1, None, 0, 0, 0, 1, None, None) == _lib.HF_EINVAL


def test_product_path_has_no_oracle_dependency():
    """The CUDA library and its binding never reference the oracle."""
    pkg = os.path.join(ROOT, "paper_2211_14346_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".cpp", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt, f
                assert "hf_oracle" not in txt and "liboracle" not in txt, f
