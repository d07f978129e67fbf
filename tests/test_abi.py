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


def test_binding_structs_match_the_header(tmp_path):
    """Every ctypes structure of the binding has the size and the field
    offsets of the C structure of the same name in include/hf.h (compiled
    with the host C compiler), so that no field is misplaced across the ABI."""
    import shutil
    from paper_2211_14346_gb300 import _lib
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = [v for k, v in vars(_lib).items()
               if k.startswith("hf_") and isinstance(v, type) and issubclass(v, C.Structure)]
    assert len(structs) >= 10
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "hf.h"', "int main(void) {"]
    for s in structs:
        n = s.__name__
        lines.append('printf("%s %%zu\\n", sizeof(%s));' % (n, n))
        for f in s._fields_:
            lines.append('printf("%s.%s %%zu\\n", offsetof(%s, %s));' % (n, f[0], n, f[0]))
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = dict(l.split() for l in subprocess.run([str(exe)], capture_output=True, text=True,
                                                 check=True).stdout.splitlines())
    for s in structs:
        n = s.__name__
        assert int(got[n]) == C.sizeof(s), (n, got[n], C.sizeof(s))
        for f in s._fields_:
            assert int(got["%s.%s" % (n, f[0])]) == getattr(s, f[0]).offset, (n, f[0])
