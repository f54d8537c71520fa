"""The C-ABI library builds, loads and exports every entry point that
include/cvo.h declares (no compute calls: this runs without a GPU)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "cvo.h")


def _declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(cvo_[a-z_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib_path():
    from paper_1904_02266_gb300 import build
    return build.build()


def test_header_declares_the_documented_entry_points():
    names = _declared()
    for n in ("cvo_create", "cvo_destroy", "cvo_set_cloud", "cvo_release_cloud", "cvo_eval",
              "cvo_align", "cvo_strerror"):
        assert n in names


def test_library_exports_every_declared_symbol(lib_path):
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\bT (cvo_[a-z_]+)\b", out))
    missing = [n for n in _declared() if n not in exported]
    assert not missing, missing
    lib = ctypes.CDLL(lib_path)
    for n in _declared():
        assert getattr(lib, n) is not None


def test_binding_names_match_the_header(lib_path):
    import paper_1904_02266_gb300 as cvo
    assert sorted(cvo.EXPORTS) == _declared()
    for n in _declared():
        assert callable(getattr(cvo, n))


def test_host_only_calls(lib_path):
    import paper_1904_02266_gb300 as cvo
    p = cvo.cvo_params_default()
    assert p.ell0 == 0.15 and p.kcut == 1e-3 and p.max_iters == 200 and p.feat_dim == 5
    assert cvo.strerror(cvo.CVO_ERR_OUT_OF_BUDGET) == "CVO_ERR_OUT_OF_BUDGET"
    lib = cvo.load_library()
    assert lib.cvo_stream(None) is None
    bad = cvo.cvo_params_default()
    bad.kcut = 0.0
    out = ctypes.c_void_p()
    assert lib.cvo_create(ctypes.byref(bad), 0, 0, ctypes.byref(out)) == cvo.CVO_ERR_INVALID_ARG


def test_struct_layouts_match_the_header(lib_path):
    """ctypes mirrors of the ABI structs have the C sizes and field offsets
    (checked by compiling a tiny C program against the header)."""
    import paper_1904_02266_gb300 as cvo
    structs = [cvo.cvo_params, cvo.cvo_eval_result, cvo.cvo_stats, cvo.cvo_iter_profile,
               cvo.cvo_batch_info, cvo.cvo_request, cvo.cvo_result, cvo.cvo_serve_params,
               cvo.cvo_serve_stats, cvo.cvo_frontend_params, cvo.cvo_tune_space,
               cvo.cvo_tune_report]
    lines = []
    for st in structs:
        name = st.__name__
        lines.append(f'printf("%zu\\n", sizeof({name}));')
        for f, _ in st._fields_:
            lines.append(f'printf("%zu\\n", offsetof({name}, {f}));')
    src = ('#include <stdio.h>\n#include <stddef.h>\n#include "cvo.h"\nint main(void){'
           + "".join(lines) + 'return 0;}\n')
    tmp = os.path.join(ROOT, "paper_1904_02266_gb300", "_build")
    os.makedirs(tmp, exist_ok=True)
    c = os.path.join(tmp, "abi_sizes.c")
    exe = os.path.join(tmp, "abi_sizes")
    with open(c, "w") as fh:
        fh.write(src)
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), "-o", exe, c], check=True)
    got = [int(v) for v in subprocess.run([exe], capture_output=True, text=True,
                                          check=True).stdout.split()]
    want = []
    for st in structs:
        want.append(ctypes.sizeof(st))
        want.extend(getattr(st, f).offset for f, _ in st._fields_)
    assert got == want
