"""The C-ABI library builds, loads and exports every entry point include/ace.h declares (no GPU)."""

import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "ace.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*([a-z_][a-z0-9_]*)\s*\(", text, flags=re.M)
    return sorted(set(n for n in names if n not in ("if", "return")))


@pytest.fixture(scope="module")
def lib():
    from paper_2101_03155_gb300 import build

    path = build.build()
    return ctypes.CDLL(path)


def test_header_parses():
    names = declared_functions()
    for must in ("ace_build", "ace_apply", "exchange_energy", "ace_build_batched", "ace_get", "ace_destroy",
                 "ace_last_error", "ace_pair_count"):
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, f"declared in include/ace.h but not exported: {missing}"


def test_binding_covers_the_abi():
    from paper_2101_03155_gb300 import ace

    assert sorted(ace.EXPORTED) == declared_functions()
    for n in ace.EXPORTED:
        assert callable(getattr(ace, n))


def test_host_side_checks_without_gpu(lib):
    """Argument checks that run before any CUDA call return ACE_ERR_ARG / UNSUPPORTED_GRID."""
    from paper_2101_03155_gb300 import ace

    ace.load()
    assert ace.ace_grid_supported(96) and ace.ace_grid_supported(160) and ace.ace_grid_supported(15)
    assert not ace.ace_grid_supported(97) and not ace.ace_grid_supported(14) and not ace.ace_grid_supported(512)
    d = ace.make_desc((96, 96, 97), np.eye(3) * 10, 4)
    with pytest.raises(ace.AceError) as e:
        ace.ace_build(d, np.zeros((4, 96, 96, 97), np.float32))
    assert e.value.status == ace.ACE_ERR_UNSUPPORTED_GRID
    d = ace.make_desc((16, 16, 16), np.zeros((3, 3)), 4)
    with pytest.raises(ace.AceError) as e:
        ace.ace_build(d, np.zeros((4, 16, 16, 16), np.float32))
    assert e.value.status == ace.ACE_ERR_ARG
    assert "singular" in ace.ace_last_error()
    h = ctypes.c_void_p()
    assert lib.ace_build(None, None, 0, None, ctypes.byref(h)) == ace.ACE_ERR_ARG
    lib.ace_destroy(None)  # no-op
    # graph entry points: counts and NULL handles are checked before any CUDA call
    lib.ace_graph_create.argtypes = [ctypes.c_int] + [ctypes.c_void_p] * 7
    assert lib.ace_graph_create(0, None, None, 0, None, None, None, ctypes.byref(h)) == ace.ACE_ERR_ARG
    assert lib.ace_graph_create(1, None, None, 0, None, None, None, None) == ace.ACE_ERR_ARG
    assert lib.ace_graph_launch(None, None) == ace.ACE_ERR_ARG
    assert lib.ace_graph_sync(None) == ace.ACE_ERR_ARG
    assert lib.ace_graph_size(None) == 0
    lib.ace_graph_destroy(None)  # no-op
    # SCDM: orbital count, point count (at least one per orbital) and precision are checked first
    a = np.zeros((4, 3), np.float32)
    for n, npts, prec in ((0, 3, ace.ACE_MIXED), (1025, 4096, ace.ACE_MIXED), (4, 3, ace.ACE_MIXED), (4, 8, 7)):
        st = ace.load().ace_scdm(n, npts, prec, a.ctypes.data, ace.ACE_F32, a.ctypes.data, None, None, None, None)
        assert st == ace.ACE_ERR_ARG, (n, npts, prec)
    assert "norb" in ace.ace_last_error() or "precision" in ace.ace_last_error()


def test_product_path_does_not_import_oracle():
    import subprocess
    import sys

    code = ("import sys; import paper_2101_03155_gb300 as p; p.ace.load(); "
            "bad=[m for m in sys.modules if m == 'oracle' or m.startswith('oracle.')]; "
            "assert not bad, bad")
    subprocess.run([sys.executable, "-c", code], cwd=ROOT, check=True)


def test_descriptor_layout_matches_header(tmp_path):
    """The binding's ace_desc has the C layout: a C program compiled against include/ace.h prints
    sizeof and every field offset, and the ctypes structure must agree."""
    import shutil
    import subprocess

    from paper_2101_03155_gb300 import ace

    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    fields = [f[0] for f in ace.AceDesc._fields_]
    src = tmp_path / "layout.c"
    src.write_text(
        '#include <stddef.h>\n#include <stdio.h>\n#include "ace.h"\nint main(void) {\n'
        '  printf("%zu\\n", sizeof(ace_desc));\n'
        + "".join(f'  printf("%zu\\n", offsetof(ace_desc, {f}));\n' for f in fields)
        + "  return 0;\n}\n"
    )
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.dirname(HEADER), str(src), "-o", str(exe)], check=True)
    out = [int(x) for x in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()]
    assert out[0] == ctypes.sizeof(ace.AceDesc)
    assert out[1:] == [getattr(ace.AceDesc, f).offset for f in fields]


def test_scdm_binding_checks_shapes_before_the_library():
    """The Python binding of ace_scdm refuses mismatched input and output arrays itself."""
    from paper_2101_03155_gb300 import ace

    a = np.zeros((4, 64), np.float32)
    for out in (np.zeros((4, 64), np.float64), np.zeros((4, 65), np.float32)):
        with pytest.raises(ValueError):
            ace.ace_scdm(a, out)
