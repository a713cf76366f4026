"""CPU-side checks of the C ABI library (no GPU): it builds for sm_103a,
loads, exports every function include/xdrop.h declares, and refuses to run
without a GPU instead of falling back to the CPU."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(xdrop_\w+)\s*\(", src))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_2309_07270_gb300 import build, xdrop
    build.build()
    return xdrop.load()


def test_header_declares_the_abi():
    names = declared_functions()
    for must in ("xdrop_init", "xdrop_submit", "xdrop_sync", "xdrop_free"):
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_binding_names_match_header():
    from paper_2309_07270_gb300 import xdrop
    assert set(xdrop.EXPORTS) == set(declared_functions())


def test_no_cpu_fallback_without_gpu(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is visible")
    from paper_2309_07270_gb300 import xdrop
    with pytest.raises(xdrop.XdropError) as ei:
        xdrop.xdrop_init(0)
    assert ei.value.code in (xdrop.XDROP_ECUDA, xdrop.XDROP_EINVAL)


def test_record_layouts():
    from paper_2309_07270_gb300 import workloads, xdrop
    assert xdrop.PAIR_DTYPE.itemsize == 20 and xdrop.RESULT_DTYPE.itemsize == 28
    assert workloads.PAIR_DTYPE == xdrop.PAIR_DTYPE


def test_binding_constants_match_header():
    """Every #define XDROP_* of the header has the same value in the binding."""
    from paper_2309_07270_gb300 import xdrop
    src = open(os.path.join(ROOT, "include", "xdrop.h")).read()
    defs = re.findall(r"#define\s+(XDROP_\w+)\s+\(?(-?(?:0x[0-9a-fA-F]+|\d+))\)?u?", src)
    assert len(defs) >= 13
    for name, val in defs:
        assert getattr(xdrop, name) == int(val, 0), name


# C struct of include/xdrop.h -> its ctypes mirror in the binding
MIRRORS = {"xdrop_scoring": "Scoring", "xdrop_stats": "Stats", "xdrop_serve_stats": "ServeStats",
           "xdrop_kmer_params": "KmerParams", "xdrop_seed_stats": "SeedStats",
           "xdrop_accept_params": "AcceptParams"}


def test_struct_layouts_match_the_header(tmp_path):
    """Size and every field offset of each parameter/statistics struct, as
    the C compiler lays it out from the header, equal the binding's ctypes
    mirror."""
    import ctypes
    import shutil
    import subprocess

    from paper_2309_07270_gb300 import xdrop
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no gcc")
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "xdrop.h"', "int main(void) {"]
    for cname, pyname in MIRRORS.items():
        cls = getattr(xdrop, pyname)
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for field, _ in cls._fields_:
            lines.append(f'printf("{cname} {field} %zu\\n", offsetof({cname}, {field}));')
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run([gcc, "-I", os.path.join(ROOT, "include"), "-o", str(exe), str(src)], check=True)
    got = {}
    for ln in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n"):
        if ln:
            c, f, v = ln.split()
            got[(c, f)] = int(v)
    for cname, pyname in MIRRORS.items():
        cls = getattr(xdrop, pyname)
        assert got[(cname, "size")] == ctypes.sizeof(cls), cname
        for field, _ in cls._fields_:
            assert got[(cname, field)] == getattr(cls, field).offset, (cname, field)


def test_new_entry_points_refuse_a_null_context(lib):
    """Argument checks come before any CUDA call: no GPU needed to see them."""
    import ctypes

    from paper_2309_07270_gb300 import xdrop
    n = ctypes.c_size_t()
    prm = xdrop.KmerParams(31, 1, 20, 30, 0)
    assert lib.xdrop_find_candidates(None, ctypes.byref(prm), None, None, 0,
                                     ctypes.byref(n)) == xdrop.XDROP_EINVAL
    assert lib.xdrop_get_seed_stats(None, ctypes.byref(xdrop.SeedStats())) == xdrop.XDROP_EINVAL
    acc = xdrop.AcceptParams(1, -1, 1500, 1000)
    assert lib.xdrop_accept_device(None, None, None, 0, None, 0, ctypes.byref(acc),
                                   None) == xdrop.XDROP_EINVAL
    assert lib.xdrop_best_seeds_device(None, None, None, 0, 1, None) == xdrop.XDROP_EINVAL
