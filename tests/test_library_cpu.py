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
