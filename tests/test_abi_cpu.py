"""CPU-only checks of the C ABI library: it loads, exports every symbol that
include/act.h declares, and its host-side grid logic matches Table 2.
No CUDA call that needs a GPU is made here."""
import ctypes
import os
import re

import pytest

from paper_2607_16629_gb300 import act

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "act.h")


def _declared_symbols():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^ACT_API\s+[\w\s\*]*?\b(act_\w+)\s*\(", text, flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(act.LIB_PATH):
        import __graft_entry__
        __graft_entry__.build()
    return act.load_library()


def test_header_declares_the_binding_exports():
    assert _declared_symbols() == sorted(act.EXPORTS)


def test_library_exports_every_declared_symbol(lib):
    raw = ctypes.CDLL(act.LIB_PATH)
    for name in _declared_symbols():
        assert hasattr(raw, name), name


def test_status_strings(lib):
    assert act.status_name(act.ACT_OK) == "ACT_OK"
    assert act.status_name(act.ACT_ERR_NONFINITE) == "ACT_ERR_NONFINITE"
    assert act.status_name(99) == "ACT_ERR_UNKNOWN"


@pytest.mark.parametrize("sig,ranges,total", [
    ("EEG", [(0, 256, 16), (0.5, 15, 0.5), (-4, 1, 0.5), (-10, 10, 0.5)], 185600),
    ("EMG", [(0, 200, 32), (20, 450, 10), (-4, 0, 0.3), (-10, 10, 0.75)], 113778),
    ("Radar", [(0, 256, 16), (10, 8533, 100), (-4, 0, 0.3), (-10, 10, 0.75)], 520128),
])
def test_grid_from_ranges_reproduces_table2(lib, sig, ranges, total):
    d = act.act_grid_from_ranges(256, 256.0, *ranges)
    got = d.tc.count * d.fc.count * d.logdt.count * d.c.count
    assert got == total
    assert d.fc.lo == ranges[1][0] and d.fc.step == ranges[1][2]


def test_grid_from_ranges_rejects_bad_input(lib):
    with pytest.raises(act.ActError) as e:
        act.act_grid_from_ranges(256, 256.0, (0, 256, 0), (1, 2, 1), (0, 1, 1), (0, 1, 1))
    assert e.value.status == act.ACT_ERR_INVALID_ARG
    with pytest.raises(act.ActError):
        act.act_grid_from_ranges(0, 256.0, (0, 256, 16), (1, 2, 1), (0, 1, 1), (0, 1, 1))
    with pytest.raises(act.ActError):
        act.act_grid_from_ranges(4096, 256.0, (0, 256, 16), (1, 2, 1), (0, 1, 1), (0, 1, 1))
    with pytest.raises(act.ActError):
        act.act_grid_from_ranges(256, 256.0, (5, 5, 1), (1, 2, 1), (0, 1, 1), (0, 1, 1))


def test_struct_layouts_match_header(lib):
    assert ctypes.sizeof(act.act_atom) == 40
    assert ctypes.sizeof(act.act_axis) == 24
    assert act.act_grid_desc.tc.offset == 16


def test_null_handles_are_rejected(lib):
    L = act.load_library()
    assert L.act_grid_size(None, None, None) == act.ACT_ERR_INVALID_ARG
    assert L.act_decompose(None, None, 1, 1, None, None, None, None, None) == act.ACT_ERR_INVALID_ARG
    assert L.act_dictionary_build(None, 1, None) == act.ACT_ERR_INVALID_ARG
    L.act_destroy(None)
