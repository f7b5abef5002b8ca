"""The C ABI: libbyo.so builds for sm_103a, loads without a GPU, and exports
every function that include/byo.h declares; the Python binding covers them all.
No compute call is made here."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "byo.h")


def _declared():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(byo_[a-z0-9_]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def lib():
    from paper_2405_11671_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_hot_path_calls():
    names = set(_declared())
    for want in ("byo_graph_build", "byo_insert_batch", "byo_delete_batch", "byo_degree", "byo_num_vertices",
                 "byo_num_edges", "byo_bfs", "byo_cc", "byo_pagerank", "byo_tc"):
        assert want in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    from paper_2405_11671_gb300 import _byo
    bound = {name for name, _, _ in _byo.SIGNATURES}
    assert set(_declared()) <= bound, set(_declared()) - bound


def test_binding_struct_layouts():
    from paper_2405_11671_gb300 import _byo
    assert ctypes.sizeof(_byo.byo_bfs_iter) == 72
    assert _byo.byo_bfs_iter.t_ns.offset == 64
    assert ctypes.sizeof(_byo.byo_sched) == 40 and _byo.byo_sched.mlp.offset == 24
    assert _byo.byo_sched.action.offset == 32 and _byo.byo_sched.flags.offset == 36


def test_binding_constants_match_header():
    """Every numeric #define of include/byo.h has the same value in the binding."""
    from paper_2405_11671_gb300 import _byo
    txt = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    defs = re.findall(r"^#define[ \t]+(BYO_[A-Z0-9_]+)[ \t]+(\S.*?)[ \t]*$", txt, flags=re.M)
    assert len(defs) >= 8
    for name, val in defs:
        plain = re.fullmatch(r"(0x[0-9A-Fa-f]+|\d+)u?", val)
        shift = re.fullmatch(r"\((\d+)u?\s*<<\s*(\d+)\)", val)
        assert plain or shift, (name, val)
        want = int(plain.group(1), 0) if plain else int(shift.group(1)) << int(shift.group(2))
        assert hasattr(_byo, name), name
        assert getattr(_byo, name) == want, name
