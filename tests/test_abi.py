"""The C-ABI library builds for sm_103a, loads, and exports every entry point
that include/gc.h declares (no GPU needed: nothing is computed here)."""
import ctypes
import os
import re

from paper_1710_01144_gb300 import build as gcbuild
from paper_1710_01144_gb300 import gc

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_entry_points():
    hdrs = [os.path.join(ROOT, "include", f) for f in os.listdir(os.path.join(ROOT, "include"))
            if f.endswith(".h")]
    names = set()
    for h in hdrs:
        text = re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
        names |= set(re.findall(r"\b(gc_[a-z0-9_]+)\s*\(", text))
    return names


def test_library_builds_and_exports_every_declared_symbol():
    path = gcbuild.build()
    lib = ctypes.CDLL(path)
    names = declared_entry_points()
    assert {"gc_load_csr", "gc_group_farness", "gc_marginal_gains", "gc_greedy"} <= names
    for name in names:
        assert hasattr(lib, name), name


def test_binding_lists_header_symbols():
    assert declared_entry_points() <= set(gc.EXPORTS)


def test_struct_layouts_match_header():
    text = open(os.path.join(ROOT, "include", "gc.h")).read()
    opts = re.sub(r"/\*.*?\*/", "", text[text.index("typedef struct gc_opts"):text.index("} gc_opts;")], flags=re.S)
    ofields = re.findall(r"(int32_t|uint32_t)\s+(\w+);", opts)
    assert [f for _, f in ofields] == [f for f, _ in gc.Opts._fields_]
    assert ctypes.sizeof(gc.Opts) == 4 * len(ofields)
    assert ctypes.sizeof(gc.Stats) == 8 * 57
    stats = text[text.index("typedef struct gc_stats"):text.index("} gc_stats;")]
    fields = re.findall(r"(int64_t|double)\s+(\w+);", stats)
    assert [f for _, f in fields] == [f for f, _ in gc.Stats._fields_]
