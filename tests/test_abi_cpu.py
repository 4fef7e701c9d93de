"""The C ABI library builds, loads and exports what include/*.h declares;
invalid inputs are rejected on the host with clear errors (no GPU needed)."""
import ctypes
import glob
import os
import re

import numpy as np
import pytest

from paper_2406_13881_b300 import _native, build, workload as wl

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(ompdart_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return names


def test_library_builds_and_exports_every_declared_symbol():
    build.build()
    lib = ctypes.CDLL(_native.LIB_PATH)
    names = declared_functions()
    assert {"ompdart_analyze", "ompdart_plan_create", "ompdart_plan_run"} <= names
    for n in sorted(names):
        assert hasattr(lib, n), n
    # and the binding declares every one of them
    assert names <= set(_native.EXPORTS), sorted(names - set(_native.EXPORTS))


@pytest.mark.parametrize("case,msg", [
    ("entry_pred", "entry block must have no predecessors"),
    ("var_range", "access variable out of range"),
    ("succ_range", "successor id out of range"),
    ("kind_zero", "access kind"),
    ("reserved", "reserved access bits"),
    ("offsets", "non-decreasing"),
])
def test_invalid_inputs_rejected_on_host(case, msg):
    g = wl.from_lists([[1], [2], []], [[(0, 1, 0)], [(1, 2, 1)], []], 4)
    if case == "entry_pred":
        g.succ = np.array([1, 2, 0], dtype=np.int32)
        g.succ_off = np.array([0, 1, 2, 3], dtype=np.int32)
    elif case == "var_range":
        g.acc = g.acc.copy(); g.acc[0] = wl.pack_access([9], [1], [0])[0]
    elif case == "succ_range":
        g.succ = np.array([1, 7], dtype=np.int32)
    elif case == "kind_zero":
        g.acc = g.acc.copy(); g.acc[0] = np.uint32(3)
    elif case == "reserved":
        g.acc = g.acc.copy(); g.acc[0] |= np.uint32(1 << 28)
    elif case == "offsets":
        g.succ_off = np.array([0, 2, 1, 2], dtype=np.int32)
    with pytest.raises(_native.OmpdartError) as ei:
        _native.analyze(g)
    assert ei.value.code == _native.E_INVALID
    assert msg in str(ei.value)


def test_call_accesses_without_table_rejected():
    g = wl.from_lists([[1], []], [[], []], 2)
    g.acc = np.array([0x80000000], dtype=np.uint32)
    g.acc_off = np.array([0, 1, 1], dtype=np.int32)
    with pytest.raises(_native.OmpdartError) as ei:
        _native.analyze(g)
    assert ei.value.code == _native.E_INVALID


@pytest.mark.parametrize("first,later,msg", [
    ("kind_zero", "var_range", "access kind"),
    ("var_range", "kind_zero", "access variable out of range"),
    ("succ_range", "entry_pred", "successor id out of range"),
    ("entry_pred", "succ_range", "entry block must have no predecessors"),
])
def test_first_invalid_entry_decides_on_large_inputs(first, later, msg):
    """Large inputs are checked in parallel ranges; the message is still the
    one of the lowest-indexed bad entry, as in a sequential scan."""
    n, per = 300_000, 4
    succ_off = np.arange(n + 1, dtype=np.int32)
    succ_off[-1] = n - 1                      # the last block has no successor
    succ = np.arange(1, n, dtype=np.int32)
    acc_off = (np.arange(n + 1) * per).astype(np.int32)
    acc = wl.pack_access(np.arange(n * per) % 8, np.full(n * per, 1), np.zeros(n * per, dtype=np.int64))
    acc = np.asarray(acc, dtype=np.uint32).copy()
    bad = {"kind_zero": lambda i: acc.__setitem__(i, np.uint32(3)),
           "var_range": lambda i: acc.__setitem__(i, wl.pack_access([9], [1], [0])[0]),
           "succ_range": lambda i: succ.__setitem__(i, n + 5),
           "entry_pred": lambda i: succ.__setitem__(i, 0)}
    lo, hi = (10, len(acc) - 5) if first in ("kind_zero", "var_range") else (5, len(succ) - 3)
    bad[first](lo)
    bad[later](hi)
    g = wl.CFG(n_blocks=n, n_vars=8, entry=0, succ_off=succ_off, succ=succ, acc_off=acc_off, acc=acc)
    with pytest.raises(_native.OmpdartError) as ei:
        _native.analyze(g)
    assert ei.value.code == _native.E_INVALID
    assert msg in str(ei.value)
