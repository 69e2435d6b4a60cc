"""The C-ABI library loads and exports every entry point include/pipe.h
declares (no compute calls: runs without a GPU)."""
import ctypes
import os
import re

import paper_1209_3332_gb300 as P
from paper_1209_3332_gb300 import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    src = open(os.path.join(ROOT, "include", "pipe.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(?:int|void|long long|double)\s+(\w+)\s*\(", src)))


def test_library_builds_and_exports_every_declared_symbol():
    build.build()
    lib = ctypes.CDLL(P.LIB_PATH)
    names = declared()
    assert len(names) >= 13
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(P.EXPORTS) == names


def test_default_params_match_the_workload():
    p = P.default_params()
    assert (p.h, p.dome_thresh, p.area_min, p.area_max, p.glcm_levels, p.n_offsets) == (20, 10, 20, 1500, 8, 4)
    assert [tuple(o) for o in p.offsets] == [(1, 0), (0, 1), (1, 1), (1, -1)]
    assert p.hbm_budget_bytes == 40 << 30
