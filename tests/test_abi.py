"""The C-ABI library loads and exports every function include/wf.h declares
(no GPU needed: nothing is called)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "wf.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(wf_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("wf_plan_create", "wf_solve", "wf_fluct", "wf_set_schedule", "wf_plan_destroy", "wf_strerror"):
        assert n in names


def test_library_exports_every_declared_symbol():
    import paper_1210_4931_gb300 as wf
    from paper_1210_4931_gb300 import build

    build.build()
    lib = wf.load()
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing
    assert set(wf.EXPORTS) <= set(_declared())


def test_strerror_without_gpu():
    import paper_1210_4931_gb300 as wf

    lib = wf.load()
    assert lib.wf_strerror(wf.WF_EDIVERGE) == b"diverged"
