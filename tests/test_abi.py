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


def test_solve_records_as_json_lines(tmp_path):
    """Per-solve metrics log: one JSON object per line with the trace, timing
    percentiles, chi^2 / n_dof and the caller's fields (no GPU needed)."""
    import json

    import numpy as np

    import paper_1210_4931_gb300 as wf

    rep = {"status": wf.WF_OK, "iters": 3, "converged": True, "final_residual": 5e-7, "chi2_over_ndof": 0.998,
           "n_dof": 1200, "tau": 0.01, "launches": 24, "refine_sweeps": 0, "mixed_lc": 0,
           "iter_ms_trace": np.array([1.0, 2.0, 3.0]), "lambda_trace": np.array([4.0, 1.0, 1.0]),
           "L_trace": np.array([10, 32, 32], dtype=np.int32)}
    path = tmp_path / "solves.jsonl"
    wf.append_jsonl(str(path), rep, nside=16, lmax=32)
    wf.append_jsonl(str(path), dict(rep, iters=4), nside=16, lmax=32, err_vs_oracle=3e-12)
    lines = [json.loads(x) for x in path.read_text().splitlines()]
    assert len(lines) == 2 and lines[1]["iters"] == 4 and lines[1]["err_vs_oracle"] == 3e-12
    assert lines[0]["iter_ms_p50"] == 2.0 and lines[0]["lambda_trace"] == [4.0, 1.0, 1.0]
    assert lines[0]["L_trace"] == [10, 32, 32] and lines[0]["chi2_over_ndof"] == 0.998


def test_binding_structs_match_the_library():
    """Every struct the binding mirrors has the size the library was built with
    (load() refuses a library whose layouts differ); unknown names give 0."""
    import ctypes

    import paper_1210_4931_gb300 as wf

    lib = wf.load()
    for st in wf.ABI_STRUCTS:
        assert lib.wf_abi_sizeof(st.__name__.encode()) == ctypes.sizeof(st), st.__name__
    assert lib.wf_abi_sizeof(b"wf_plan") == 0 and lib.wf_abi_sizeof(None) == 0
    # every struct the header defines is covered
    src = re.sub(r"/\*.*?\*/", "", open(os.path.join(ROOT, "include", "wf.h")).read(), flags=re.S)
    defined = set(re.findall(r"typedef struct\s*\{[^{}]*\}\s*(wf_[a-z_]+)\s*;", src))
    assert defined == {st.__name__ for st in wf.ABI_STRUCTS}
