"""The bounds-checking build of the library (SCAL3R_DEBUG_BOUNDS).

It stands in for an allocation-level memory checker.  Each forward or
backward call on a wide-weight handle registers the byte range of every
tensor it was given and of its workspace.  Every plain global load and store
of the wide-weight kernels must then fall inside one of those ranges; one
that does not is skipped and reported as SCAL3R_ERR_BOUNDS.  The tests:

  * CPU: the variant builds and exports the whole ABI;
  * GPU: forward and backward on ragged layouts report no violation and
    still match the oracle, under both losses and per-matrix rates, with a
    chunk long enough for the weight-sized reductions to split over K;
  * GPU: registering o 32 bytes short is reported, and the one store that
    falls outside is skipped, while every access stays inside the real
    buffer (nothing is made to fault).

The GPU cases run in a child process so that the package loads the
bounds-checking library there (SCAL3R_TTT_LIBRARY).
"""
import ctypes
import json
import os
import re
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", h) for h in ("scal3r_ttt.h", "scal3r_gcm.h")]
TOL = 2e-2


def _bounds_lib():
    from paper_2604_08542_gb300 import build as b
    try:
        b._nvcc()
    except RuntimeError as e:   # no nvcc on this machine
        pytest.skip(str(e))
    return b.build(variant="bounds")   # a compile error fails the test


def _declared():
    names = set()
    for h in HEADERS:
        names |= set(re.findall(r"\b(scal3r_(?:ttt|gcm)_\w+)\s*\(", open(h).read()))
    return names


def test_bounds_variant_builds_and_exports_the_abi():
    lib = ctypes.CDLL(_bounds_lib())
    missing = [n for n in sorted(_declared()) if not hasattr(lib, n)]
    assert not missing, missing


@pytest.mark.gpu
def test_ordinary_build_reports_no_bounds_checking():
    import torch
    import paper_2604_08542_gb300 as ttt
    layer = ttt.TTT(1, 256, 512, dtype=torch.bfloat16)
    assert ttt.scal3r_ttt_debug_bounds(layer.handle, -1, 0) == ttt.SCAL3R_ERR_UNSUPPORTED
    layer.close()


@pytest.mark.gpu
def test_bounds_build_clean_runs_and_planted_violation():
    lib = _bounds_lib()
    env = dict(os.environ, SCAL3R_TTT_LIBRARY=lib)
    r = subprocess.run([sys.executable, os.path.join(ROOT, "tests", "_bounds_child.py")], env=env,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    out = json.loads(r.stdout.strip().splitlines()[-1])
    assert out["library"] == lib
    for case in ("dot", "dot_per_matrix", "mse", "d64_dot", "d64_per_matrix_ckpt2", "d64_mse"):
        res = out[case]
        assert res["status"] == 0, (case, res)
        bad = {n: e for n, e in res["errors"].items() if not e <= TOL}
        assert not bad, (case, res["errors"])
    for case in ("planted", "d64_planted"):
        p = out[case]
        assert p["status"] == 9, (case, p)     # SCAL3R_ERR_BOUNDS
        assert p["tail_untouched"] and p["before_tail_written"], (case, p)
        assert p["status_after_restore"] == 0, (case, p)
