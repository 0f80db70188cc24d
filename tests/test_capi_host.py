"""Host-side checks of the C ABI (CPU, no compute calls).

The library must build, load, and export every symbol the public header
declares; the Python binding exposes the same names.
"""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", n) for n in ("scal3r_ttt.h", "scal3r_gcm.h")]


def _declared():
    src = "".join(open(h).read() for h in HEADERS)
    return sorted(set(re.findall(r"\b(scal3r_(?:ttt|gcm)_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def libpath():
    from paper_2604_08542_gb300 import build
    return build.build()


def test_header_declares_the_abi():
    names = _declared()
    for n in ("scal3r_ttt_init", "scal3r_ttt_forward", "scal3r_ttt_backward", "scal3r_ttt_destroy",
              "scal3r_ttt_workspace_size", "scal3r_ttt_plan", "scal3r_ttt_get_status",
              "scal3r_ttt_error_string"):
        assert n in names


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\sT\s+(scal3r_(?:ttt|gcm)_\w+)", out))
    missing = [n for n in _declared() if n not in exported]
    assert not missing, missing


def test_library_loads_and_binding_names_match(libpath):
    import ctypes
    import paper_2604_08542_gb300 as ttt
    lib = ctypes.CDLL(libpath)
    for n in _declared():
        assert hasattr(lib, n)
        assert hasattr(ttt, n), f"binding lacks {n}"
    assert ttt.load_library().scal3r_ttt_error_string(0) == b"ok"
    assert "timed out" in ttt.error_string(ttt.SCAL3R_ERR_TIMEOUT)


def test_init_without_a_device_fails_cleanly(libpath):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import paper_2604_08542_gb300 as ttt
    cfg = ttt.scal3r_ttt_config(16, 64, 128, ttt.SCAL3R_BF16, 0, 0, 1e-6, 0)
    with pytest.raises(ttt.Scal3rError) as e:
        ttt.scal3r_ttt_init(cfg)
    assert e.value.status in (ttt.SCAL3R_ERR_NO_DEVICE, ttt.SCAL3R_ERR_CUDA)


def test_config_struct_matches_the_header(libpath):
    # the binding's structure has the header's fields in the header's order
    import re
    import paper_2604_08542_gb300 as ttt
    hdr = open(os.path.join(ROOT, "include", "scal3r_ttt.h")).read()
    body = hdr[hdr.index("typedef struct scal3r_ttt_config {"):hdr.index("} scal3r_ttt_config;")]
    names = re.findall(r"^\s*(?:int32_t|float)\s+(\w+);", body, flags=re.M)
    assert names == [n for n, _ in ttt.scal3r_ttt_config._fields_]
    assert ttt.scal3r_ttt_config(1, 64, 128, 1, 0, 0, 1e-6, 0).deterministic == 1


def test_bad_config_rejected_before_device_query(libpath):
    import paper_2604_08542_gb300 as ttt
    bad = [ttt.scal3r_ttt_config(0, 64, 128, 1, 0, 0, 1e-6, 0),        # no heads
           ttt.scal3r_ttt_config(16, 64, 128, 7, 0, 0, 1e-6, 0),       # bad dtype
           ttt.scal3r_ttt_config(16, 64, 128, 1, 5, 0, 1e-6, 0),       # bad loss
           ttt.scal3r_ttt_config(16, 64, 128, 1, 0, 9, 1e-6, 0),       # bad norm
           ttt.scal3r_ttt_config(16, 64, 128, 1, 0, 0, 1e-6, -1),      # negative checkpoint interval
           ttt.scal3r_ttt_config(16, 64, 128, 1, 0, 0, 1e-6, 0, 2),    # bad rate layout
           ttt.scal3r_ttt_config(16, 64, 128, 1, 0, 0, 1e-6, 0, 0, 2),  # bad model
           ttt.scal3r_ttt_config(16, 64, 128, 1, 0, 0, 1e-6, 0, 0, 0, 3)]   # bad determinism flag
    for c in bad:
        with pytest.raises(ttt.Scal3rError) as e:
            ttt.scal3r_ttt_init(c)
        assert e.value.status == ttt.SCAL3R_ERR_INVALID_ARG
    for c in (ttt.scal3r_ttt_config(16, 32, 128, 1, 0, 0, 1e-6, 0),     # BF16 needs D=64, F=128 or wide
              ttt.scal3r_ttt_config(16, 48, 100, 0, 0, 0, 1e-6, 0),     # FP32 shape not built
              ttt.scal3r_ttt_config(4, 64, 64, 1, 0, 0, 1e-6, 0, 0, 1),  # linear model: float32 only
              ttt.scal3r_ttt_config(4, 64, 128, 0, 0, 0, 1e-6, 0, 0, 1),  # linear model: hidden_dim = head_dim
              ttt.scal3r_ttt_config(4, 64, 64, 0, 0, 0, 1e-6, 0, 1, 1)):  # linear model: one rate per token
        with pytest.raises(ttt.Scal3rError) as e:
            ttt.scal3r_ttt_init(c)
        assert e.value.status == ttt.SCAL3R_ERR_UNSUPPORTED
