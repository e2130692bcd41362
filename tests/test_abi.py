"""The C-ABI library builds for sm_103a, loads without a GPU and exports every
entry point include/tomo.h declares; the binding's signatures cover them."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "tomo.h")


def declared():
    src = open(HEADER).read()
    return sorted(set(re.findall(r"TOMO_API\s+[\w\s\*]+?\b((?:tomo|dadmm|quant)_\w+)\s*\(", src)))


@pytest.fixture(scope="module")
def libpath():
    from paper_2410_06106_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = declared()
    for want in ("tomo_geometry_create", "tomo_project", "tomo_backproject", "dadmm_step",
                 "quant_kmeans", "quant_jpeg", "dadmm_create", "tomo_last_error"):
        assert want in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_signatures_match_header(libpath):
    from paper_2410_06106_gb300 import api
    assert set(declared()) <= set(api.SIGNATURES)


def test_calls_without_gpu_fail_loudly(libpath):
    """no CPU fallback: without a device the first call reports a CUDA error"""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2410_06106_gb300 import api
    with pytest.raises(api.TomoError):
        api.Geometry(8, 13, A=4)


def test_binding_constants_match_header():
    """the binding's mode, variant and launch-shape codes are the header's"""
    from paper_2410_06106_gb300 import api
    src = open(HEADER).read()
    defs = dict((k, int(v)) for k, v in re.findall(r"#define\s+(DADMM_\w+)\s+(-?\d+)", src))
    assert defs["DADMM_MODE_BATCHED"] == api.MODE_BATCHED and defs["DADMM_MODE_PLAIN"] == api.MODE_PLAIN
    assert defs["DADMM_VARIANT_SEGMENTS"] == 0 and defs["DADMM_VARIANT_CONSENSUS"] == 1
    tunes = {"wide": "DADMM_TUNE_WIDE", "auto": "DADMM_TUNE_AUTO", "narrow": "DADMM_TUNE_NARROW",
             "pairs": "DADMM_TUNE_PAIRS", "quads": "DADMM_TUNE_QUADS", "widepairs": "DADMM_TUNE_WIDE_PAIRS"}
    code = open(os.path.join(ROOT, "paper_2410_06106_gb300", "api.py")).read()
    mapping = dict(re.findall(r'"(\w+)": (\d+)', code[code.index("tunes = {"):code.index("}", code.index("tunes = {"))]))
    assert {k: int(v) for k, v in mapping.items()} == {k: defs[v] for k, v in tunes.items()}
