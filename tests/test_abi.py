"""The C-ABI library loads and exports every entry point that include/albm.h
declares; the binding's struct matches the header's field list (no GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "albm.h")


def _declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lbm_[a-z_]+)\s*\(", text)))


def _lib_path():
    from paper_1501_04741_gb300 import build
    return build.build()


def test_header_declares_the_paper_calls():
    names = _declared()
    for n in ("lbm_create", "lbm_primal_step", "lbm_objective", "lbm_adjoint_step",
              "lbm_gradient", "lbm_destroy"):
        assert n in names


def test_library_exports_every_declared_symbol():
    lib = ctypes.CDLL(_lib_path())
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_lists_every_symbol():
    from paper_1501_04741_gb300 import albm
    assert sorted(albm.EXPORTS) == _declared()


def test_params_struct_matches_header():
    from paper_1501_04741_gb300 import albm
    text = open(HEADER).read()
    body = text[text.index("typedef struct {"):text.index("} lbm_params;")]
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    fields = []
    for decl in body.split(";"):
        decl = decl.strip()
        if not decl or decl.startswith("typedef"):
            decl = decl.replace("typedef struct {", "").strip()
            if not decl:
                continue
        m = re.match(r"(int|double)\s+(.*)", decl)
        assert m, decl
        for name in m.group(2).split(","):
            fields.append(re.sub(r"\[.*\]", "", name).strip())
    assert fields == [f[0] for f in albm.LbmParams._fields_]


def test_create_without_gpu_fails_cleanly():
    import torch
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    from paper_1501_04741_gb300 import albm, inputs
    P = inputs.channel2d(dims=(8, 6, 1), nsteps=2)
    with pytest.raises(albm.AlbmError):
        albm.Solver(P, inputs.theta_uniform(P, 0), stream=0)
