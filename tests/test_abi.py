"""The C-ABI library builds, loads without a GPU, and exports every function include/*.h
declares (no compute calls here)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*(tomg_[a-z0-9_]+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def so():
    from paper_2001_01655_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_api():
    names = declared_functions()
    for must in ["tomg_ctx_create", "tomg_problem_create", "tomg_set_fixed_dofs",
                 "tomg_set_density", "tomg_setup", "tomg_solve", "tomg_last_error"]:
        assert must in names


def test_every_declared_symbol_exported(so):
    missing = [n for n in declared_functions() if not hasattr(so, n)]
    assert not missing, missing


def test_binding_matches_header():
    from paper_2001_01655_gb300 import tomg
    assert set(tomg._SIGS) <= set(declared_functions())


def test_options_default_without_gpu(so):
    from paper_2001_01655_gb300 import tomg
    o = tomg.default_options()
    assert o.rtol == 1e-8 and o.omega == 0.5 and o.soc_beta == 0.003 and o.n_pre == o.n_post == 1
    assert o.pc == tomg.PC["gmg"] and o.max_iter == 1000


def test_no_gpu_fails_loudly(so):
    import torch
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    from paper_2001_01655_gb300 import tomg
    with pytest.raises(tomg.TomgError):
        tomg.Context(0)
