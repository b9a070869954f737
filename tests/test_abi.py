"""The C-ABI library builds for sm_103a, loads, and exports every function
include/*.h declares (ecg.h and ecg_nn.h).  No compute call is made
(CPU-only test)."""
import os
import re

import pytest

from paper_2305_19013_gb300 import build as B
from paper_2305_19013_gb300 import ecg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions(only=None):
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if only and fn != only:
            continue
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"^\s*(?:int|void|size_t|const char\s*\*)\s+(ecg_\w+)\s*\(", text, flags=re.M)
    return names


def test_header_declares_the_boundary():
    names = declared_functions("ecg.h")
    for required in ("ecg_create", "ecg_solve", "ecg_destroy", "ecg_strerror"):
        assert required in names
    assert set(names) == set(ecg.SIGNATURES), "binding and header disagree"
    from paper_2305_19013_gb300 import warmstart

    assert set(declared_functions("ecg_nn.h")) == set(warmstart.SIGNATURES), "network binding and header disagree"


def test_library_builds_loads_and_exports_every_symbol():
    path = B.build()
    assert os.path.exists(path)
    lib = ecg.load()
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_strerror_and_no_device_failure():
    lib = ecg.load()
    assert ecg.strerror(0) == "converged"
    assert "breakdown" in ecg.strerror(-4)
    import torch

    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import numpy as np

    from paper_2305_19013_gb300 import workloads as W

    p = W.poisson2d(8, 2, seed=1)
    with pytest.raises(ecg.EcgError) as ei:
        ecg.Solver.from_problem(p)
    assert ei.value.code == ecg.ECUDA
