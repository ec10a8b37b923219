"""CPU-side checks of the C ABI: the library builds, loads and exports every symbol
declared in include/eptv.h (no compute calls without a GPU)."""
import ctypes
import os
import re

from paper_1009_2288_b300 import build as B
from paper_1009_2288_b300 import eptv as E

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "eptv.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(eptv3?_[a-z_0-9]+)\s*\(", src)))


def test_library_builds_and_exports_every_declared_symbol():
    path = B.build()
    lib = ctypes.CDLL(path)
    names = declared_functions()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(E.EXPORTED) == names


def test_default_params_and_version_without_gpu():
    p = E.params()
    assert p.n_gd == 10 and p.cgls_iters == 3 and abs(p.lam - 2000.0) < 1e-12
    assert p.max_trials == 4 and p.sigma_q == 0.9
    assert E.version().startswith("eptv-b300")


def test_python_defaults_match_library_defaults():
    from paper_1009_2288_b300.inputs import EptvParams
    a, b = E.params(), E.params(EptvParams())
    for f, _ in E.Params._fields_:
        assert getattr(a, f) == getattr(b, f), f


def test_sm103a_only_build_flags():
    assert B.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]
