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


def test_cone_geometry_argument_errors_without_gpu():
    """eptv3_create_geometry validates its descriptor before it touches the device: sizes,
    pitches, the source inside the volume's circle, more than 65535 views -- each comes
    back as EPTV_ERR_ARG with a message, and no handle."""
    import pytest
    from paper_1009_2288_b300 import inputs as I
    base = dict(nx=16, ny=16, nz=24, dx=1.0, dy=1.0, dz=1.0, n_views=12, nu=40, nv=64, du=0.9, dv=0.5,
                u_off=0.25, v_off=0.1, sid=30.0, sdd=45.0)
    for change, msg in ((dict(nx=0), "sizes"), (dict(du=0.0), "pitches"), (dict(sid=11.0), "half-diagonal"),
                        (dict(sdd=25.0), "half-diagonal"), (dict(n_views=70000), "65535 views")):
        d = dict(base, **change)
        with pytest.raises(E.EptvError) as ei:
            E.Geometry3(I.ConeGeometry(**d))
        assert ei.value.code == -1 and msg in str(ei.value), change
