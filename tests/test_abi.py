"""The C-ABI library builds, loads and exports every function include/ns3d.h declares;
host-side validation works without a GPU (no compute calls here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2211_16718_gb300 import build as B
    B.build()
    from paper_2211_16718_gb300 import ns3d
    return ns3d.lib()


def _declared_functions():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if not h.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", h)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(ns3d_\w+)\s*\(", src, flags=re.M):
            names.add(m.group(1))
    return names


def test_every_declared_symbol_is_exported(lib):
    names = _declared_functions()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), f"{n} declared in include/ but not exported"
    from paper_2211_16718_gb300 import ns3d
    assert set(ns3d.EXPORTS) <= names


def test_default_params_are_the_papers(lib):
    from paper_2211_16718_gb300 import ns3d
    p = ns3d.default_params(8, 9, 10)
    assert (p.nx, p.ny, p.nz) == (8, 9, 10)
    assert p.gamma == 1.4 and p.prandtl == 0.72 and p.weno_eps == 1e-6 and p.weno_p == 2
    assert p.rk == ns3d.NS3D_RK4 and p.precision == ns3d.NS3D_FP64 and p.mu_eff == 0.0


def test_strerror(lib):
    from paper_2211_16718_gb300 import ns3d
    for code in (0, -1, -2, -3, -4, -5, -99):
        assert isinstance(lib.ns3d_strerror(code), bytes)
    assert b"non-physical" in lib.ns3d_strerror(ns3d.NS3D_ENONPHYSICAL)


@pytest.mark.parametrize("field,value", [("nx", 0), ("ny", -3), ("lx", 0.0), ("lz", float("nan")),
                                         ("gamma", 1.0), ("mu_eff", -1e-3), ("weno_eps", 0.0), ("weno_p", 3),
                                         ("harten_delta", -0.1), ("rk", 7), ("precision", 9)])
def test_init_rejects_bad_parameters_before_touching_the_device(lib, field, value):
    from paper_2211_16718_gb300 import ns3d
    p = ns3d.default_params(8, 8, 8)
    setattr(p, field, value)
    ctx = ctypes.c_void_p()
    rc = lib.ns3d_init(ctypes.byref(p), None, ctypes.byref(ctx))
    assert rc == ns3d.NS3D_EINVAL and not ctx.value


def test_null_arguments(lib):
    from paper_2211_16718_gb300 import ns3d
    assert lib.ns3d_init(None, None, None) == ns3d.NS3D_EINVAL
    assert lib.ns3d_rhs(None, None, None) == ns3d.NS3D_EINVAL
    assert lib.ns3d_rk_step(None, None, 0.1, 1) == ns3d.NS3D_EINVAL
    assert lib.ns3d_stats(None, None, None) == ns3d.NS3D_EINVAL
    assert lib.ns3d_rhs_vjp(None, None, None, None) == ns3d.NS3D_EINVAL
    assert lib.ns3d_rk_step_vjp(None, None, None, 0.1) == ns3d.NS3D_EINVAL
    assert lib.ns3d_functional(None, None, 0, None, None) == ns3d.NS3D_EINVAL
    assert lib.ns3d_traj_forward(None, None, 0.1, 1, 1) == ns3d.NS3D_EINVAL
    assert lib.ns3d_traj_vjp(None, None) == ns3d.NS3D_EINVAL
    assert lib.ns3d_step_host(None, None, 0.1, 1, None) == ns3d.NS3D_EINVAL
    assert lib.ns3d_set_zorder(None, 0) == ns3d.NS3D_EINVAL
    assert lib.ns3d_set_variant(None, 0) == ns3d.NS3D_EINVAL
    assert lib.ns3d_dt_from_cfl(None, None, 0.4, None) == ns3d.NS3D_EINVAL
    fn = lib.ns3d_batch_set_dt_from_cfl
    fn.restype, fn.argtypes = ctypes.c_int, [ctypes.c_void_p, ctypes.c_double, ctypes.c_void_p]
    assert fn(None, 0.4, None) == ns3d.NS3D_EINVAL
    lib.ns3d_free(None)


def test_binding_refuses_without_library(monkeypatch, tmp_path):
    """No silent fallback: a missing library is a loud error."""
    from paper_2211_16718_gb300 import ns3d
    monkeypatch.setattr(ns3d, "LIBPATH", str(tmp_path / "absent.so"))
    monkeypatch.setattr(ns3d, "_lib", None)
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        ns3d.lib()
