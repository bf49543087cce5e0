"""CPU-only checks of the boundary: the library builds, loads and exports every
entry point declared in include/tp.h, and the Python binding exposes the same
names.  No compute call is made (there is no GPU here)."""

import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "tp.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(tp_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def libpath():
    from paper_2509_22110_gb300 import build

    try:
        return build.build()
    except RuntimeError as e:  # pragma: no cover
        pytest.skip(f"nvcc unavailable: {e}")


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("tp_create", "tp_destroy", "tp_mesh_upload", "tp_tree_build", "tp_energy", "tp_gradient",
              "tp_far_model_load", "tp_last_error"):
        assert n in names


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT (tp_[a-z_0-9]+)$", out, flags=re.M))
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing


def test_library_loads_and_binding_names_match(libpath):
    import ctypes

    lib = ctypes.CDLL(libpath)
    for n in declared_functions():
        assert hasattr(lib, n), n
    from paper_2509_22110_gb300 import _tp

    for n in declared_functions():
        assert hasattr(_tp, n), f"binding lacks {n}"
    assert _tp.tp_version().startswith("tpgpu")


def test_oracle_library_loads(oracle_mod):
    import ctypes

    lib = ctypes.CDLL(oracle_mod._SO)
    assert hasattr(lib, "or_energy")


def test_noalloc_binding_rejects_wrong_dtypes_on_the_host():
    """The allocation-free entry point reads V as [nv][3] FP64 and F as [nt][3] int32 on
    the device; the binding must refuse other dtypes and shapes before any call."""
    torch = pytest.importorskip("torch")
    from paper_2509_22110_gb300 import _tp

    V = torch.zeros((4, 3), dtype=torch.float64)
    F = torch.zeros((2, 3), dtype=torch.int32)
    e = torch.zeros(1, dtype=torch.float64)
    g = torch.zeros((4, 3), dtype=torch.float64)
    with pytest.raises(TypeError):
        _tp.tp_gradient_direct_noalloc(V.float(), F, e, g)
    with pytest.raises(TypeError):
        _tp.tp_gradient_direct_noalloc(V, F.long(), e, g)
    with pytest.raises(TypeError):
        _tp.tp_gradient_direct_noalloc(V, F, e, g.float())
    with pytest.raises(ValueError):
        _tp.tp_gradient_direct_noalloc(V, F, e, g[:3])
    with pytest.raises(ValueError):
        _tp.tp_gradient_direct_noalloc(V[:, :2].contiguous(), F, e, g)
    with pytest.raises(ValueError):  # host tensors: the entry point takes device pointers only
        _tp.tp_gradient_direct_noalloc(V, F, e, g)


def test_checked_build_exports_the_same_symbols(libpath):
    """The checked build (device-side bounds checks, -DTP_DEBUG=1) compiles and
    exports the same entry points as the release library."""
    from paper_2509_22110_gb300 import build

    dbg = build.build(debug=True)
    assert os.path.basename(dbg) == "libtp_debug.so"

    def exported(p):
        out = subprocess.run(["nm", "-D", "--defined-only", p], capture_output=True, text=True, check=True).stdout
        return set(re.findall(r"\bT (tp_[a-z_0-9]+)$", out, flags=re.M))

    assert exported(dbg) == exported(libpath)
