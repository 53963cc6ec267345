"""The C-ABI library builds for sm_103a, loads without a GPU and exports every
entry point declared in include/*.h (no compute call is made here)."""
import ctypes
import glob
import os
import re

from paper_2503_12473_gb300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*(cdg_[a-z0-9_]+)\s*\(", src, flags=re.M):
            names.add(m.group(1))
    return names


def test_library_exports_every_declared_symbol():
    lib = ctypes.CDLL(B.build())
    names = declared_symbols()
    assert len(names) >= 15
    missing = [n for n in sorted(names) if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_names_match_header():
    from paper_2503_12473_gb300 import oecdg
    assert set(oecdg.EXPORTED) == declared_symbols()


def test_no_cpu_fallback_in_product_path():
    """The product package never imports the oracle."""
    pkg = os.path.join(ROOT, "paper_2503_12473_gb300")
    for path in glob.glob(os.path.join(pkg, "**", "*.py"), recursive=True):
        src = open(path).read()
        assert "oracle" not in re.findall(r"^\s*(?:from|import)\s+(\w+)", src, flags=re.M), path


def _desc(**kw):
    from paper_2503_12473_gb300 import oecdg as G
    base = dict(dim=2, nx=8, ny=8, k=2, basis=G.BASIS_Q, system=G.EULER, bc=G.PERIODIC, oe=1, rk=G.RK_SSP3,
                ax=0.0, bx=1.0, ay=0.0, by=1.0, gamma=1.4, adv_x=1.0, adv_y=1.0, cfl=0.3)
    base.update(kw)
    return G.MeshDesc(**base).c()


def test_host_argument_checks_need_no_gpu():
    """Descriptor and argument checks run on the host before any CUDA call, so
    they answer here without a GPU: cdg_init_mesh, cdg_oe_damp_noalloc and
    cdg_math_eval return CDG_EINVAL / CDG_EUNSUPPORTED as include/oecdg.h states."""
    from paper_2503_12473_gb300 import oecdg as G
    L = G.load()
    EINVAL, EUNS = G.CDG_EINVAL, G.CDG_EUNSUPPORTED
    cases = [(dict(dim=3), EINVAL), (dict(nx=1), EINVAL), (dict(ny=1), EINVAL), (dict(bc=3), EINVAL),
             (dict(bc=(G.PERIODIC, G.TRANSMISSIVE, G.PERIODIC, G.PERIODIC)), EINVAL),  # unpaired periodic side
             (dict(bc=G.REFLECTIVE, system=G.ADVECTION), EINVAL), (dict(bc=G.REFLECTIVE, system=G.BURGERS), EINVAL),
             (dict(system=3), EINVAL), (dict(rk=0), EINVAL), (dict(rk=5), EINVAL), (dict(basis=2), EINVAL),
             (dict(k=0), EUNS), (dict(k=4), EUNS), (dict(bx=0.0), EINVAL), (dict(by=-1.0), EINVAL),
             (dict(cfl=0.0), EINVAL), (dict(gamma=1.0), EINVAL), (dict(nx=65536, ny=65536), EINVAL)]
    for kw, want in cases:
        d = _desc(**kw)
        h = ctypes.c_void_p(1)
        assert L.cdg_init_mesh(ctypes.byref(d), None, ctypes.byref(h)) == want, kw
        assert h.value is None, kw  # *out is NULL on error
    assert L.cdg_init_mesh(None, None, ctypes.byref(ctypes.c_void_p())) == EINVAL
    assert L.cdg_init_mesh(ctypes.byref(_desc()), None, None) == EINVAL
    # the no-alloc OE: its own scope (Q^2 / P^2 advection and Euler) and scratch limit
    a, b = ctypes.c_void_p(16), ctypes.c_void_p(32)  # never dereferenced: the checks fail first
    for kw, want in [(dict(k=3), EUNS), (dict(basis=G.BASIS_P), EUNS), (dict(system=G.BURGERS), EUNS),
                     (dict(nx=1), EINVAL), (dict(nx=2048, ny=2048), EINVAL), (dict(bc=G.REFLECTIVE), EUNS),
                     (dict(bc=(G.PERIODIC, G.PERIODIC, G.TRANSMISSIVE, G.TRANSMISSIVE)), EUNS)]:
        assert L.cdg_oe_damp_noalloc(ctypes.byref(_desc(**kw)), a, 0.1, b, None) == want, kw
    # the scratch limit, one block of 256 cells past it (the largest accepted
    # meshes run on the GPU in test_zz_no_alloc.py)
    for kw in (dict(nx=512, ny=2730),  # 2D Euler: 5,460 blocks; 5,458 fit
               dict(dim=1, nx=5589504 + 1, system=G.ADVECTION)):  # 1D advection: 21,835; 21,834 fit
        assert L.cdg_oe_damp_noalloc(ctypes.byref(_desc(**kw)), a, 0.1, b, None) == EINVAL, kw
    assert L.cdg_oe_damp_noalloc(ctypes.byref(_desc()), a, -1.0, b, None) == EINVAL
    assert L.cdg_oe_damp_noalloc(ctypes.byref(_desc()), a, 0.1, a, None) == EINVAL  # aliasing
    assert L.cdg_oe_damp_noalloc(ctypes.byref(_desc()), None, 0.1, b, None) == EINVAL
    # the kernels' reciprocal / square root entry: bad op, null pointers, and n = 0 (no launch)
    assert L.cdg_math_eval(7, a, 4, b, None) == EINVAL
    assert L.cdg_math_eval(G.MATH_SQRT, None, 4, b, None) == EINVAL
    assert L.cdg_math_eval(G.MATH_RCP, None, 0, None, None) == G.CDG_OK
    assert L.cdg_last_error(None) == b""


def test_binding_fails_loudly_without_device_memory():
    """No CPU fallback: the binding refuses host tensors and arrays, and on a
    machine without a GPU creating a context raises instead of running
    anything on the CPU."""
    import numpy as np
    import pytest
    import torch
    from paper_2503_12473_gb300 import oecdg as G
    assert G._ptr(None) is None
    with pytest.raises(ValueError):
        G._ptr(torch.zeros(3, dtype=torch.float64))
    with pytest.raises(TypeError):
        G._ptr(np.zeros(3))
    if not torch.cuda.is_available():
        with pytest.raises(Exception):
            G.Context(G.MeshDesc(nx=8, ny=8))


def test_noalloc_binding_checks_sizes_and_devices_before_any_launch():
    """cdg_oe_damp_noalloc takes its sizes from the mesh description alone, so
    the binding refuses, before loading or launching anything, tensors whose
    element count is not the description's state size, and states that are
    not device memory."""
    import pytest
    import torch
    from paper_2503_12473_gb300 import oecdg as G
    desc = G.MeshDesc(dim=2, nx=8, ny=6)
    n = 2 * 4 * 9 * 8 * 6
    good = torch.zeros(n, dtype=torch.float64)
    short = torch.zeros(n - 1, dtype=torch.float64)
    for a, b in ((short, good), (good, short)):
        with pytest.raises(ValueError, match="elements"):
            G.cdg_oe_damp_noalloc(desc, a, 1e-3, b)
    with pytest.raises(ValueError):  # host memory, right size: refused, no CPU fallback
        G.cdg_oe_damp_noalloc(desc, good, 1e-3, good.clone())
    with pytest.raises(TypeError):
        G.cdg_oe_damp_noalloc(desc, good.numpy(), 1e-3, good)
