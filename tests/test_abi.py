"""C-ABI library checks that need no GPU: it loads, exports every symbol the
header declares, and rejects bad descriptors on the host before any CUDA call."""
import ctypes
import os
import re

import pytest

import paper_2502_04189_b300 as F
from paper_2502_04189_b300 import _abi

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_symbols():
    txt = open(os.path.join(ROOT, "include", "fizzy_proj.h")).read()
    return sorted(set(re.findall(r"\b(fizzy_[a-z_]+)\s*\(", txt)))


def test_library_exports_every_declared_symbol():
    L = _abi.lib()
    declared = header_symbols()
    assert declared, "no declarations parsed"
    for name in declared:
        assert hasattr(L, name), name
    assert sorted(_abi.EXPORTED) == declared


def test_errstr():
    L = _abi.lib()
    assert L.fizzy_proj_errstr(0) == b"ok"
    assert L.fizzy_proj_errstr(-5) == b"not converged"
    assert L.fizzy_proj_errstr(-99) == b"unknown error"


def base(**kw):
    d = dict(nx=16, ny=12, nz=8, dx=1 / 16, dy=1 / 12, dz=1 / 8)
    d.update(kw)
    return d


@pytest.mark.parametrize("kw,code", [
    (dict(nx=1), -1), (dict(nz=1), -1), (dict(dx=0.0), -1), (dict(dz=-1.0), -1),
    (dict(rho_l=0.0), -1), (dict(rho_g=-1.0), -1), (dict(dt=0.0), -1), (dict(bcx=7), -1),
    (dict(precision=3), -1), (dict(max_refine=99), -1), (dict(nx=10), -2), (dict(ny=14), -2),
    (dict(nx=2048), -2), (dict(zf=[0.0, 0.5, 0.4, 1.0], nz=3), -1)])
def test_plan_rejects_bad_descriptors(kw, code):
    d, keep = F.make_desc(**base(**kw))
    h = ctypes.c_void_p()
    rc = _abi.lib().fizzy_proj_plan(ctypes.byref(h), ctypes.byref(d), None)
    assert rc == code
    assert not h.value
    assert _abi.lib().fizzy_proj_workspace_bytes(ctypes.byref(d)) == 0


def test_null_plan_calls_are_safe():
    L = _abi.lib()
    assert L.fizzy_proj_destroy(None) == 0
    assert L.fizzy_proj_solve(None, *([None] * 7), None, None) == -1
    assert L.fizzy_proj_plan(None, None, None) == -1
    assert L.fizzy_proj_launches_per_solve(None) == 0


def test_crop_fill_rejects_bad_arguments():
    """Argument checks run before any CUDA call."""
    import ctypes
    L = _abi.lib()
    six = (ctypes.c_void_p * 6)(*([8] * 6))
    ok = dict(tx=4, ty=4, tz=4, nx=2, ny=2, nz=2, ox=0, oy=0, oz=0, bcx=0, bcy=0)

    def call(src=six, dst=six, **kw):
        a = dict(ok, **kw)
        return L.fizzy_crop_fill(src, a["tx"], a["ty"], a["tz"], dst, a["nx"], a["ny"], a["nz"],
                                 a["ox"], a["oy"], a["oz"], a["bcx"], a["bcy"], None)
    assert call(src=None) == -1
    assert call(dst=None) == -1
    assert call(src=(ctypes.c_void_p * 6)(8, 8, 8, None, 8, 8)) == -1
    for bad in (dict(tx=0), dict(nz=0), dict(oy=-1), dict(bcx=2), dict(bcy=-1)):
        assert call(**bad) == -1, bad


def test_inject_stall_rejects_a_null_batch():
    assert _abi.lib().fizzy_proj_batch_inject_stall(None, 0, 1) == -1


def test_periodic_z_descriptor_checks():
    """periodic_z must be 0 or 1; it adds the Sherman-Morrison tables to the
    plan's footprint; the allocation-free entry point refuses it before any
    CUDA call."""
    d, keep = F.make_desc(**base())
    d.periodic_z = 2
    h = ctypes.c_void_p()
    assert _abi.lib().fizzy_proj_plan(ctypes.byref(h), ctypes.byref(d), None) == -1
    assert not h.value
    assert F.workspace_bytes(**base(periodic_z=True)) > F.workspace_bytes(**base())
    d, keep = F.make_desc(**base(periodic_z=True))
    fake = [ctypes.c_void_p(8)] * 7
    assert _abi.lib().fizzy_proj_solve_noalloc(ctypes.byref(d), *fake, None) == -2


def test_workspace_bytes_scale():
    b1 = F.workspace_bytes(**base())
    b2 = F.workspace_bytes(**base(nz=16))
    bm = F.workspace_bytes(**base(precision=1))
    assert 0 < b1 < b2
    assert bm > b1
    big = F.workspace_bytes(nx=512, ny=512, nz=512, dx=1, dy=1, dz=1, precision=1)
    assert 4e9 < big < 8e9


def test_dirichlet_and_mixed_boundary_descriptors():
    """bc 2 (Dirichlet), 3 (Neumann near, Dirichlet far) and 4 (Dirichlet
    near, Neumann far) are valid plan kinds; 3 and 4 need an even extent
    (the DCT-IV runs as a half-length complex FFT); 5 is invalid.  The
    allocation-free entry point refuses them before any CUDA call."""
    for bc in (2, 3, 4):
        assert F.workspace_bytes(**base(bcx=bc)) > 0
        assert F.workspace_bytes(**base(bcy=bc)) > 0
    assert F.workspace_bytes(**base(bcx=2, nx=27)) > 0       # DST-II: any radix-2/3 extent
    for bc in (3, 4):
        d, keep = F.make_desc(**base(bcx=bc, nx=27))
        h = ctypes.c_void_p()
        assert _abi.lib().fizzy_proj_plan(ctypes.byref(h), ctypes.byref(d), None) == -2
        assert not h.value
    d, keep = F.make_desc(**base(bcy=5))
    h = ctypes.c_void_p()
    assert _abi.lib().fizzy_proj_plan(ctypes.byref(h), ctypes.byref(d), None) == -1
    d, keep = F.make_desc(**base(bcx=2))
    fake = [ctypes.c_void_p(8)] * 7
    assert _abi.lib().fizzy_proj_solve_noalloc(ctypes.byref(d), *fake, None) == -2
    assert _abi.lib().fizzy_poisson_solve(None, None, None, None, None) == -1


def test_batch_tuning_struct_matches_header():
    """The ctypes mirror of fizzy_batch_tuning lists the header's int fields
    in the header's order (a mismatch would shift every field)."""
    import re
    from paper_2502_04189_b300 import _abi
    hdr = open(os.path.join(os.path.dirname(__file__), "..", "include", "fizzy_proj.h")).read()
    body = re.search(r"typedef struct fizzy_batch_tuning \{(.*?)\} fizzy_batch_tuning;", hdr, re.S).group(1)
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    names = re.findall(r"int\s+(\w+)\s*;", body)
    assert names == [n for n, _ in _abi.Tuning._fields_]
    assert ctypes.sizeof(_abi.Tuning) == 4 * len(names)

