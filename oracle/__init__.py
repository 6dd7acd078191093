"""FP64 CPU oracle of the variable-density pressure-correction projection.

TEST INFRASTRUCTURE ONLY: tests/, ``__graft_entry__.smoke()`` and the CPU
baseline / reference leg of ``bench.py`` are the only callers.  The product
path (the CUDA library and its binding) never imports this package, and this
package imports nothing from the product.

``oracle.c`` holds the plain definitions (see its header); this module builds
it with gcc (OpenMP over independent lines) and wraps it with numpy arrays.
``exact.py`` holds an exact rational-arithmetic restatement for tiny grids.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "_oracle.so")
# tests that plant mistakes in a copy of oracle.c load that copy through this variable
_ALT = os.environ.get("FIZZY_ORACLE_SO")
_lock = threading.Lock()
_lib = None

PERIODIC = 0
NEUMANN = 1


def build(force: bool = False) -> str:
    """Compile oracle.c into _oracle.so (gcc -O2 -fopenmp)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=gnu11", "-o", tmp, _SRC, "-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            if _ALT:
                L = ctypes.CDLL(_ALT)
            else:
                build()
                L = ctypes.CDLL(_LIB)
            d = ctypes.POINTER(ctypes.c_double)
            I, D = ctypes.c_int, ctypes.c_double
            g = [I, I, I, D, D, d, I, I, I]  # nx ny nz dx dy zf bcx bcy bcz
            L.ora_grad.argtypes = g + [d, d, d, d]
            L.ora_div.argtypes = g + [d, d, d, d]
            L.ora_apply_L.argtypes = g + [d, d]
            L.ora_rhs.argtypes = g + [D, D, D, d, d, d, d, d, d, d]
            L.ora_correct.argtypes = g + [D, D, D, d, d, d, d, d, d, d]
            L.ora_poisson_fft.argtypes = g + [d, d]
            L.ora_poisson_fft.restype = I
            L.ora_poisson_dense.argtypes = g + [d, d]
            L.ora_poisson_dense.restype = I
            L.ora_project.argtypes = g + [D, D, D, d, d, d, d, d, d, d, d, d, I]
            L.ora_project.restype = I
            L.ora_apply_vc.argtypes = g + [D, D, d, d, d]
            L.ora_project_vc.argtypes = g + [D, D, D, d, d, d, d, d, d]
            L.ora_project_vc.restype = I
            L.ora_acdi_rhs.argtypes = g + [D, D, D, d, d, d, d, d]
            L.ora_fft.argtypes = [I, d, d, d, d, I]
            L.ora_dft.argtypes = [I, d, d, d, d, I]
            L.ora_weighted_mean.argtypes = [I, I, I, d, d]
            L.ora_weighted_mean.restype = D
            L.ora_num_threads.restype = I
            _lib = L
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _c(a):
    return np.ascontiguousarray(a, dtype=np.float64)


class Grid:
    """Grid of nx*ny*nz cells; zf = nz+1 z face coordinates; bcx/bcy/bcz 0 periodic,
    1 walls (z defaults to walls)."""

    def __init__(self, nx, ny, nz, dx, dy, zf, bcx=PERIODIC, bcy=PERIODIC, bcz=NEUMANN):
        self.nx, self.ny, self.nz = int(nx), int(ny), int(nz)
        self.dx, self.dy = float(dx), float(dy)
        self.zf = _c(zf)
        assert self.zf.shape == (self.nz + 1,)
        self.bcx, self.bcy, self.bcz = int(bcx), int(bcy), int(bcz)

    @property
    def shape(self):
        return (self.nz, self.ny, self.nx)

    def args(self):
        return (self.nx, self.ny, self.nz, self.dx, self.dy, _p(self.zf), self.bcx, self.bcy,
                self.bcz)

    @classmethod
    def of_case(cls, case):
        s = case.spec
        return cls(s.nx, s.ny, s.nz, case.dx, case.dy, case.zf, s.bcx, s.bcy,
                   getattr(s, "bcz", NEUMANN))


def grad(g: Grid, q):
    q = _c(q)
    gx, gy, gz = (np.empty(g.shape) for _ in range(3))
    lib().ora_grad(*g.args(), _p(q), _p(gx), _p(gy), _p(gz))
    return gx, gy, gz


def div(g: Grid, u, v, w):
    u, v, w = _c(u), _c(v), _c(w)
    out = np.empty(g.shape)
    lib().ora_div(*g.args(), _p(u), _p(v), _p(w), _p(out))
    return out


def apply_L(g: Grid, p):
    p = _c(p)
    out = np.empty(g.shape)
    lib().ora_apply_L(*g.args(), _p(p), _p(out))
    return out


def weighted_mean(g: Grid, a):
    a = _c(a)
    return lib().ora_weighted_mean(g.nx, g.ny, g.nz, _p(g.zf), _p(a))


def rhs(g: Grid, rho_l, rho_g, dt, phi, pn, pnm1, u, v, w):
    arrs = [_c(a) for a in (phi, pn, pnm1, u, v, w)]
    f = np.empty(g.shape)
    lib().ora_rhs(*g.args(), rho_l, rho_g, dt, *[_p(a) for a in arrs], _p(f))
    return f


def correct(g: Grid, rho_l, rho_g, dt, phi, pn, pnm1, p, u, v, w):
    """Returns corrected copies of u, v, w."""
    arrs = [_c(a) for a in (phi, pn, pnm1, p)]
    uo, vo, wo = (np.array(a, dtype=np.float64, copy=True, order="C") for a in (u, v, w))
    lib().ora_correct(*g.args(), rho_l, rho_g, dt, *[_p(a) for a in arrs], _p(uo), _p(vo), _p(wo))
    return uo, vo, wo


def poisson(g: Grid, f, dense: bool = False):
    f = _c(f)
    p = np.empty(g.shape)
    fn = lib().ora_poisson_dense if dense else lib().ora_poisson_fft
    st = fn(*g.args(), _p(f), _p(p))
    if st != 0:
        raise RuntimeError("oracle poisson failed with status %d" % st)
    return p


def project(g: Grid, rho_l, rho_g, dt, phi, pn, pnm1, u, v, w, dense: bool = False):
    """Whole projection.  Returns dict(p, u, v, w, f, relres, divmax, fmax)."""
    arrs = [_c(a) for a in (phi, pn, pnm1)]
    uo, vo, wo = (np.array(a, dtype=np.float64, copy=True, order="C") for a in (u, v, w))
    p = np.empty(g.shape)
    f = np.empty(g.shape)
    diag = np.zeros(3)
    st = lib().ora_project(*g.args(), rho_l, rho_g, dt, *[_p(a) for a in arrs], _p(uo), _p(vo),
                           _p(wo), _p(p), _p(f), _p(diag), 1 if dense else 0)
    if st != 0:
        raise RuntimeError("oracle projection failed with status %d" % st)
    return dict(p=p, u=uo, v=vo, w=wo, f=f, relres=diag[0], divmax=diag[1], fmax=diag[2])


def project_case(case, dense: bool = False):
    s = case.spec
    return project(Grid.of_case(case), s.rho_l, s.rho_g, s.dt, case.phi, case.pn, case.pnm1,
                   case.u, case.v, case.w, dense=dense)


def apply_vc(g: Grid, rho_l, rho_g, phi, p):
    """D(beta_f G p), beta_f = 1/rho_f (the unsplit variable-coefficient operator)."""
    phi, p = _c(phi), _c(p)
    out = np.empty(g.shape)
    lib().ora_apply_vc(*g.args(), rho_l, rho_g, _p(phi), _p(p), _p(out))
    return out


def project_vc(g: Grid, rho_l, rho_g, dt, phi, u, v, w):
    """Variable-coefficient projection without splitting, dense (<= 4096 cells):
    D(beta_f G p) = D(u*)/dt, u = u* - dt beta_f G p.
    Returns dict(p, u, v, w, relres, divmax)."""
    phi = _c(phi)
    uo, vo, wo = (np.array(a, dtype=np.float64, copy=True, order="C") for a in (u, v, w))
    p = np.empty(g.shape)
    diag = np.zeros(2)
    st = lib().ora_project_vc(*g.args(), rho_l, rho_g, dt, _p(phi), _p(uo), _p(vo), _p(wo), _p(p),
                              _p(diag))
    if st != 0:
        raise RuntimeError("oracle variable-coefficient projection failed with status %d" % st)
    return dict(p=p, u=uo, v=vo, w=wo, relres=diag[0], divmax=diag[1])


def acdi_rhs(g: Grid, eps, gam, phi, u, v, w, delta=1e-100):
    """Right-hand side of the ACDI phase-field transport (Jain 2022) in
    conservative face-flux form: d phi/dt = rhs."""
    arrs = [_c(a) for a in (phi, u, v, w)]
    out = np.empty(g.shape)
    lib().ora_acdi_rhs(*g.args(), eps, gam, delta, *[_p(a) for a in arrs], _p(out))
    return out


def fft(x, sign=-1):
    x = np.asarray(x, dtype=np.complex128)
    n = x.size
    re, im = _c(x.real), _c(x.imag)
    orr, oi = np.empty(n), np.empty(n)
    lib().ora_fft(n, _p(re), _p(im), _p(orr), _p(oi), int(sign))
    return orr + 1j * oi


def dft(x, sign=-1):
    x = np.asarray(x, dtype=np.complex128)
    n = x.size
    re, im = _c(x.real), _c(x.imag)
    orr, oi = np.empty(n), np.empty(n)
    lib().ora_dft(n, _p(re), _p(im), _p(orr), _p(oi), int(sign))
    return orr + 1j * oi


def num_threads() -> int:
    return lib().ora_num_threads()
