"""B300-native variable-density pressure-correction projection (CaNS-Fizzy hot path).

Python binding of the C ABI in include/fizzy_proj.h.  Every step of the
projection runs in the CUDA library libfizzyproj.so; this module only
marshals arguments (torch tensors provide device pointers and streams).
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _abi
from ._abi import Stats

PERIODIC = 0
NEUMANN = 1
DIRICHLET = 2             # p = 0 on both boundary faces (fizzy_poisson_solve only)
NEUMANN_DIRICHLET = 3     # zero flux near, p = 0 far (fizzy_poisson_solve only)
DIRICHLET_NEUMANN = 4     # p = 0 near, zero flux far (fizzy_poisson_solve only)
FP64 = 0
MIXED = 1
FLAG_CHECK = 1
FLAG_FUSED_XY = 4  # cluster-fused x-y FP32 passes (mixed, nx = ny = 256 or 512)


class FizzyError(RuntimeError):
    def __init__(self, code, msg=""):
        self.code = code
        super().__init__("fizzy_proj error %d (%s)%s" % (code, _abi.ERRORS.get(code, "?"),
                                                          ": " + msg if msg else ""))


def _stream_handle(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _ptr(t):
    if t.dtype.__str__() != "torch.float64" or not t.is_contiguous() or not t.is_cuda:
        raise ValueError("expected a contiguous float64 CUDA tensor")
    return ctypes.c_void_p(t.data_ptr())


def make_desc(nx, ny, nz, dx, dy, zf=None, dz=None, bcx=PERIODIC, bcy=PERIODIC, rho_l=1.0,
              rho_g=1e-3, dt=1e-4, precision=FP64, tol=0.0, max_refine=0, flags=0, div_tol=0.0,
              periodic_z=False):
    d = _abi.Desc()
    d.nx, d.ny, d.nz = int(nx), int(ny), int(nz)
    d.dx, d.dy = float(dx), float(dy)
    keep = None
    if zf is not None:
        keep = np.ascontiguousarray(zf, dtype=np.float64)
        d.zf = keep.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        d.dz = 0.0
    else:
        d.dz = float(dz)
    d.bc_x, d.bc_y = int(bcx), int(bcy)
    d.rho_l, d.rho_g, d.dt = float(rho_l), float(rho_g), float(dt)
    d.precision, d.tol, d.max_refine, d.flags = int(precision), float(tol), int(max_refine), int(flags)
    d.div_tol = float(div_tol)
    d.periodic_z = 1 if periodic_z else 0
    return d, keep


def workspace_bytes(**kw) -> int:
    d, _keep = make_desc(**kw)
    return int(_abi.lib().fizzy_proj_workspace_bytes(ctypes.byref(d)))


def _host_ptr(a):
    """Address of a host array (CPU tensor or numpy)."""
    if hasattr(a, "data_ptr"):
        return ctypes.c_void_p(a.data_ptr())
    return ctypes.c_void_p(a.ctypes.data)


class Plan:
    """A projection plan (fizzy_proj_plan / fizzy_proj_destroy)."""

    def __init__(self, nx, ny, nz, dx, dy, zf=None, dz=None, bcx=PERIODIC, bcy=PERIODIC,
                 rho_l=1.0, rho_g=1e-3, dt=1e-4, precision=FP64, tol=0.0, max_refine=0,
                 check=False, stream=None, div_tol=0.0, periodic_z=False, fused_xy=False):
        self.shape = (int(nz), int(ny), int(nx))
        self.precision = precision
        flags = (FLAG_CHECK if check else 0) | (FLAG_FUSED_XY if fused_xy else 0)
        d, keep = make_desc(nx, ny, nz, dx, dy, zf, dz, bcx, bcy, rho_l, rho_g, dt, precision,
                            tol, max_refine, flags, div_tol, periodic_z)
        h = ctypes.c_void_p()
        rc = _abi.lib().fizzy_proj_plan(ctypes.byref(h), ctypes.byref(d),
                                        ctypes.c_void_p(0) if stream is None else _stream_handle(stream))
        del keep
        if rc != 0:
            raise FizzyError(rc)
        self._h = h
        self.max_refine = int(max_refine) if max_refine > 0 else _abi.DEFAULT_MAX_REFINE

    @classmethod
    def for_case(cls, case, precision=FP64, check=False, **kw):
        s = case.spec
        return cls(s.nx, s.ny, s.nz, case.dx, case.dy, zf=case.zf, bcx=s.bcx, bcy=s.bcy,
                   rho_l=s.rho_l, rho_g=s.rho_g, dt=s.dt, precision=precision, check=check,
                   periodic_z=getattr(s, "bcz", NEUMANN) == PERIODIC, **kw)

    def _check(self, rc):
        if rc not in (0, -5):
            raise FizzyError(rc, _abi.lib().fizzy_proj_last_error(self._h).decode())
        return rc

    def solve(self, phi, pn, pnm1, u, v, w, p_out, stats=False, stream=None):
        """One projection on CUDA float64 tensors; u, v, w are overwritten with u.
        Returns a stats dict if stats=True (synchronises), else None (async)."""
        st = Stats() if stats else None
        rc = _abi.lib().fizzy_proj_solve(self._h, _ptr(phi), _ptr(pn), _ptr(pnm1), _ptr(u), _ptr(v),
                                         _ptr(w), _ptr(p_out), ctypes.byref(st) if st else None,
                                         _stream_handle(stream))
        self._check(rc)
        return st.as_dict() if st else None

    def solve_host(self, phi, pn, pnm1, u, v, w, p_out, stats=False, stream=None):
        """End-to-end solve on host arrays (numpy or CPU tensors, pinned preferred)."""
        hp = _host_ptr
        st = Stats() if stats else None
        rc = _abi.lib().fizzy_proj_solve_host(self._h, hp(phi), hp(pn), hp(pnm1), hp(u), hp(v),
                                              hp(w), hp(p_out), ctypes.byref(st) if st else None,
                                              _stream_handle(stream))
        self._check(rc)
        return st.as_dict() if st else None

    def solve_host_async(self, phi, pn, pnm1, u_in, v_in, w_in, u, v, w, p_out, stream=None):
        """Queue a pipelined end-to-end solve on pinned host arrays (u_in, v_in,
        w_in hold u*; u, v, w, p_out receive the results); the arrays must stay
        alive and untouched until host_wait()."""
        hp = _host_ptr
        self._check(_abi.lib().fizzy_proj_solve_host_async(
            self._h, hp(phi), hp(pn), hp(pnm1), hp(u_in), hp(v_in), hp(w_in), hp(u), hp(v), hp(w),
            hp(p_out), _stream_handle(stream)))

    def host_wait(self):
        """Block until every queued host solve's results are in host memory."""
        self._check(_abi.lib().fizzy_proj_host_wait(self._h))

    def poisson(self, f, p_out, stats=False, stream=None):
        """The plan's fast direct Poisson solve L_h p = f (fizzy_poisson_solve)
        on CUDA float64 tensors, with any x/y boundary kind the plan holds.
        Returns a stats dict if stats=True (synchronises), else None."""
        st = Stats() if stats else None
        rc = _abi.lib().fizzy_poisson_solve(self._h, _ptr(f), _ptr(p_out),
                                            ctypes.byref(st) if st else None, _stream_handle(stream))
        self._check(rc)
        return st.as_dict() if st else None

    def solve_vc(self, phi, u, v, w, p_out, max_iter=500, tol=0.0, stream=None):
        """Variable-coefficient projection WITHOUT the splitting
        (fizzy_proj_solve_vc): D(beta_f G p) = D(u*)/dt by conjugate gradients
        preconditioned with this plan's constant-coefficient solve; u, v, w
        are overwritten with u.  A mixed plan preconditions with its FP32
        solve (flexible CG); an FP64 plan with its FP64 solve.  Returns the
        stats dict (iterations = CG iterations); raises unless converged."""
        st = Stats()
        rc = _abi.lib().fizzy_proj_solve_vc(self._h, _ptr(phi), _ptr(u), _ptr(v), _ptr(w), _ptr(p_out),
                                            int(max_iter), float(tol), ctypes.byref(st),
                                            _stream_handle(stream))
        if rc != 0:
            raise FizzyError(rc, _abi.lib().fizzy_proj_last_error(self._h).decode())
        return st.as_dict()

    def acdi_step(self, phi, u, v, w, eps, gamma, dt=0.0, rhs_out=None, phi_out=None, stream=None):
        """One explicit stage of the ACDI phase-field transport
        (fizzy_acdi_step) on this plan's grid: rhs_out = d phi/dt,
        phi_out = phi + dt rhs (either may be None; phi_out may be phi)."""
        nul = ctypes.c_void_p(0)
        rc = _abi.lib().fizzy_acdi_step(self._h, _ptr(phi), _ptr(u), _ptr(v), _ptr(w), float(eps),
                                        float(gamma), float(dt),
                                        nul if rhs_out is None else _ptr(rhs_out),
                                        nul if phi_out is None else _ptr(phi_out), _stream_handle(stream))
        if rc != 0:
            raise FizzyError(rc, _abi.lib().fizzy_proj_last_error(self._h).decode())

    def stats(self, stream=None):
        st = Stats()
        self._check(_abi.lib().fizzy_proj_get_stats(self._h, ctypes.byref(st), _stream_handle(stream)))
        return st.as_dict()

    def set_timing(self, enable: bool, only: str | None = None):
        """Per-kernel CUDA-event timing: all kernels, or only the kernel slot
        named `only` (two events per launch of that kernel)."""
        mode = 0
        if enable:
            mode = 1 if only is None else 2 + self.slot_names().index(only)
        self._check(_abi.lib().fizzy_proj_set_timing(self._h, mode))

    def slot_names(self):
        L = _abi.lib()
        n = L.fizzy_proj_timing(self._h, -1, None, None, None)
        self._check(min(n, 0))
        names = []
        for idx in range(n):
            name = ctypes.c_char_p()
            L.fizzy_proj_timing(self._h, idx, ctypes.byref(name), None, None)
            names.append(name.value.decode())
        return names

    def timing(self):
        """{kernel name: (total ms, launches)} accumulated since set_timing(True)."""
        L = _abi.lib()
        out = {}
        n = L.fizzy_proj_timing(self._h, -1, None, None, None)
        self._check(min(n, 0))
        for idx in range(n):
            name, ms, cnt = ctypes.c_char_p(), ctypes.c_double(), ctypes.c_int()
            L.fizzy_proj_timing(self._h, idx, ctypes.byref(name), ctypes.byref(ms), ctypes.byref(cnt))
            if cnt.value:
                out[name.value.decode()] = (ms.value, cnt.value)
        return out

    def set_physics(self, rho_l, rho_g, dt, stream=None):
        self._check(_abi.lib().fizzy_proj_set_physics(self._h, float(rho_l), float(rho_g), float(dt),
                                                      _stream_handle(stream)))

    def launches_per_solve(self) -> int:
        return int(_abi.lib().fizzy_proj_launches_per_solve(self._h))

    def close(self):
        if getattr(self, "_h", None):
            _abi.lib().fizzy_proj_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class Batch:
    """Uneven-size projections in one persistent launch under a CUDA graph
    (fizzy_proj_batch_*).  plans: list of Plan; arrays: per instance the 7
    float64 CUDA tensors (phi, p_n, p_nm1, u, v, w, p_out), fixed for the
    batch's lifetime."""

    def __init__(self, plans, arrays, tuning=None, stream=None):
        n = len(plans)
        self._plans = list(plans)
        self._arrays = [t for inst in arrays for t in inst]  # keep tensors alive
        if len(self._arrays) != 7 * n:
            raise ValueError("need 7 arrays per instance")
        hp = (ctypes.c_void_p * n)(*[p._h.value for p in plans])
        ha = (ctypes.c_void_p * (7 * n))(*[_ptr(t).value for t in self._arrays])
        tun = None
        if tuning is not None:
            tun = _abi.Tuning(**tuning)
        h = ctypes.c_void_p()
        rc = _abi.lib().fizzy_proj_batch_create(ctypes.byref(h), n, hp, ha,
                                                ctypes.byref(tun) if tun else None,
                                                _stream_handle(stream))
        if rc != 0:
            raise FizzyError(rc)
        self._h = h

    def solve(self, stream=None):
        rc = _abi.lib().fizzy_proj_batch_solve(self._h, _stream_handle(stream))
        if rc != 0:
            raise FizzyError(rc)

    def status(self, stream=None) -> int:
        return int(_abi.lib().fizzy_proj_batch_status(self._h, _stream_handle(stream)))

    def autotune(self, reps=3, stream=None):
        t = _abi.Tuning()
        ms = ctypes.c_double()
        rc = _abi.lib().fizzy_proj_batch_autotune(self._h, int(reps), ctypes.byref(t),
                                                  ctypes.byref(ms), _stream_handle(stream))
        if rc != 0:
            raise FizzyError(rc)
        return t.as_dict(), ms.value

    def inject_stall(self, inst=-1, spin_limit=0):
        """Test support (fizzy_proj_batch_inject_stall): instance inst's first
        dependency wait never completes and every wait gives up after
        spin_limit polls; inject_stall() restores the defaults."""
        rc = _abi.lib().fizzy_proj_batch_inject_stall(self._h, int(inst), int(spin_limit))
        if rc != 0:
            raise FizzyError(rc)

    def info(self):
        n, g, sm = ctypes.c_int(), ctypes.c_int(), ctypes.c_size_t()
        _abi.lib().fizzy_proj_batch_info(self._h, ctypes.byref(n), ctypes.byref(g), ctypes.byref(sm))
        return {"items": n.value, "grid": g.value, "smem": sm.value}

    def close(self):
        if getattr(self, "_h", None):
            _abi.lib().fizzy_proj_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class _DevArray:
    """__cuda_array_interface__ over a raw device pointer (no ownership)."""

    def __init__(self, ptr, shape):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": "<f8",
                                         "data": (int(ptr), False), "version": 3, "strides": None}


def device_view(ptr, shape):
    """A float64 CUDA tensor viewing server-owned memory (valid until release)."""
    import torch
    return torch.as_tensor(_DevArray(ptr, shape), device="cuda")


class Server:
    """Serving runtime (fizzy_serve_*): request slots on their own streams, a
    device plan cache keyed by geometry, HBM-budget admission."""

    def __init__(self, hbm_budget_bytes, slots=8):
        h = ctypes.c_void_p()
        rc = _abi.lib().fizzy_serve_create(ctypes.byref(h), int(hbm_budget_bytes), int(slots))
        if rc != 0:
            raise FizzyError(rc)
        self._h = h
        self.slots = int(slots)

    def admit(self, **desc):
        """Returns (rc, slot, [7 device pointers]); rc 0 admitted, -7 busy, -3 over budget."""
        d, keep = make_desc(**desc)
        slot = ctypes.c_int(-1)
        ptrs = (ctypes.c_void_p * 7)()
        rc = _abi.lib().fizzy_serve_admit(self._h, ctypes.byref(d), ctypes.byref(slot), ptrs)
        del keep
        if rc not in (0, -3, -7):
            raise FizzyError(rc)
        return rc, slot.value, [ptrs[i] for i in range(7)]

    def stream(self, slot):
        """The slot's stream (a torch ExternalStream, made once per slot)."""
        cache = self.__dict__.setdefault("_streams", {})
        if slot not in cache:
            import torch
            st = ctypes.c_void_p()
            _abi.lib().fizzy_serve_stream(self._h, int(slot), ctypes.byref(st))
            cache[slot] = torch.cuda.ExternalStream(st.value)
        return cache[slot]

    def launch(self, slot):
        rc = _abi.lib().fizzy_serve_launch(self._h, int(slot))
        if rc != 0:
            raise FizzyError(rc)

    def poll(self):
        buf = (ctypes.c_int * self.slots)()
        n = _abi.lib().fizzy_serve_poll(self._h, buf, self.slots)
        if n < 0:
            raise FizzyError(n)
        return [buf[i] for i in range(n)]

    def stats(self, slot):
        st = Stats()
        rc = _abi.lib().fizzy_serve_stats(self._h, int(slot), ctypes.byref(st))
        if rc not in (0, -5):
            raise FizzyError(rc)
        return st.as_dict()

    def release(self, slot):
        rc = _abi.lib().fizzy_serve_release(self._h, int(slot))
        if rc != 0:
            raise FizzyError(rc)

    def info(self):
        used, cached, built, busy = ctypes.c_size_t(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _abi.lib().fizzy_serve_info(self._h, ctypes.byref(used), ctypes.byref(cached),
                                    ctypes.byref(built), ctypes.byref(busy))
        return {"bytes_used": used.value, "plans_cached": cached.value, "plans_built": built.value,
                "slots_busy": busy.value}

    def close(self):
        if getattr(self, "_h", None):
            _abi.lib().fizzy_serve_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def crop_fill(src, dst, offset, bcx=PERIODIC, bcy=PERIODIC, stream=None):
    """fizzy_crop_fill: dst[f] (six float64 CUDA tensors, shape (nz, ny, nx))
    = periodic crop of src[f] (shape (tz, ty, tx)) from offset (oz, oy, ox),
    with the wall faces of u, v and w zeroed; asynchronous on `stream`."""
    if len(src) != 6 or len(dst) != 6:
        raise ValueError("expected six source and six destination fields")
    tz, ty, tx = src[0].shape
    nz, ny, nx = dst[0].shape
    if any(t.shape != (tz, ty, tx) for t in src) or any(t.shape != (nz, ny, nx) for t in dst):
        raise ValueError("fields of one side must share a shape")
    crop_fill_ptrs([_ptr(t).value for t in src], (tz, ty, tx), [_ptr(t).value for t in dst],
                   (nz, ny, nx), offset, bcx, bcy, stream)


def crop_fill_ptrs(src, src_shape, dst, dst_shape, offset, bcx=PERIODIC, bcy=PERIODIC, stream=None):
    """crop_fill on raw device pointers: six float64 sources of shape
    src_shape = (tz, ty, tx) and six destinations of shape (nz, ny, nx)."""
    tz, ty, tx = (int(v) for v in src_shape)
    nz, ny, nx = (int(v) for v in dst_shape)
    sp = (ctypes.c_void_p * 6)(*src[:6])
    dp = (ctypes.c_void_p * 6)(*dst[:6])
    oz, oy, ox = (int(o) for o in offset)
    rc = _abi.lib().fizzy_crop_fill(sp, tx, ty, tz, dp, nx, ny, nz, ox, oy, oz, int(bcx), int(bcy),
                                    _stream_handle(stream))
    if rc != 0:
        raise FizzyError(rc)


def solve_noalloc(phi, pn, pnm1, u, v, w, p_out, stream=None, **desc):
    """Allocation-free FP64 projection for small grids (fizzy_proj_solve_noalloc).

    For callers that may not allocate device memory: it needs no plan and
    works in a static scratch array inside the library (at most
    NOALLOC_MAX_CELLS = 262144 cells; nx, ny <= 512).  Calls that overlap on
    the GPU share that scratch and race; serialise them.  desc takes the
    keyword arguments of make_desc (precision FP64, no flags)."""
    d, keep = make_desc(**desc)
    rc = _abi.lib().fizzy_proj_solve_noalloc(ctypes.byref(d), _ptr(phi), _ptr(pn), _ptr(pnm1),
                                             _ptr(u), _ptr(v), _ptr(w), _ptr(p_out),
                                             _stream_handle(stream))
    del keep
    if rc != 0:
        raise FizzyError(rc)


def probe_fma_rate(precision=FP64, iters=20000, op=0, chains=8, stream=None):
    """Arithmetic issue rate of the GPU (fizzy_probe_fma_rate): precision FP64
    times FP64 chains, MIXED FP32 chains; op 0 multiply-adds, 1 adds,
    2 multiplies, 3 multiply-adds and adds in turn; chains independent chains
    per thread (4, 8 or 16).  Returns (instructions per second, kernel
    milliseconds)."""
    rate, ms = ctypes.c_double(), ctypes.c_double()
    rc = _abi.lib().fizzy_probe_fma_rate(int(precision), int(op), int(chains), int(iters),
                                         ctypes.byref(rate), ctypes.byref(ms), _stream_handle(stream))
    if rc != 0:
        raise FizzyError(rc)
    return rate.value, ms.value
