"""Seeded synthetic inputs for the pressure-correction projection.

This module only *builds input fields*: grids, phase-field bubbles, predicted
velocities and old pressures. It holds none of the projection's arithmetic
(no density map, no right-hand side, no Poisson solve, no correction), so both
the CPU oracle tests and the CUDA path can be fed from it.

The paper's own workloads (the emulsion in forced isotropic turbulence and the
rising bubble of the "Examples" section, and the CI validation cases of the
"Statement of need" section) come with no data; these generators stand in for
them with bubble-laden fields of the same kind.

Layout: every array is float64 C-order ``[nz][ny][nx]`` (x fastest).
Staggered faces: ``u[k][j][i]`` sits on the x-face i+1/2, ``v`` on the y-face
j+1/2, ``w`` on the z-face k+1/2.  In a wall-bounded (Neumann) direction the
last face is the far wall and is exactly 0; the near wall face is implicit.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional

import numpy as np

PERIODIC = 0
NEUMANN = 1

# random streams (one numpy SeedSequence per (config, instance, stream))
S_VEL, S_PN, S_PNM1, S_BUBBLES, S_SIZES, S_ARRIVALS, S_NOISE = range(7)


def rng_for(config: int, instance: int, stream: int) -> np.random.Generator:
    return np.random.default_rng([int(config), int(instance), int(stream)])


@dataclasses.dataclass
class CaseSpec:
    """Recipe of one synthetic projection problem."""
    nx: int
    ny: int
    nz: int
    bcx: int = PERIODIC
    bcy: int = PERIODIC
    lx: float = 1.0           # domain lengths
    ly: float = 1.0
    lz: float = 1.0
    beta: float = 0.0         # tanh stretching of z (0 = uniform)
    n_bubbles: int = 1
    radius_cells: float = 8.0  # bubble radius in units of dx (ignored if radius is set)
    radius: Optional[float] = None
    centred: bool = False      # a single bubble at the domain centre
    rho_l: float = 1.0
    rho_g: float = 1e-3
    dt: float = 1e-4
    velocity: str = "solenoidal"   # "solenoidal" | "iid"
    noise: float = 0.01
    config: int = 0            # seed namespace
    instance: int = 0
    bcz: int = NEUMANN         # z: walls (default) or periodic (triperiodic boxes)


@dataclasses.dataclass
class Case:
    spec: CaseSpec
    dx: float
    dy: float
    zf: np.ndarray            # nz+1 face coordinates
    phi: np.ndarray
    pn: np.ndarray
    pnm1: np.ndarray
    u: np.ndarray
    v: np.ndarray
    w: np.ndarray

    @property
    def shape(self):
        return (self.spec.nz, self.spec.ny, self.spec.nx)

    @property
    def npts(self) -> int:
        return self.spec.nx * self.spec.ny * self.spec.nz


def z_faces(nz: int, lz: float = 1.0, beta: float = 0.0) -> np.ndarray:
    """Face coordinates of a z grid clustered at both walls by a tanh map.

    zf[k] = lz * (1/2 + tanh(beta (k/nz - 1/2)) / (2 tanh(beta/2))); beta = 0
    gives the uniform grid.  The end points are set exactly.
    """
    k = np.arange(nz + 1, dtype=np.float64)
    if beta == 0.0:
        zf = lz * k / nz
    else:
        zf = lz * (0.5 + np.tanh(beta * (k / nz - 0.5)) / (2.0 * np.tanh(beta / 2.0)))
    zf[0] = 0.0
    zf[-1] = lz
    return zf


def _centres_1d(n: int, length: float) -> np.ndarray:
    return (np.arange(n, dtype=np.float64) + 0.5) * (length / n)


def _place_bubbles(spec: CaseSpec, R: float, eps: float, rng) -> np.ndarray:
    """Rejection-sample non-overlapping bubble centres."""
    if spec.centred:
        return np.array([[spec.lx / 2, spec.ly / 2, spec.lz / 2]])
    lo = np.array([0.0, 0.0, 0.0])
    hi = np.array([spec.lx, spec.ly, spec.lz])
    margin = R + 2 * eps
    # keep away from walls
    walls = [spec.bcx == NEUMANN, spec.bcy == NEUMANN, spec.bcz == NEUMANN]
    for d in range(3):
        if walls[d]:
            lo[d] += margin
            hi[d] -= margin
        if hi[d] <= lo[d]:                    # too small: pin to the middle
            lo[d] = hi[d] = 0.5 * (lo[d] + hi[d])
    per = np.array([spec.lx if spec.bcx == PERIODIC else 0.0,
                    spec.ly if spec.bcy == PERIODIC else 0.0,
                    spec.lz if spec.bcz == PERIODIC else 0.0])
    dmin = 2 * R + 4 * eps
    centres = []
    tries = 0
    while len(centres) < spec.n_bubbles:
        tries += 1
        if tries > 20000:                     # crowded: keep those placed
            break
        c = lo + rng.random(3) * (hi - lo)
        ok = True
        for o in centres:
            d = c - o
            for a in range(3):
                if per[a] > 0:
                    d[a] -= per[a] * np.round(d[a] / per[a])
            if np.sqrt(np.sum(d * d)) < dmin:
                ok = False
                break
        if ok:
            centres.append(c)
    return np.array(centres)


def phase_field(spec: CaseSpec, dx: float, dy: float, zf: np.ndarray, rng) -> np.ndarray:
    """phi = max over bubbles of 1/2 (1 + tanh((R - r) / (2 eps))), eps = dx.

    r is the minimum-image distance in periodic directions.  phi = 1 inside
    each sphere (the phase whose density is rho_l).
    """
    eps = dx
    R = spec.radius if spec.radius is not None else spec.radius_cells * dx
    centres = _place_bubbles(spec, R, eps, rng)
    xc = _centres_1d(spec.nx, spec.lx)
    yc = _centres_1d(spec.ny, spec.ly)
    zc = 0.5 * (zf[:-1] + zf[1:])
    phi = np.zeros((spec.nz, spec.ny, spec.nx))
    for c in centres:
        ddx = xc - c[0]
        ddy = yc - c[1]
        if spec.bcx == PERIODIC:
            ddx -= spec.lx * np.round(ddx / spec.lx)
        if spec.bcy == PERIODIC:
            ddy -= spec.ly * np.round(ddy / spec.ly)
        ddz = zc - c[2]
        if spec.bcz == PERIODIC:
            ddz -= spec.lz * np.round(ddz / spec.lz)
        # only the box around the bubble matters (tanh saturates beyond ~20 eps)
        reach = R + 20 * eps
        ix = np.nonzero(np.abs(ddx) < reach)[0]
        iy = np.nonzero(np.abs(ddy) < reach)[0]
        iz = np.nonzero(np.abs(ddz) < reach)[0]
        if len(ix) == 0 or len(iy) == 0 or len(iz) == 0:
            continue
        r = np.sqrt(ddz[iz][:, None, None] ** 2 + ddy[iy][None, :, None] ** 2
                    + ddx[ix][None, None, :] ** 2)
        val = 0.5 * (1.0 + np.tanh((R - r) / (2.0 * eps)))
        sub = phi[np.ix_(iz, iy, ix)]
        phi[np.ix_(iz, iy, ix)] = np.maximum(sub, val)
    return phi


def pressure_modes(spec: CaseSpec, zf: np.ndarray, rng, n_modes: int = 8) -> np.ndarray:
    """Sum of 8 seeded Fourier modes of amplitude 1:
    sum_m cos(2 pi (a_m x/lx + b_m y/ly) + theta_m) cos(pi c_m z / lz),
    a_m, b_m, c_m integers in [0, 4], theta_m uniform in [0, 2 pi); with
    periodic z the z factor is cos(2 pi c_m z / lz)."""
    zk = 2.0 if spec.bcz == PERIODIC else 1.0
    xc = _centres_1d(spec.nx, spec.lx) / spec.lx
    yc = _centres_1d(spec.ny, spec.ly) / spec.ly
    zc = 0.5 * (zf[:-1] + zf[1:]) / spec.lz
    zs = np.empty((spec.nz, n_modes))
    xys = np.empty((n_modes, spec.ny * spec.nx))
    for m in range(n_modes):
        a, b, c = rng.integers(0, 5, size=3)
        th = rng.random() * 2 * np.pi
        xys[m] = np.cos(2 * np.pi * (a * xc[None, :] + b * yc[:, None]) + th).ravel()
        zs[:, m] = np.cos(zk * np.pi * c * zc)
    return (zs @ xys).reshape(spec.nz, spec.ny, spec.nx)  # sum over the modes


def _random_periodic_field(shape, rng, slope: float = -17.0 / 6.0) -> np.ndarray:
    """Real periodic random field on an index grid with random phases and
    amplitude |k|^slope for 0 < |k| <= n/3 (index wavenumbers)."""
    nz, ny, nx = shape
    kz = np.fft.fftfreq(nz) * nz
    ky = np.fft.fftfreq(ny) * ny
    kx = np.fft.rfftfreq(nx) * nx
    kmax = min(nx, ny, nz) / 3.0
    import os
    import scipy.fft as sfft
    # build in chunks of kz planes (the phases are drawn in plane order)
    spec = np.zeros((nz, ny, kx.size), dtype=np.complex128)
    k2xy = ky[:, None] ** 2 + kx[None, :] ** 2
    step = max(1, (1 << 22) // max(1, k2xy.size))
    for a0 in range(0, nz, step):
        a1 = min(nz, a0 + step)
        kk = np.sqrt(kz[a0:a1, None, None] ** 2 + k2xy[None])
        amp = np.where((kk > 0) & (kk <= kmax), np.power(np.maximum(kk, 1e-30), slope), 0.0)
        ph = rng.random(kk.shape) * 2 * np.pi
        spec[a0:a1].real = amp * np.cos(ph)
        spec[a0:a1].imag = amp * np.sin(ph)
    return sfft.irfftn(spec, s=shape, axes=(0, 1, 2), workers=os.cpu_count() or 1)


def solenoidal_velocity(spec: CaseSpec, dx: float, dy: float, zf: np.ndarray, rng):
    """Discrete curl of an edge-centred random vector potential.

    A_x lives on x-edges (i, j+1/2, k+1/2), A_y on y-edges (i+1/2, j, k+1/2),
    A_z on z-edges (i+1/2, j+1/2, k); the staggered curl of such a potential
    has zero discrete divergence.  Envelopes sin(pi s / L) make the potential
    vanish on wall edges so the normal velocity is exactly 0 on every wall
    (none along a periodic direction).
    """
    nz, ny, nx = spec.nz, spec.ny, spec.nx
    shape = (nz, ny, nx)
    Ax = _random_periodic_field(shape, rng)
    Ay = _random_periodic_field(shape, rng)
    Az = _random_periodic_field(shape, rng)
    zfe = zf[1:]                              # z of edge k+1/2
    pz = spec.bcz == PERIODIC
    if not pz:                                # A_x, A_y vanish on z walls
        envz = np.sin(np.pi * zfe / spec.lz)
        envz[-1] = 0.0
        Ax *= envz[:, None, None]
        Ay *= envz[:, None, None]
    if spec.bcx == NEUMANN:                   # A_y, A_z vanish on x walls
        xe = (np.arange(nx) + 1.0) / nx
        envx = np.sin(np.pi * xe)
        envx[-1] = 0.0
        Ay *= envx[None, None, :]
        Az *= envx[None, None, :]
    if spec.bcy == NEUMANN:                   # A_x, A_z vanish on y walls
        ye = (np.arange(ny) + 1.0) / ny
        envy = np.sin(np.pi * ye)
        envy[-1] = 0.0
        Ax *= envy[None, :, None]
        Az *= envy[None, :, None]
    dzf = np.diff(zf)

    def shm(a, axis, periodic):
        """value at index-1 along axis (wrap if periodic, else 0 at the first)."""
        if periodic:
            return np.roll(a, 1, axis=axis)
        out = np.zeros_like(a)
        sl = [slice(None)] * 3
        sl2 = [slice(None)] * 3
        sl[axis] = slice(1, None)
        sl2[axis] = slice(0, -1)
        out[tuple(sl)] = a[tuple(sl2)]
        return out

    px = spec.bcx == PERIODIC
    py = spec.bcy == PERIODIC
    # u(i+1/2, j, k) = dAz/dy - dAy/dz
    u = (Az - shm(Az, 1, py)) / dy - (Ay - shm(Ay, 0, pz)) / dzf[:, None, None]
    # v(i, j+1/2, k) = dAx/dz - dAz/dx
    v = (Ax - shm(Ax, 0, pz)) / dzf[:, None, None] - (Az - shm(Az, 2, px)) / dx
    # w(i, j, k+1/2) = dAy/dx - dAx/dy
    w = (Ay - shm(Ay, 2, px)) / dx - (Ax - shm(Ax, 1, py)) / dy
    return u, v, w


def zero_walls(spec: CaseSpec, u, v, w):
    if spec.bcx == NEUMANN:
        u[:, :, -1] = 0.0
    if spec.bcy == NEUMANN:
        v[:, -1, :] = 0.0
    if spec.bcz == NEUMANN:
        w[-1, :, :] = 0.0


def make_case(spec: CaseSpec) -> Case:
    dx = spec.lx / spec.nx
    dy = spec.ly / spec.ny
    zf = z_faces(spec.nz, spec.lz, spec.beta)
    phi = phase_field(spec, dx, dy, zf, rng_for(spec.config, spec.instance, S_BUBBLES))
    pn = pressure_modes(spec, zf, rng_for(spec.config, spec.instance, S_PN))
    pnm1 = pressure_modes(spec, zf, rng_for(spec.config, spec.instance, S_PNM1))
    rv = rng_for(spec.config, spec.instance, S_VEL)
    shape = (spec.nz, spec.ny, spec.nx)
    if spec.velocity == "iid":
        u = rv.uniform(-1.0, 1.0, shape)
        v = rv.uniform(-1.0, 1.0, shape)
        w = rv.uniform(-1.0, 1.0, shape)
    else:
        u, v, w = solenoidal_velocity(spec, dx, dy, zf, rv)
        zero_walls(spec, u, v, w)
        rms = math.sqrt((np.sum(u * u) + np.sum(v * v) + np.sum(w * w)) / (3 * u.size))
        if rms > 0:
            u /= rms
            v /= rms
            w /= rms
        if spec.noise > 0:
            rn = rng_for(spec.config, spec.instance, S_NOISE)
            u += rn.uniform(-spec.noise, spec.noise, shape)
            v += rn.uniform(-spec.noise, spec.noise, shape)
            w += rn.uniform(-spec.noise, spec.noise, shape)
    zero_walls(spec, u, v, w)
    return Case(spec=spec, dx=dx, dy=dy, zf=zf, phi=phi, pn=pn, pnm1=pnm1, u=u, v=v, w=w)


# ---------------------------------------------------------------------------
# Workload recipes
# ---------------------------------------------------------------------------

def drop32_spec() -> CaseSpec:
    """32^3 unit box, periodic x/y, walls in z, one drop of radius 0.25 at the
    centre, rho_l = 1, rho_g = 1e-3, i.i.d. uniform[-1, 1] face velocities,
    dt = 1e-3."""
    return CaseSpec(nx=32, ny=32, nz=32, n_bubbles=1, radius=0.25, centred=True,
                    rho_l=1.0, rho_g=1e-3, dt=1e-3, velocity="iid", noise=0.0,
                    config=0)


def bubbles_spec(n: int = 256, n_bubbles: int = 40, radius_cells: float = 8.0,
                 beta: float = 0.0, config: int = 1) -> CaseSpec:
    """n^3 unit box, periodic x/y, walls in z, n_bubbles drops of the given
    radius (cells), density ratio 1000, k^-5/3 solenoidal u* of rms 1 plus
    uniform[-0.01, 0.01] noise, dt = 1e-4."""
    return CaseSpec(nx=n, ny=n, nz=n, n_bubbles=n_bubbles, radius_cells=radius_cells,
                    beta=beta, rho_l=1.0, rho_g=1e-3, dt=1e-4, velocity="solenoidal",
                    noise=0.01, config=config)


def bubbles256_spec() -> CaseSpec:
    return bubbles_spec(256, 40, 8.0, 0.0, config=1)


def bubbles512_stretched_spec() -> CaseSpec:
    return bubbles_spec(512, 400, 6.0, 1.5, config=2)


def bubbles384_stretched_spec() -> CaseSpec:
    """The 512^3 stretched recipe at 384^3 (a length of the register-resident
    passes that is not a power of two: 384 = 2 x 24 x 8); 170 drops keep the
    gas fraction of the 512^3 case."""
    return bubbles_spec(384, 170, 6.0, 1.5, config=70)


def emulsion_spec(n: int = 256, n_drops: int = 400, radius_cells: float = 8.0,
                  config: int = 5) -> CaseSpec:
    """n^3 unit triperiodic box (periodic x, y and z), standing in for the
    paper's liquid-liquid emulsion in forced homogeneous isotropic turbulence
    (its weak-scaling case): n_drops drops of the given radius (cells; 400 of
    radius 8 fill about 5 % of 256^3), drops of density 0.8 in a carrier of
    density 1 (an oil-in-water-like ratio; rho0 is then the drop density), a
    k^-5/3 solenoidal u* of rms 1 with no wall envelope plus
    uniform[-0.01, 0.01] noise, dt = 1e-4."""
    return CaseSpec(nx=n, ny=n, nz=n, n_bubbles=n_drops, radius_cells=radius_cells,
                    rho_l=0.8, rho_g=1.0, dt=1e-4, velocity="solenoidal", noise=0.01,
                    config=config, bcz=PERIODIC)


def emulsion256_spec() -> CaseSpec:
    return emulsion_spec(256, 400, 8.0, config=5)


BATCH_XY = (32, 48, 64, 96, 128, 192)
SERVE_XY = (64, 96, 128, 192, 256, 384)


def batch_specs(n_instances: int = 64, config: int = 3) -> list:
    """Uneven batch: nx, ny drawn from {32,...,192}, nz uniform in [32, 192],
    periodic or Neumann x/y, 1-20 drops of radius 4-10 cells, density ratio
    uniform in [10, 1000].  Cubic cells of size 1/nx."""
    specs = []
    for inst in range(n_instances):
        r = rng_for(config, inst, S_SIZES)
        nx = int(r.choice(BATCH_XY))
        ny = int(r.choice(BATCH_XY))
        nz = int(r.integers(32, 193))
        bcx = int(r.integers(0, 2))
        bcy = int(r.integers(0, 2))
        nb = int(r.integers(1, 21))
        rad = float(r.uniform(4.0, 10.0))
        ratio = float(r.uniform(10.0, 1000.0))
        h = 1.0 / nx
        specs.append(CaseSpec(nx=nx, ny=ny, nz=nz, bcx=bcx, bcy=bcy, lx=1.0, ly=ny * h,
                              lz=nz * h, n_bubbles=nb, radius_cells=rad, rho_l=1.0,
                              rho_g=1.0 / ratio, dt=1e-4, velocity="solenoidal",
                              noise=0.01, config=config, instance=inst))
    return specs


def serve_specs(n_requests: int, config: int = 4):
    """Request stream: Poisson arrivals (mean 2000 req/s), nx, ny drawn from
    {64,...,384}, nz uniform in [64, 384], 30 % with tanh-stretched z
    (beta uniform in [1, 2]); fields as in the batch recipe.  Returns
    (arrival_times_s, specs)."""
    ra = rng_for(config, 0, S_ARRIVALS)
    gaps = ra.exponential(1.0 / 2000.0, size=n_requests)
    t = np.cumsum(gaps)
    specs = []
    for inst in range(n_requests):
        r = rng_for(config, inst, S_SIZES)
        nx = int(r.choice(SERVE_XY))
        ny = int(r.choice(SERVE_XY))
        nz = int(r.integers(64, 385))
        bcx = int(r.integers(0, 2))
        bcy = int(r.integers(0, 2))
        beta = float(r.uniform(1.0, 2.0)) if r.random() < 0.3 else 0.0
        nb = int(r.integers(1, 21))
        rad = float(r.uniform(4.0, 10.0))
        ratio = float(r.uniform(10.0, 1000.0))
        h = 1.0 / nx
        specs.append(CaseSpec(nx=nx, ny=ny, nz=nz, bcx=bcx, bcy=bcy, lx=1.0, ly=ny * h,
                              lz=nz * h, beta=beta, n_bubbles=nb, radius_cells=rad,
                              rho_l=1.0, rho_g=1.0 / ratio, dt=1e-4, velocity="solenoidal",
                              noise=0.01, config=config, instance=inst))
    return t, specs
