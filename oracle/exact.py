"""Exact rational-arithmetic projection on tiny grids (test infrastructure only).

A second, independent restatement of the discrete definitions of the
projection (paper, "Methods and Implementation strategy": staggered
second-order finite differences, pressure correction with the
constant-coefficient splitting; "Mathematical model": linear property map),
evaluated with ``fractions.Fraction`` so there is no rounding at all:

    rho = rho_g + phi (rho_l - rho_g) at centres; rho_f = mean of the two
    neighbours; beta_f = 1/rho_f; rho0 = min(rho_l, rho_g); phat = 2 p^n - p^(n-1);
    f = (rho0/dt) D u* + D[(1 - rho0 beta_f) G phat] minus its dzf-weighted mean;
    D G p = f with sum dzf p = 0 (exact Gaussian elimination, gauge row last);
    u = u* - dt [G p / rho0 + (beta_f - 1/rho0) G phat] on non-wall faces.

Only used to write and check the fixtures under tests/golden/.
"""
from __future__ import annotations

from fractions import Fraction as Q


class ExactGrid:
    def __init__(self, nx, ny, nz, dx, dy, zf, bcx, bcy, bcz=1):
        self.nx, self.ny, self.nz = nx, ny, nz
        self.dx, self.dy = Q(dx), Q(dy)
        self.zf = [Q(z) for z in zf]
        self.bcx, self.bcy, self.bcz = bcx, bcy, bcz

    def dzf(self, k):
        return self.zf[k + 1] - self.zf[k]

    def zc(self, k):
        return (self.zf[k] + self.zf[k + 1]) / 2

    def dzc(self, k):  # spacing at z-face k+1/2 (k = nz-1: across the periodic boundary)
        if k == self.nz - 1:
            return (self.dzf(0) + self.dzf(self.nz - 1)) / 2
        return self.zc(k + 1) - self.zc(k)

    def cells(self):
        for k in range(self.nz):
            for j in range(self.ny):
                for i in range(self.nx):
                    yield i, j, k

    def idx(self, i, j, k):
        return (k * self.ny + j) * self.nx + i


def _grad(g, q):
    gx, gy, gz = {}, {}, {}
    for i, j, k in g.cells():
        c = q[(i, j, k)]
        if i < g.nx - 1:
            gx[(i, j, k)] = (q[(i + 1, j, k)] - c) / g.dx
        else:
            gx[(i, j, k)] = (q[(0, j, k)] - c) / g.dx if g.bcx == 0 else Q(0)
        if j < g.ny - 1:
            gy[(i, j, k)] = (q[(i, j + 1, k)] - c) / g.dy
        else:
            gy[(i, j, k)] = (q[(i, 0, k)] - c) / g.dy if g.bcy == 0 else Q(0)
        if k < g.nz - 1:
            gz[(i, j, k)] = (q[(i, j, k + 1)] - c) / g.dzc(k)
        else:
            gz[(i, j, k)] = (q[(i, j, 0)] - c) / g.dzc(k) if g.bcz == 0 else Q(0)
    return gx, gy, gz


def _div(g, u, v, w):
    out = {}
    for i, j, k in g.cells():
        ue = Q(0) if (g.bcx == 1 and i == g.nx - 1) else u[(i, j, k)]
        if i > 0:
            uw = u[(i - 1, j, k)]
        else:
            uw = u[(g.nx - 1, j, k)] if g.bcx == 0 else Q(0)
        vn = Q(0) if (g.bcy == 1 and j == g.ny - 1) else v[(i, j, k)]
        if j > 0:
            vs = v[(i, j - 1, k)]
        else:
            vs = v[(i, g.ny - 1, k)] if g.bcy == 0 else Q(0)
        wt = Q(0) if (g.bcz == 1 and k == g.nz - 1) else w[(i, j, k)]
        if k > 0:
            wb = w[(i, j, k - 1)]
        else:
            wb = w[(i, j, g.nz - 1)] if g.bcz == 0 else Q(0)
        out[(i, j, k)] = (ue - uw) / g.dx + (vn - vs) / g.dy + (wt - wb) / g.dzf(k)
    return out


def _beta(g, rho_l, rho_g, phi):
    def rho(c):
        return rho_g + phi[c] * (rho_l - rho_g)
    bx, by, bz = {}, {}, {}
    for i, j, k in g.cells():
        c = (i, j, k)
        ie = i + 1 if i < g.nx - 1 else (0 if g.bcx == 0 else None)
        jn = j + 1 if j < g.ny - 1 else (0 if g.bcy == 0 else None)
        bx[c] = 1 / ((rho(c) + rho((ie, j, k))) / 2) if ie is not None else Q(0)
        by[c] = 1 / ((rho(c) + rho((i, jn, k))) / 2) if jn is not None else Q(0)
        kt = k + 1 if k < g.nz - 1 else (0 if g.bcz == 0 else None)
        bz[c] = 1 / ((rho(c) + rho((i, j, kt))) / 2) if kt is not None else Q(0)
    return bx, by, bz


def _wmean(g, a):
    num = sum(g.dzf(k) * a[(i, j, k)] for i, j, k in g.cells())
    den = sum(g.dzf(k) for _, _, k in g.cells())
    return num / den


def _solve(g, f):
    """Exact Gaussian elimination on D G p = f with the last row replaced by the
    gauge row sum dzf_k p = 0."""
    cells = list(g.cells())
    n = len(cells)
    cols = []
    for c in cells:  # assemble column by column: L applied to unit vectors
        e = {d: Q(0) for d in cells}
        e[c] = Q(1)
        gx, gy, gz = _grad(g, e)
        cols.append(_div(g, gx, gy, gz))
    A = [[cols[cidx][r] for cidx in range(n)] for r in cells]
    b = [f[r] for r in cells]
    A[n - 1] = [g.dzf(c[2]) for c in cells]
    b[n - 1] = Q(0)
    for k in range(n):
        piv = next(r for r in range(k, n) if A[r][k] != 0)
        A[k], A[piv] = A[piv], A[k]
        b[k], b[piv] = b[piv], b[k]
        for r in range(k + 1, n):
            if A[r][k] != 0:
                m = A[r][k] / A[k][k]
                A[r] = [A[r][c] - m * A[k][c] for c in range(n)]
                b[r] -= m * b[k]
    x = [Q(0)] * n
    for k in range(n - 1, -1, -1):
        s = b[k] - sum(A[k][c] * x[c] for c in range(k + 1, n))
        x[k] = s / A[k][k]
    return {cells[i]: x[i] for i in range(n)}


def project(g: ExactGrid, rho_l, rho_g, dt, phi, pn, pnm1, u, v, w):
    """All field arguments: dict (i, j, k) -> Fraction.  Returns (f, p, u, v, w)."""
    rho_l, rho_g, dt = Q(rho_l), Q(rho_g), Q(dt)
    rho0 = min(rho_l, rho_g)
    ph = {c: 2 * pn[c] - pnm1[c] for c in g.cells()}
    gx, gy, gz = _grad(g, ph)
    bx, by, bz = _beta(g, rho_l, rho_g, phi)
    fx = {c: (1 - rho0 * bx[c]) * gx[c] for c in g.cells()}
    fy = {c: (1 - rho0 * by[c]) * gy[c] for c in g.cells()}
    fz = {c: (1 - rho0 * bz[c]) * gz[c] for c in g.cells()}
    d1 = _div(g, u, v, w)
    d2 = _div(g, fx, fy, fz)
    f = {c: rho0 / dt * d1[c] + d2[c] for c in g.cells()}
    m = _wmean(g, f)
    f = {c: f[c] - m for c in g.cells()}
    p = _solve(g, f)
    px, py, pz = _grad(g, p)
    uo, vo, wo = dict(u), dict(v), dict(w)
    for c in g.cells():
        i, j, k = c
        if not (g.bcx == 1 and i == g.nx - 1):
            uo[c] = u[c] - dt * (px[c] / rho0 + (bx[c] - 1 / rho0) * gx[c])
        if not (g.bcy == 1 and j == g.ny - 1):
            vo[c] = v[c] - dt * (py[c] / rho0 + (by[c] - 1 / rho0) * gy[c])
        if not (g.bcz == 1 and k == g.nz - 1):
            wo[c] = w[c] - dt * (pz[c] / rho0 + (bz[c] - 1 / rho0) * gz[c])
    return f, p, uo, vo, wo


# ---------------------------------------------------------------------------
# The Poisson problem alone with the CaNS solver's boundary kinds in x and y:
# 0 periodic, 1 Neumann at both ends, 2 Dirichlet at both ends (p = 0 on the
# boundary faces), 3 Neumann near / Dirichlet far, 4 Dirichlet near /
# Neumann far.  Beyond a Neumann face the ghost value equals the cell value,
# beyond a Dirichlet face it is its negative.
# ---------------------------------------------------------------------------
def _ghost(bc, side, qc):
    dirichlet = bc == 2 or (bc == 3 and side == 1) or (bc == 4 and side == 0)
    return -qc if dirichlet else qc


def lap_bc(g: ExactGrid, q):
    """L_h q written out cell by cell: (neighbour - centre)/h on every face,
    ghost values beyond boundary faces, z faces as in the projection."""
    out = {}
    for i, j, k in g.cells():
        qc = q[(i, j, k)]
        if i < g.nx - 1:
            qe = q[(i + 1, j, k)]
        else:
            qe = q[(0, j, k)] if g.bcx == 0 else _ghost(g.bcx, 1, qc)
        if i > 0:
            qw = q[(i - 1, j, k)]
        else:
            qw = q[(g.nx - 1, j, k)] if g.bcx == 0 else _ghost(g.bcx, 0, qc)
        if j < g.ny - 1:
            qn = q[(i, j + 1, k)]
        else:
            qn = q[(i, 0, k)] if g.bcy == 0 else _ghost(g.bcy, 1, qc)
        if j > 0:
            qs = q[(i, j - 1, k)]
        else:
            qs = q[(i, g.ny - 1, k)] if g.bcy == 0 else _ghost(g.bcy, 0, qc)
        if k < g.nz - 1:
            wt = (q[(i, j, k + 1)] - qc) / g.dzc(k)
        else:
            wt = (q[(i, j, 0)] - qc) / g.dzc(k) if g.bcz == 0 else Q(0)
        if k > 0:
            wb = (qc - q[(i, j, k - 1)]) / g.dzc(k - 1)
        else:
            wb = (qc - q[(i, j, g.nz - 1)]) / g.dzc(g.nz - 1) if g.bcz == 0 else Q(0)
        out[(i, j, k)] = (((qe - qc) - (qc - qw)) / g.dx / g.dx + ((qn - qc) - (qc - qs)) / g.dy / g.dy
                          + (wt - wb) / g.dzf(k))
    return out


def poisson_bc(g: ExactGrid, f):
    """Exact solution of L_h p = f.  Singular (no Dirichlet face in x or y):
    the last equation is replaced by the gauge row sum dzf_k p = 0 and f is
    taken as given (the caller passes a compatible f).  Otherwise p is
    unique."""
    cells = list(g.cells())
    n = len(cells)
    cols = []
    for c in cells:
        e = {d: Q(0) for d in cells}
        e[c] = Q(1)
        cols.append(lap_bc(g, e))
    A = [[cols[ci][r] for ci in range(n)] for r in cells]
    b = [f[r] for r in cells]
    if g.bcx <= 1 and g.bcy <= 1:
        A[n - 1] = [g.dzf(c[2]) for c in cells]
        b[n - 1] = Q(0)
    for k in range(n):
        piv = next(r for r in range(k, n) if A[r][k] != 0)
        A[k], A[piv] = A[piv], A[k]
        b[k], b[piv] = b[piv], b[k]
        for r in range(k + 1, n):
            if A[r][k] != 0:
                m = A[r][k] / A[k][k]
                A[r] = [A[r][c] - m * A[k][c] for c in range(n)]
                b[r] -= m * b[k]
    x = [Q(0)] * n
    for k in range(n - 1, -1, -1):
        s = b[k] - sum(A[k][c] * x[c] for c in range(k + 1, n))
        x[k] = s / A[k][k]
    return {cells[i]: x[i] for i in range(n)}
