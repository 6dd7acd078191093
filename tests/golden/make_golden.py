"""Write the exact-arithmetic projection fixtures in this folder.

The paper prints no worked numerical example, so these fixtures are the
projection's discrete definitions evaluated in exact rational arithmetic
(oracle/exact.py) on tiny grids with dyadic inputs (exactly representable in
binary64).  Stored outputs are the exact rationals rounded once to binary64.
Calls only oracle/.  Run: python tests/golden/make_golden.py
"""
import json
import os
import sys
from fractions import Fraction as Q

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))
from oracle import exact  # noqa: E402

CITATION = ("Paper, 'Methods and Implementation strategy': staggered second-order finite "
            "differences, pressure correction split into a constant-coefficient Poisson "
            "equation (Dong & Shen 2012; Dodd & Ferrante 2014; Frantzis & Grigoriadis 2019); "
            "'Mathematical model': density mapped linearly over the phase field.  Values: exact "
            "rational evaluation of the discrete definitions (oracle/exact.py), rounded to binary64.")

CASES = [
    dict(name="p3x4x3_pp_uniform", nx=3, ny=4, nz=3, dx="1/4", dy="1/4",
         zf=["0", "1/4", "1/2", "3/4"], bcx=0, bcy=0, rho_l="1", rho_g="1/16", dt="1/32", seed=11),
    dict(name="p4x3x4_np_stretched", nx=4, ny=3, nz=4, dx="1/4", dy="1/2",
         zf=["0", "1/8", "1/2", "7/8", "1"], bcx=1, bcy=0, rho_l="1/8", rho_g="1", dt="1/16", seed=23),
    dict(name="p2x3x3_nn_stretched", nx=2, ny=3, nz=3, dx="1/2", dy="1/4",
         zf=["0", "1/4", "1/2", "1"], bcx=1, bcy=1, rho_l="1", rho_g="1/4", dt="1/8", seed=37),
    # periodic z (triperiodic boxes; bcz = 0)
    dict(name="p3x2x4_ppp_uniform", nx=3, ny=2, nz=4, dx="1/4", dy="1/2",
         zf=["0", "1/4", "1/2", "3/4", "1"], bcx=0, bcy=0, bcz=0, rho_l="1/8", rho_g="1",
         dt="1/16", seed=41),
    dict(name="p2x3x4_npp_stretched", nx=2, ny=3, nz=4, dx="1/2", dy="1/4",
         zf=["0", "1/8", "3/8", "1/2", "1"], bcx=1, bcy=0, bcz=0, rho_l="1", rho_g="1/4",
         dt="1/8", seed=53),
]


def lcg(seed):
    state = seed
    while True:
        state = (1103515245 * state + 12345) % (1 << 31)
        yield state


def make(case):
    nx, ny, nz = case["nx"], case["ny"], case["nz"]
    bcz = case.get("bcz", 1)
    g = exact.ExactGrid(nx, ny, nz, Q(case["dx"]), Q(case["dy"]), [Q(z) for z in case["zf"]],
                        case["bcx"], case["bcy"], bcz)
    r = lcg(case["seed"])
    cells = list(g.cells())
    phi = {c: Q(next(r) % 17, 16) for c in cells}
    pn = {c: Q(next(r) % 17 - 8, 8) for c in cells}
    pnm1 = {c: Q(next(r) % 17 - 8, 8) for c in cells}
    u = {c: Q(next(r) % 33 - 16, 16) for c in cells}
    v = {c: Q(next(r) % 33 - 16, 16) for c in cells}
    w = {c: Q(next(r) % 33 - 16, 16) for c in cells}
    for (i, j, k) in cells:
        if case["bcx"] == 1 and i == nx - 1:
            u[(i, j, k)] = Q(0)
        if case["bcy"] == 1 and j == ny - 1:
            v[(i, j, k)] = Q(0)
        if bcz == 1 and k == nz - 1:
            w[(i, j, k)] = Q(0)
    f, p, uo, vo, wo = exact.project(g, Q(case["rho_l"]), Q(case["rho_g"]), Q(case["dt"]), phi,
                                     pn, pnm1, u, v, w)

    def arr(d):
        return [float(d[c]) for c in cells]  # x fastest, [nz][ny][nx] order

    out = dict(case)
    out.update(citation=CITATION, layout="[nz][ny][nx], x fastest",
               inputs=dict(phi=arr(phi), pn=arr(pn), pnm1=arr(pnm1), u=arr(u), v=arr(v), w=arr(w)),
               expected=dict(f=arr(f), p=arr(p), u=arr(uo), v=arr(vo), w=arr(wo)))
    return out


# The Poisson problem alone with Dirichlet and mixed x/y boundaries (bc 2 DD,
# 3 Neumann near / Dirichlet far, 4 Dirichlet near / Neumann far): the
# boundary kinds of the CaNS fast solver the paper's "Methods and
# Implementation strategy" builds on.
CITATION_POISSON = ("Paper, 'Methods and Implementation strategy': staggered second-order finite "
                    "differences, fast direct FFT-based Poisson solver of CaNS (Costa 2018) with "
                    "Dirichlet and mixed boundary kinds.  Values: exact rational solution of the "
                    "discrete equations (oracle/exact.py, poisson_bc), rounded to binary64.")

POISSON_CASES = [
    dict(name="dd_p_uniform", nx=4, ny=3, nz=3, dx="1/4", dy="1/3", zf=["0", "1/3", "2/3", "1"],
         bcx=2, bcy=0, bcz=1, seed=61),
    dict(name="nd_dn_stretched", nx=3, ny=4, nz=4, dx="1/2", dy="1/4",
         zf=["0", "1/8", "1/2", "7/8", "1"], bcx=3, bcy=4, bcz=1, seed=67),
    dict(name="dn_n_periodic_z", nx=4, ny=2, nz=3, dx="1/4", dy="1/2", zf=["0", "1/4", "5/8", "1"],
         bcx=4, bcy=1, bcz=0, seed=71),
    dict(name="dd_dd_uniform", nx=3, ny=3, nz=2, dx="1/3", dy="1/3", zf=["0", "1/2", "1"],
         bcx=2, bcy=2, bcz=1, seed=73),
]


def make_poisson(case):
    nx, ny, nz = case["nx"], case["ny"], case["nz"]
    g = exact.ExactGrid(nx, ny, nz, Q(case["dx"]), Q(case["dy"]), [Q(z) for z in case["zf"]],
                        case["bcx"], case["bcy"], case["bcz"])
    r = lcg(case["seed"])
    cells = list(g.cells())
    f = {c: Q(next(r) % 65 - 32, 8) for c in cells}
    p = exact.poisson_bc(g, f)
    out = dict(case)
    out.update(citation=CITATION_POISSON, layout="[nz][ny][nx], x fastest",
               inputs=dict(f=[float(f[c]) for c in cells]),
               expected=dict(p=[float(p[c]) for c in cells]))
    return out


if __name__ == "__main__":
    for case in CASES:
        data = make(case)
        path = os.path.join(HERE, "exact_%s.json" % case["name"])
        with open(path, "w") as fh:
            json.dump(data, fh, indent=1)
        print("wrote", path)
    for case in POISSON_CASES:
        data = make_poisson(case)
        path = os.path.join(HERE, "poisson_%s.json" % case["name"])
        with open(path, "w") as fh:
            json.dump(data, fh, indent=1)
        print("wrote", path)
