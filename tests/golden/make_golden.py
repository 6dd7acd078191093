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


if __name__ == "__main__":
    for case in CASES:
        data = make(case)
        path = os.path.join(HERE, "exact_%s.json" % case["name"])
        with open(path, "w") as fh:
            json.dump(data, fh, indent=1)
        print("wrote", path)
