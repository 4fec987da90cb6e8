"""Property test of the library's descriptor checks (host only, no device
work): seeded random descriptors, each field usually valid and sometimes not,
are either accepted (positive workspace size) or refused with
CR_E_INVALID_ARG, never anything else, and the decision equals the documented
rules restated here: walls and HLLC only for Euler, HLLC not with D1,
Gauss-Lobatto points without the blending and flux limiters, Burgers and
variable advection 1D, gravity only for Euler, time-dependent ghost states
only for scalar equations, no per-side override of a periodic direction,
finite (and for Euler admissible) given ghost states."""
import math
import random

import pytest

from paper_2502_07517_gb300 import crkfr


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2502_07517_gb300 import build
    build.build()
    crkfr.lib()


def _pick(r, valid, invalid, p_bad=0.03):
    return r.choice(invalid) if invalid and r.random() < p_bad else r.choice(valid)


def _draw(r):
    f = {
        "dim": _pick(r, [1, 2], [0, 3]),
        "nx": _pick(r, [1, 3, 17], [0, -2]),
        "ny": _pick(r, [1, 5, 12], [0, -1]),
        "bc_x": _pick(r, [0, 0, 0, 1, 1, 2, 3, 4], [-1, 5]),
        "bc_y": _pick(r, [0, 0, 0, 1, 1, 2, 3, 4], [-1, 5]),
        "degree": _pick(r, [1, 2, 3, 4], [0, 5]),
        "equation": _pick(r, [0, 1, 1, 2, 3, 4], [-1, 5]),
        "source": _pick(r, [0] * 6 + [1, 2], [-1, 3]),
        "g": _pick(r, [0.0, -1.0], [math.inf, math.nan]),
        "limiter": _pick(r, [0, 8, 16, 24, 31, 15], [32, -1]),
        "alpha_mode": _pick(r, [0, 0, 1, 2], [-1, 3]),
        "alpha_fixed": _pick(r, [0.0, 0.5, 1.0], [1.5, -0.1, math.nan]),
        "precision": _pick(r, [0, 1], [2, -1]),
        "dissipation": _pick(r, [0, 1, 2], [-1, 3]),
        "central": _pick(r, [0, 1], [-1, 2]),
        "points": _pick(r, [0, 0, 0, 1], [-1, 2]),
        "sides": [_pick(r, [0] * 9 + [1, 2, 3, 4], [-1, 5], 0.02) for _ in range(4)],
        # rho, momenta, energy / moments: admissible for Euler and ten-moment
        "state": [2.0, 0.3, -0.2, 1.5, 0.7, 1.1] if r.random() > 0.1 else
                 r.choice([[math.nan] * 6, [-1.0, 0, 0, 1.0, 1.0, 1.0], [1.0, 0, 0, 0.0, 0, 0]]),
        "bc_flux": _pick(r, [0, 0, 0, 1], [-1, 2]),
        "terms": _pick(r, [0] * 6 + [3, 16], [-1, 17]),
        "gamma": _pick(r, [1.4, 5.0 / 3.0], [1.0, math.nan]),
        "dom": r.random() > 0.03,
    }
    return f


def _desc(f):
    d = crkfr.cr_mesh_desc()
    d.dim, d.nx, d.ny = f["dim"], f["nx"], f["ny"]
    d.x0, d.x1, d.y0, d.y1 = 0.0, 1.0 if f["dom"] else 0.0, 0.0, 1.0
    d.bc_x, d.bc_y = f["bc_x"], f["bc_y"]
    d.degree, d.equation, d.gamma = f["degree"], f["equation"], f["gamma"]
    d.adv[0], d.adv[1] = 1.0, 0.5
    d.source = f["source"]
    d.gravity[0], d.gravity[1] = 0.0, f["g"]
    d.limiter, d.alpha_mode, d.alpha_fixed = f["limiter"], f["alpha_mode"], f["alpha_fixed"]
    d.precision = f["precision"]
    d.dissipation, d.central, d.points = f["dissipation"], f["central"], f["points"]
    for s in range(4):
        d.bc_side[s] = f["sides"][s]
        for v in range(6):
            d.bc_state[s][v] = f["state"][v]
    d.bc_flux = f["bc_flux"]
    d.bc_time_terms = f["terms"]
    d.bc_time_span[0], d.bc_time_span[1] = 0.0, 1.0
    d.adv_poly[2] = 1.0
    return d


def _nvars(f):
    return {0: 1, 1: 3 if f["dim"] == 1 else 4, 2: 6, 3: 1, 4: 1}[f["equation"]]


def _ghost_ok(f):
    M = _nvars(f)
    g = f["state"]
    if not all(math.isfinite(x) for x in g[:M]):
        return False
    if f["equation"] == 1:
        kin = 0.5 * g[1] ** 2 if f["dim"] == 1 else 0.5 * (g[1] ** 2 + g[2] ** 2)
        return g[0] > 0 and (f["gamma"] - 1.0) * (g[M - 1] - kin / g[0]) > 0
    if f["equation"] == 2:
        p11, p22 = 2 * g[3] - g[1] ** 2 / g[0], 2 * g[5] - g[2] ** 2 / g[0]
        p12 = 2 * g[4] - g[1] * g[2] / g[0]
        return g[0] > 0 and p11 > 0 and p11 * p22 - p12 * p12 > 0
    return True


def _expected_ok(f):
    """The documented acceptance rules, written independently of the library."""
    if f["dim"] not in (1, 2) or not 1 <= f["degree"] <= 4:
        return False
    if f["nx"] < 1 or (f["dim"] == 2 and f["ny"] < 1) or not f["dom"]:
        return False
    if not 0 <= f["bc_x"] <= 4 or (f["dim"] == 2 and not 0 <= f["bc_y"] <= 4):
        return False
    if not 0 <= f["equation"] <= 4:
        return False
    nside = 4 if f["dim"] == 2 else 2
    for s in range(nside):
        dirbc = f["bc_x"] if s < 2 else f["bc_y"]
        if not 0 <= f["sides"][s] <= 4:
            return False
        if f["sides"][s] != 0 and dirbc == 0:
            return False
        bc = f["sides"][s] or dirbc
        if bc == 2 and f["equation"] != 1:
            return False
        if bc in (3, 4) and not _ghost_ok(f):
            return False
    if f["equation"] in (3, 4) and f["dim"] != 1:
        return False
    if not 0 <= f["terms"] <= 16 or not 0 <= f["bc_flux"] <= 1:
        return False
    if f["bc_flux"] == 1 and (f["equation"] != 1 or f["dissipation"] == 1):
        return False
    if f["terms"] > 0 and _nvars(f) != 1:
        return False
    if not 0 <= f["dissipation"] <= 2 or f["central"] not in (0, 1) or f["points"] not in (0, 1):
        return False
    if f["points"] == 1 and (f["limiter"] & 7 or f["alpha_mode"] == 1):
        return False
    if f["equation"] == 1 and not f["gamma"] > 1.0:
        return False
    if f["precision"] not in (0, 1) or f["alpha_mode"] not in (0, 1, 2):
        return False
    if f["alpha_mode"] == 1 and not 0.0 <= f["alpha_fixed"] <= 1.0:
        return False
    if not 0 <= f["source"] <= 2:
        return False
    if f["source"] == 1 and f["equation"] != 2:
        return False
    if f["source"] == 2 and (f["equation"] != 1 or not math.isfinite(f["g"])):
        return False
    return 0 <= f["limiter"] <= 31


def test_descriptor_decisions():
    r = random.Random(20250207)
    accepted = refused = 0
    for i in range(4000):
        f = _draw(r)
        try:
            nbytes = crkfr.cr_workspace_bytes(_desc(f))
            ok = True
            assert nbytes > 0
        except crkfr.CrError as err:
            assert err.status == -1, (i, err)   # CR_E_INVALID_ARG
            ok = False
        assert ok == _expected_ok(f), (i, f, ok)
        accepted += ok
        refused += not ok
    # both decisions are exercised in quantity
    assert accepted > 400 and refused > 400, (accepted, refused)
