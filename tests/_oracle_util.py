"""Test helper: build an oracle description from a workload problem dict."""
import oracle

_EQ = {"linadv": oracle.EQ_LINADV, "euler": oracle.EQ_EULER, "tenmoment": oracle.EQ_TENMOMENT,
       "burgers": oracle.EQ_BURGERS, "varadv": oracle.EQ_VARADV}
_BC = {"periodic": oracle.BC_PERIODIC, "outflow": oracle.BC_OUTFLOW, "wall": oracle.BC_WALL,
       "dirichlet": oracle.BC_DIRICHLET, "inflow": oracle.BC_INFLOW}
SIDES = ("x-", "x+", "y-", "y+")
_LIM = {"blend": oracle.LIM_BLEND, "mh": oracle.LIM_MH, "flux": oracle.LIM_FLUX,
        "scaling": oracle.LIM_SCALING, "traces": oracle.LIM_TRACES}


def oracle_desc(prob, alpha_fixed=None, **over):
    lim = 0
    for name in prob["limiter"]:
        lim |= _LIM[name]
    src = prob.get("source")
    kw = dict(dim=prob["dim"], nx=prob["nx"], ny=prob["ny"], x0=prob["x0"], x1=prob["x1"],
              y0=prob["y0"], y1=prob["y1"], bc_x=_BC[prob["bc_x"]], bc_y=_BC[prob["bc_y"]],
              degree=prob["degree"], equation=_EQ[prob["equation"]], gamma=prob["gamma"],
              adv=tuple(prob["adv"]), limiter=lim)
    if src and "gravity" in src:
        kw.update(source=oracle.SRC_GRAVITY, gravity=tuple(src["gravity"]))
    elif src:
        kw.update(source=oracle.SRC_TENMOMENT, src_amp=src["amp"], src_k=src["k"], src_cx=src["cx"],
                  src_cy=src["cy"])
    sides = prob.get("bc_side") or {}
    states = prob.get("bc_state") or {}
    kw.update(bc_side=tuple(_BC[sides[s]] if s in sides else 0 for s in SIDES),
              bc_state=[states.get(s) for s in SIDES])
    kw.update(points={"gl": oracle.POINTS_GL, "gll": oracle.POINTS_GLL}[prob.get("points", "gl")])
    if prob.get("bc_flux") == "hllc":
        kw.update(bc_flux=1)
    if "adv_poly" in prob:
        kw.update(adv_poly=tuple(prob["adv_poly"]))
    bt = prob.get("bc_time")
    if bt:
        kw.update(bc_time=(tuple(bt["span"]), {SIDES.index(s): c for s, c in bt["coef"].items()}))
    if alpha_fixed is not None:
        kw.update(alpha_mode=oracle.ALPHA_FIXED, alpha_fixed=alpha_fixed)
    kw.update(over)
    return oracle.make_desc(**kw)
