"""Test helper: build an oracle description from a workload problem dict."""
import oracle

_EQ = {"linadv": oracle.EQ_LINADV, "euler": oracle.EQ_EULER, "tenmoment": oracle.EQ_TENMOMENT,
       "burgers": oracle.EQ_BURGERS}
_BC = {"periodic": oracle.BC_PERIODIC, "outflow": oracle.BC_OUTFLOW, "wall": oracle.BC_WALL}
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
    if src:
        kw.update(source=1, src_amp=src["amp"], src_k=src["k"], src_cx=src["cx"],
                  src_cy=src["cy"])
    if alpha_fixed is not None:
        kw.update(alpha_mode=oracle.ALPHA_FIXED, alpha_fixed=alpha_fixed)
    kw.update(over)
    return oracle.make_desc(**kw)
