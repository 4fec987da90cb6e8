"""Python binding of libcrkfr.so (include/cr.h): argument marshalling only.

Every step of the method runs in the library's CUDA kernels.  PyTorch supplies
device memory (the workspace and device state tensors) and the CUDA stream.
The library must have been built (paper_2502_07517_gb300.build.build());
loading fails loudly otherwise, there is no fallback.
"""
import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libcrkfr.so")

CR_OK = 0
STATUS = {0: "CR_OK", -1: "CR_E_INVALID_ARG", -2: "CR_E_INVALID_STATE", -3: "CR_E_INADMISSIBLE",
          -4: "CR_E_TIMEOUT", -5: "CR_E_CUDA", -6: "CR_E_NOMEM", -7: "CR_E_UNSUPPORTED",
          -8: "CR_E_TOO_LARGE"}
CR_EQ_LINADV, CR_EQ_EULER, CR_EQ_TENMOMENT, CR_EQ_BURGERS, CR_EQ_VARADV = 0, 1, 2, 3, 4
CR_BC_PERIODIC, CR_BC_OUTFLOW, CR_BC_WALL, CR_BC_DIRICHLET, CR_BC_INFLOW = 0, 1, 2, 3, 4
CR_SRC_NONE, CR_SRC_TENMOMENT, CR_SRC_GRAVITY = 0, 1, 2
CR_POINTS_GL, CR_POINTS_GLL = 0, 1
CR_LIM_BLEND, CR_LIM_MH, CR_LIM_FLUX, CR_LIM_SCALING, CR_LIM_TRACES = 1, 2, 4, 8, 16
CR_ALPHA_INDICATOR, CR_ALPHA_FIXED, CR_ALPHA_MLP = 0, 1, 2
CR_FP64, CR_FP32_BULK = 0, 1
CR_BATCH_PHASES, CR_BATCH_FUSED = 0, 1
CR_DISS_D2, CR_DISS_D1, CR_DISS_DCSX = 0, 1, 2
CR_CENTRAL_EA, CR_CENTRAL_AE = 0, 1

# C symbols declared in include/cr.h
SYMBOLS = ("cr_workspace_bytes", "cr_init_mesh", "cr_destroy", "cr_set_state", "cr_get_state",
           "cr_step", "cr_step_get", "cr_step_async", "cr_sync", "cr_get_alpha", "cr_get_means", "cr_next_dt",
           "cr_cfl_number_for", "cr_cfl_number_points", "cr_reference_tables_points",
           "cr_launches_per_step", "cr_profile_steps", "cr_cfl_number", "cr_reference_tables",
           "cr_step_static", "cr_last_error", "cr_mlp_param_count", "cr_mlp_load",
           "cr_get_features", "cr_mlp_grad", "cr_mlp_train", "cr_batch_init", "cr_batch_destroy",
           "cr_batch_config", "cr_batch_autotune", "cr_batch_step_async", "cr_batch_sync",
           "cr_batch_step", "cr_batch_last_error", "cr_batch_barrier_test")


class CrError(RuntimeError):
    def __init__(self, status, message):
        super().__init__("%s: %s" % (STATUS.get(status, status), message))
        self.status = status


class cr_mesh_desc(ctypes.Structure):
    _fields_ = [
        ("dim", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int),
        ("x0", ctypes.c_double), ("x1", ctypes.c_double),
        ("y0", ctypes.c_double), ("y1", ctypes.c_double),
        ("bc_x", ctypes.c_int), ("bc_y", ctypes.c_int),
        ("degree", ctypes.c_int), ("equation", ctypes.c_int),
        ("gamma", ctypes.c_double), ("adv", ctypes.c_double * 2),
        ("source", ctypes.c_int),
        ("src_amp", ctypes.c_double), ("src_k", ctypes.c_double),
        ("src_cx", ctypes.c_double), ("src_cy", ctypes.c_double),
        ("limiter", ctypes.c_int), ("alpha_mode", ctypes.c_int),
        ("alpha_fixed", ctypes.c_double), ("precision", ctypes.c_int),
        ("cfl", ctypes.c_double), ("cfl_safety", ctypes.c_double),
        ("stream", ctypes.c_void_p),
        ("dissipation", ctypes.c_int), ("central", ctypes.c_int),
        ("bc_side", ctypes.c_int * 4), ("bc_state", (ctypes.c_double * 6) * 4),
        ("gravity", ctypes.c_double * 2), ("points", ctypes.c_int),
        ("adv_poly", ctypes.c_double * 4), ("bc_time_terms", ctypes.c_int),
        ("bc_time_span", ctypes.c_double * 2), ("bc_time_coef", (ctypes.c_double * 16) * 4),
        ("bc_flux", ctypes.c_int),
    ]


_lib = None


def lib():
    """Load libcrkfr.so; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libcrkfr.so is missing at %s: build it with "
                               "paper_2502_07517_gb300.build.build()" % LIB_PATH)
        L = ctypes.CDLL(LIB_PATH)
        P, D, V = ctypes.POINTER(cr_mesh_desc), ctypes.POINTER(ctypes.c_double), ctypes.c_void_p
        I = ctypes.c_int
        L.cr_workspace_bytes.argtypes = [P, ctypes.POINTER(ctypes.c_size_t)]
        L.cr_init_mesh.argtypes = [P, V, ctypes.c_size_t, ctypes.POINTER(V)]
        L.cr_destroy.argtypes = [V]
        L.cr_destroy.restype = None
        L.cr_set_state.argtypes = [V, V, I]
        L.cr_get_state.argtypes = [V, V, I]
        L.cr_step.argtypes = [V, I, ctypes.c_double, ctypes.c_double, D, ctypes.POINTER(I)]
        L.cr_step_get.argtypes = [V, I, ctypes.c_double, ctypes.c_double, V, D, ctypes.POINTER(I)]
        L.cr_step_async.argtypes = [V, I, ctypes.c_double, ctypes.c_double]
        L.cr_sync.argtypes = [V, D, ctypes.POINTER(I)]
        L.cr_get_alpha.argtypes = [V, V, I]
        L.cr_get_means.argtypes = [V, V, I]
        L.cr_next_dt.argtypes = [V, D]
        L.cr_launches_per_step.argtypes = [V, ctypes.POINTER(I)]
        L.cr_profile_steps.argtypes = [V, I, ctypes.c_double, ctypes.c_double, D]
        L.cr_cfl_number.argtypes = [I, D]
        L.cr_cfl_number_for.argtypes = [I, I, D]
        L.cr_reference_tables.argtypes = [I, D, D, D]
        L.cr_cfl_number_points.argtypes = [I, I, I, D]
        L.cr_reference_tables_points.argtypes = [I, I, D, D, D]
        L.cr_step_static.argtypes = [P, V, V, ctypes.c_double]
        F = ctypes.POINTER(ctypes.c_float)
        L.cr_mlp_param_count.argtypes = [I]
        L.cr_mlp_load.argtypes = [V, F, I]
        L.cr_get_features.argtypes = [V, V, V, I]
        L.cr_mlp_grad.argtypes = [I, V, V, V, I, V, V, V]
        L.cr_mlp_train.argtypes = [I, V, V, V, I, I, I, ctypes.c_float, ctypes.c_ulonglong, F, V]
        L.cr_last_error.argtypes = [V]
        L.cr_last_error.restype = ctypes.c_char_p
        L.cr_batch_init.argtypes = [ctypes.POINTER(V), I, ctypes.POINTER(V)]
        L.cr_batch_destroy.argtypes = [V]
        L.cr_batch_destroy.restype = None
        L.cr_batch_config.argtypes = [V, I, I, I]
        L.cr_batch_autotune.argtypes = [V, I, ctypes.POINTER(I), ctypes.POINTER(I), ctypes.POINTER(I), D]
        L.cr_batch_step_async.argtypes = [V, I, ctypes.c_double]
        L.cr_batch_sync.argtypes = [V]
        L.cr_batch_step.argtypes = [V, I, ctypes.c_double]
        L.cr_batch_barrier_test.argtypes = [V, ctypes.c_ulonglong, I]
        L.cr_batch_last_error.argtypes = [V]
        L.cr_batch_last_error.restype = ctypes.c_char_p
        for s in SYMBOLS:
            if s not in ("cr_destroy", "cr_last_error", "cr_batch_destroy", "cr_batch_last_error"):
                getattr(L, s).restype = ctypes.c_int
        _lib = L
    return _lib


def _check(st, ctx=None):
    if st != CR_OK:
        msg = lib().cr_last_error(ctx)
        raise CrError(st, msg.decode() if msg else "")


def _dptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


# ------------------------------------------------------------------ C ABI ---
def cr_cfl_number(degree):
    out = ctypes.c_double()
    _check(lib().cr_cfl_number(int(degree), ctypes.byref(out)))
    return out.value


def cr_cfl_number_for(degree, dissipation):
    out = ctypes.c_double()
    _check(lib().cr_cfl_number_for(int(degree), int(dissipation), ctypes.byref(out)))
    return out.value


def cr_reference_tables(degree):
    n = degree + 1
    xi, w, D = np.zeros(n), np.zeros(n), np.zeros((n, n))
    _check(lib().cr_reference_tables(int(degree), _dptr(xi), _dptr(w), _dptr(D)))
    return xi, w, D


def cr_cfl_number_points(degree, dissipation, points):
    out = ctypes.c_double()
    _check(lib().cr_cfl_number_points(int(degree), int(dissipation), int(points), ctypes.byref(out)))
    return out.value


def cr_reference_tables_points(degree, points):
    n = degree + 1
    xi, w, D = np.zeros(n), np.zeros(n), np.zeros((n, n))
    _check(lib().cr_reference_tables_points(int(degree), int(points), _dptr(xi), _dptr(w), _dptr(D)))
    return xi, w, D


def cr_workspace_bytes(desc):
    out = ctypes.c_size_t()
    _check(lib().cr_workspace_bytes(ctypes.byref(desc), ctypes.byref(out)))
    return out.value


class Context:
    """Owns a cr_ctx and (when the caller gave none) the torch workspace tensor."""

    def __init__(self, handle, workspace, desc):
        self.handle = handle
        self.workspace = workspace
        self.desc = desc

    def __del__(self):
        if getattr(self, "handle", None):
            lib().cr_destroy(self.handle)
            self.handle = None


def cr_init_mesh(desc, workspace=None):
    """Create a context.  workspace=None allocates the device workspace as a
    torch uint8 tensor on the current device (256-byte aligned)."""
    import torch
    nbytes = cr_workspace_bytes(desc)
    if workspace is None:
        workspace = torch.empty(nbytes + 256, dtype=torch.uint8, device="cuda")
    base = workspace.data_ptr()
    aligned = (base + 255) & ~255
    handle = ctypes.c_void_p()
    _check(lib().cr_init_mesh(ctypes.byref(desc), ctypes.c_void_p(aligned),
                              nbytes, ctypes.byref(handle)))
    return Context(handle, workspace, desc)


def cr_destroy(ctx):
    if ctx.handle:
        lib().cr_destroy(ctx.handle)
        ctx.handle = None


def cr_set_state(ctx, u):
    """u: numpy float64 [M][Ne][Np] (host) or a torch float64 CUDA tensor."""
    if isinstance(u, np.ndarray):
        u = np.ascontiguousarray(u, dtype=np.float64)
        _check(lib().cr_set_state(ctx.handle, u.ctypes.data, 0), ctx.handle)
    else:
        assert u.is_cuda and u.dtype.is_floating_point and u.element_size() == 8 and u.is_contiguous()
        _check(lib().cr_set_state(ctx.handle, u.data_ptr(), 1), ctx.handle)


def cr_get_state(ctx, out=None, shape=None):
    """Returns a numpy array (out=None, needs shape) or fills a torch CUDA tensor."""
    if out is None:
        out = np.empty(shape, dtype=np.float64)
    if isinstance(out, np.ndarray):
        _check(lib().cr_get_state(ctx.handle, out.ctypes.data, 0), ctx.handle)
    else:
        _check(lib().cr_get_state(ctx.handle, out.data_ptr(), 1), ctx.handle)
    return out


def cr_step(ctx, max_steps, t_final, dt_fixed=0.0):
    """Returns (t, steps); raises CrError on an inadmissible step."""
    t = ctypes.c_double()
    n = ctypes.c_int()
    _check(lib().cr_step(ctx.handle, int(max_steps), float(t_final), float(dt_fixed),
                         ctypes.byref(t), ctypes.byref(n)), ctx.handle)
    return t.value, n.value


def cr_step_get(ctx, max_steps, t_final, out, dt_fixed=0.0):
    """cr_step, then the state into out: host memory, a C-contiguous float64
    numpy array or CPU torch tensor of M * Ne * Np values (pinned: written by
    the last step's update kernel).  Returns (t, steps)."""
    want = _state_numel(ctx.desc)
    if isinstance(out, np.ndarray):
        ok = out.dtype == np.float64 and out.flags.c_contiguous and out.size == want
        ptr = out.ctypes.data
    else:
        import torch
        ok = (isinstance(out, torch.Tensor) and not out.is_cuda and out.dtype == torch.float64
              and out.is_contiguous() and out.numel() == want)
        ptr = out.data_ptr() if ok else 0
    if not ok:
        raise CrError(-1, "cr_step_get: out must be contiguous float64 host memory of %d values" % want)
    t = ctypes.c_double()
    n = ctypes.c_int()
    _check(lib().cr_step_get(ctx.handle, int(max_steps), float(t_final), float(dt_fixed), ptr,
                             ctypes.byref(t), ctypes.byref(n)), ctx.handle)
    return t.value, n.value


def cr_step_async(ctx, max_steps, t_final, dt_fixed=0.0):
    _check(lib().cr_step_async(ctx.handle, int(max_steps), float(t_final), float(dt_fixed)),
           ctx.handle)


def cr_sync(ctx):
    t = ctypes.c_double()
    n = ctypes.c_int()
    _check(lib().cr_sync(ctx.handle, ctypes.byref(t), ctypes.byref(n)), ctx.handle)
    return t.value, n.value


def cr_get_alpha(ctx, ne):
    out = np.empty(ne, dtype=np.float64)
    _check(lib().cr_get_alpha(ctx.handle, out.ctypes.data, 0), ctx.handle)
    return out


def cr_get_means(ctx, M, ne):
    """FP64 element means [M][Ne] (the conserved quantities)."""
    out = np.empty((M, ne), dtype=np.float64)
    _check(lib().cr_get_means(ctx.handle, out.ctypes.data, 0), ctx.handle)
    return out


def cr_next_dt(ctx):
    out = ctypes.c_double()
    _check(lib().cr_next_dt(ctx.handle, ctypes.byref(out)), ctx.handle)
    return out.value


def cr_launches_per_step(ctx):
    out = ctypes.c_int()
    _check(lib().cr_launches_per_step(ctx.handle, ctypes.byref(out)), ctx.handle)
    return out.value


def cr_profile_steps(ctx, max_steps, t_final, dt_fixed=0.0):
    """Runs the steps with per-kernel CUDA events; returns device ms per kernel."""
    n = cr_launches_per_step(ctx)
    ms = np.zeros(n)
    _check(lib().cr_profile_steps(ctx.handle, int(max_steps), float(t_final), float(dt_fixed),
                                  _dptr(ms)), ctx.handle)
    return ms


def _state_numel(desc):
    """M * Ne * Np of a description."""
    M = {CR_EQ_LINADV: 1, CR_EQ_BURGERS: 1, CR_EQ_VARADV: 1, CR_EQ_TENMOMENT: 6}.get(
        desc.equation, 3 if desc.dim == 1 else 4)
    ne = desc.nx * (desc.ny if desc.dim == 2 else 1)
    return M * ne * (desc.degree + 1) ** desc.dim


def cr_step_static(desc, u_in, u_out, dt):
    """One FP64 step with the library's fixed scratch array (no allocation);
    u_in, u_out are contiguous torch float64 tensors [M][Ne][Np] on the
    current CUDA device, the same tensor or disjoint ones.  Anything else is
    refused with CR_E_INVALID_ARG before the library sees the pointers."""
    import torch
    want = _state_numel(desc)
    for name, t in (("u_in", u_in), ("u_out", u_out)):
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64
                and t.is_contiguous() and t.numel() == want
                and t.device.index == torch.cuda.current_device()):
            raise CrError(-1, "cr_step_static: %s must be a contiguous float64 tensor of %d values "
                              "on the current CUDA device" % (name, want))
    a0, b0 = u_in.data_ptr(), u_out.data_ptr()
    nbytes = want * 8
    if a0 != b0 and a0 < b0 + nbytes and b0 < a0 + nbytes:
        raise CrError(-1, "cr_step_static: u_in and u_out overlap without being the same tensor")
    st = lib().cr_step_static(ctypes.byref(desc), a0, b0, float(dt))
    if st != CR_OK:
        raise CrError(st, lib().cr_last_error(None).decode())


def cr_mlp_param_count(nin):
    return lib().cr_mlp_param_count(int(nin))


def cr_mlp_load(ctx, params):
    """Load the learned-alpha network (FP32 parameter vector; stored as BF16)."""
    p = np.ascontiguousarray(params, dtype=np.float32)
    _check(lib().cr_mlp_load(ctx.handle, p.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), p.size),
           ctx.handle)


def cr_get_features(ctx, ne, npts):
    """(features [Ne][Np] float32, raw alpha [Ne] float64) of the current state."""
    f = np.empty((ne, npts), dtype=np.float32)
    a = np.empty(ne, dtype=np.float64)
    _check(lib().cr_get_features(ctx.handle, f.ctypes.data, a.ctypes.data, 0), ctx.handle)
    return f, a


def cr_get_features_device(ctx, feat, alpha_raw=None):
    """Device variant: feat is a float32 CUDA tensor [Ne][Np]; alpha_raw an
    optional float64 CUDA tensor [Ne]."""
    _check(lib().cr_get_features(ctx.handle, feat.data_ptr(),
                                 alpha_raw.data_ptr() if alpha_raw is not None else None, 1),
           ctx.handle)


def cr_mlp_grad(nin, params, X, t, grad, loss, stream=None):
    """Loss and gradient on device tensors (float32): params [P], X [n][nin], t [n]."""
    st = lib().cr_mlp_grad(int(nin), params.data_ptr(), X.data_ptr(), t.data_ptr(), int(t.numel()),
                           grad.data_ptr(), loss.data_ptr(), stream)
    if st != CR_OK:
        raise CrError(st, "cr_mlp_grad")


def cr_mlp_train(nin, params, X, t, batch, epochs, lr, seed=0, stream=None):
    """Adam training in place on device tensors; returns the last epoch's mean loss."""
    out = ctypes.c_float()
    st = lib().cr_mlp_train(int(nin), params.data_ptr(), X.data_ptr(), t.data_ptr(), int(t.numel()),
                            int(batch), int(epochs), float(lr), int(seed), ctypes.byref(out), stream)
    if st != CR_OK:
        raise CrError(st, "cr_mlp_train")
    return out.value


class Batch:
    """Owns a cr_batch; keeps its contexts alive."""

    def __init__(self, handle, ctxs):
        self.handle = handle
        self.ctxs = list(ctxs)

    def __del__(self):
        if getattr(self, "handle", None):
            lib().cr_batch_destroy(self.handle)
            self.handle = None


def _bcheck(st, b=None):
    if st != CR_OK:
        msg = lib().cr_batch_last_error(b.handle if b is not None else None)
        raise CrError(st, msg.decode() if msg else "")


def cr_batch_init(ctxs):
    arr = (ctypes.c_void_p * len(ctxs))(*[c.handle.value if isinstance(c.handle, ctypes.c_void_p)
                                          else c.handle for c in ctxs])
    out = ctypes.c_void_p()
    _bcheck(lib().cr_batch_init(arr, len(ctxs), ctypes.byref(out)))
    return Batch(out, ctxs)


def cr_batch_destroy(b):
    if b.handle:
        lib().cr_batch_destroy(b.handle)
        b.handle = None


def cr_batch_config(b, threads, mode, tiles=1):
    _bcheck(lib().cr_batch_config(b.handle, int(threads), int(mode), int(tiles)), b)


BATCH_CANDIDATES = [(t, m, k) for t in (128, 256)
                    for m, k in ((CR_BATCH_PHASES, 1), (CR_BATCH_FUSED, 1), (CR_BATCH_FUSED, 2),
                                 (CR_BATCH_FUSED, 4))]


def cr_batch_autotune(b, trial_steps=3):
    """Returns (threads, mode, tiles, ms per step of the candidates in the
    order of BATCH_CANDIDATES)."""
    t, m, k = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    ms = np.zeros(len(BATCH_CANDIDATES))
    _bcheck(lib().cr_batch_autotune(b.handle, int(trial_steps), ctypes.byref(t), ctypes.byref(m),
                                    ctypes.byref(k), _dptr(ms)), b)
    return t.value, m.value, k.value, ms


def cr_batch_step_async(b, nsteps, t_final=1e300):
    _bcheck(lib().cr_batch_step_async(b.handle, int(nsteps), float(t_final)), b)


def cr_batch_sync(b):
    _bcheck(lib().cr_batch_sync(b.handle), b)


def cr_batch_step(b, nsteps, t_final=1e300):
    _bcheck(lib().cr_batch_step(b.handle, int(nsteps), float(t_final)), b)


def cr_batch_barrier_test(b, polls, phantom):
    """Fault injection for the fused kernel's timeout path (tests)."""
    _bcheck(lib().cr_batch_barrier_test(b.handle, int(polls), int(phantom)), b)


def cr_batch_last_error(b=None):
    msg = lib().cr_batch_last_error(b.handle if b is not None else None)
    return msg.decode() if msg else ""


def cr_last_error(ctx=None):
    msg = lib().cr_last_error(ctx.handle if ctx else None)
    return msg.decode() if msg else ""


# ------------------------------------------------------ problem marshalling -
_EQ = {"linadv": CR_EQ_LINADV, "euler": CR_EQ_EULER, "tenmoment": CR_EQ_TENMOMENT,
       "burgers": CR_EQ_BURGERS, "varadv": CR_EQ_VARADV}
_BC = {"periodic": CR_BC_PERIODIC, "outflow": CR_BC_OUTFLOW, "wall": CR_BC_WALL,
       "dirichlet": CR_BC_DIRICHLET, "inflow": CR_BC_INFLOW}
_SIDES = ("x-", "x+", "y-", "y+")
_LIM = {"blend": CR_LIM_BLEND, "mh": CR_LIM_MH, "flux": CR_LIM_FLUX, "scaling": CR_LIM_SCALING,
        "traces": CR_LIM_TRACES}


def desc_from_problem(prob, precision=CR_FP64, alpha_fixed=None, stream=None, **over):
    """cr_mesh_desc from a workload problem dict (see workloads.py)."""
    d = cr_mesh_desc()
    d.dim, d.nx, d.ny = prob["dim"], prob["nx"], prob["ny"] if prob["dim"] == 2 else 1
    d.x0, d.x1, d.y0, d.y1 = prob["x0"], prob["x1"], prob["y0"], prob["y1"]
    d.bc_x, d.bc_y = _BC[prob["bc_x"]], _BC[prob["bc_y"]]
    d.degree, d.equation, d.gamma = prob["degree"], _EQ[prob["equation"]], prob["gamma"]
    d.adv[0], d.adv[1] = prob["adv"]
    src = prob.get("source")
    if src and "gravity" in src:
        d.source = CR_SRC_GRAVITY
        d.gravity[0], d.gravity[1] = src["gravity"]
    elif src:
        d.source, d.src_amp, d.src_k, d.src_cx, d.src_cy = (CR_SRC_TENMOMENT, src["amp"], src["k"],
                                                             src["cx"], src["cy"])
    d.points = {"gl": CR_POINTS_GL, "gll": CR_POINTS_GLL}[prob.get("points", "gl")]
    for k, a in enumerate(prob.get("adv_poly") or ()):
        d.adv_poly[k] = a
    d.bc_flux = 1 if prob.get("bc_flux") == "hllc" else 0
    bt = prob.get("bc_time")
    if bt:
        d.bc_time_span[0], d.bc_time_span[1] = bt["span"]
        d.bc_time_terms = max(len(c) for c in bt["coef"].values())
        for s, c in bt["coef"].items():
            for k, a in enumerate(c):
                d.bc_time_coef[_SIDES.index(s)][k] = a
    sides, states = prob.get("bc_side") or {}, prob.get("bc_state") or {}
    for i, s in enumerate(_SIDES):
        d.bc_side[i] = _BC[sides[s]] if s in sides else 0
        for v, x in enumerate(states.get(s) or ()):
            d.bc_state[i][v] = x
    lim = 0
    for name in prob["limiter"]:
        lim |= _LIM[name]
    d.limiter = lim
    if alpha_fixed is not None:
        d.alpha_mode, d.alpha_fixed = CR_ALPHA_FIXED, alpha_fixed
    d.precision = precision
    d.cfl, d.cfl_safety = 0.0, 0.98
    d.stream = stream
    for k, v in over.items():
        setattr(d, k, v)
    return d
