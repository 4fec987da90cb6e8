"""Benchmark of the GB300 cRKFR step (one JSON line on rank 0).

Workload: 2D Euler (gamma 1.4), degree N = 4 (25 Gauss-Legendre points per
element, 4 variables), 512 x 512 elements on [-5,5]^2 periodic, isentropic
vortex with a seeded 1% density perturbation, all limiters on (blending with
MUSCL-Hancock subcells, flux limiter, scaling limiter); one step = one
cRKFR time step at the CFL time step over the whole mesh.

Metric: DOF-updates/s = solution points x steps / second (whole job).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--mode fp64|fp32] [--impl ours|reference]

With N > 1 (launched by torch.distributed.run) every rank runs an independent
replica of the workload (different seed): weak scaling, no collective on the
data path; timing is the max over ranks.
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2502_07517_gb300 import workloads as wl  # noqa: E402

WORKLOAD = dict(name="euler2d_vortex_512x512_N4", nx=512, degree=4)
MEASURED_PEAKS = os.path.join(ROOT, "MEASURED_PEAKS.json")
# ALU peaks from the unit counts and the maximum SM clock: 152 SMs; FP64 2 FMA
# lanes per SM per clock (1.25 TFLOP/s nominal), FP32 128 FMA lanes per SM.
SM_COUNT, SM_MAX_MHZ = 152, 2070.0
# DRAM bytes (read + write) per element of the dominant kernel, from one ncu
# capture of the current kernel at 384x384 (147,456 elements; the traffic
# scales with the element count): FP64 k_local 589.5 MB, FP32 bulk k_local
# 283.4 MB (the k_local summaries under profiles/).
NCU_TRAFFIC_PER_ELEMENT = {("fp64", "k_local"): 589.46e6 / 147456, ("fp32", "k_local"): 283.41e6 / 147456}
PEAK_FP64_TFLOPS = SM_COUNT * 2 * 2 * SM_MAX_MHZ * 1e6 / 1e12
PEAK_FP32_TFLOPS = SM_COUNT * 128 * 2 * SM_MAX_MHZ * 1e6 / 1e12


# ---------------------------------------------------------------------------
# Algorithmic FLOP model of one step (add/sub/mul/div/sqrt = 1, fma = 2).
# Per-evaluation costs: (M, flux per direction, wave speed, 2nd constraint,
# indicator variable, source).
EQ_COST = {"linadv1d": (1, 1, 1, 0, 0, 0), "linadv2d": (1, 1, 1, 0, 0, 0),
           "euler1d": (3, 10, 10, 5, 6, 0), "euler2d": (4, 14, 12, 7, 8, 0),
           "tenmoment1d": (6, 24, 8, 19, 9, 8), "tenmoment2d": (6, 24, 8, 19, 9, 8)}
TABLEAU = {1: (2, 1, 1), 2: (3, 2, 2), 3: (4, 3, 4), 4: (6, 12, 5)}  # stages, nnz(A), nnz(b)


def flop_model(dim, N, eq, source=False):
    """Per solution point flops of (k_local, k_face, k_update) for one step with
    all limiters on (the face kernel's flops are spread over the element's points)."""
    M, fl, sp, c2, ind, src = EQ_COST[eq]
    n = N + 1
    NP = n ** dim
    nslot = (4 * n if dim == 2 else 2) / NP  # face-node slots per point
    S, nnza, nnzb = TABLEAU[N]
    loc = nnza * M * 2                                # stage values
    loc += S * (dim * fl + (src if source else 0))    # fluxes and source at the points
    loc += nnzb * (dim + 2) * M * 2                   # F, (G), U, S accumulation
    loc += (S - 1) * M * dim * 2 * n                  # D contractions (1/dx, 1/dy in the tables)
    loc += nnzb * nslot * (M * 2 * n + fl + 2 * M)    # EA traces and fluxes
    loc += M * dim * 2 * n                            # high-order volume part (likewise)
    loc += nslot * (2 * M * 2 * n + sp)               # U and u^n traces, wave speed
    loc += dim * M * 9 + 2 * dim * M * 2 + 2 * dim * fl + dim * M * 5 + 2 * dim * M  # MUSCL-Hancock
    loc += 4 * dim * c2                               # admissibility of face/evolved states
    loc += dim * (N / n) * (2 * fl + 2 * sp + 5 * M)  # subcell Rusanov fluxes
    loc += dim * M * 3 + nslot * M * 2 + M * 7        # low-order residual, face data, partial update
    face_nodes = (2 * n if dim == 2 else 1) / NP      # face nodes per point
    face = face_nodes * (M * 4 + 2 * fl + 2 * sp + 5 * M + 3 * M + 2 * 2 * 2 * (2 * M + c2) + 3 * M)
    upd = dim * (M * 4 + 4) + 2 * M + nslot * M * 2 * n + (1 + nslot) * c2 + ind + 2 * n * dim + 1
    return loc, face, upd


# ---------------------------------------------------------------------------
class ClockSampler:
    """nvidia-smi samples (200 ms) while the timed region runs."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            self.proc.wait()
            self.thread.join(timeout=2)

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[4:8]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def aggregate_timing(ms, nodes, steps, world, tdist=None, device="cpu"):
    """Replicas: every rank timed its own workload of `nodes` solution points for
    `steps` steps; the job's time is the slowest rank's and its throughput counts
    the points of all ranks.  Returns (ms_max, DOF-updates/s)."""
    if world > 1:
        import torch
        t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
        tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
        ms = float(t.item())
    return ms, world * nodes * steps / (ms * 1e-3)


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), \
        int(os.environ.get("LOCAL_RANK", 0))


def make_workload(seed, nx=None, degree=None):
    prob, u = wl.euler2d_vortex(nx=nx or WORKLOAD["nx"], degree=degree or WORKLOAD["degree"], seed=seed)
    return prob, u


def _host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


_SAMPLES = {}


def _oracle_sample(job):
    """One replica: the oracle, as it stands, on an nx x nx sample of the bench
    recipe, whole steps until target_s has passed (at least one).  Returns
    (point updates, seconds)."""
    nx, target_s, seed = job
    import oracle
    from tests._oracle_util import oracle_desc
    if (nx, seed) not in _SAMPLES:  # generated once per process, outside the timing
        prob, u = make_workload(seed, nx=nx)
        _SAMPLES[(nx, seed)] = (oracle_desc(prob), u)
    d, u = _SAMPLES[(nx, seed)]
    steps, t0 = 0, time.perf_counter()
    while True:
        u, st = oracle.step(d, u, oracle.dt(d, u))
        steps += 1
        el = time.perf_counter() - t0
        if el >= target_s or st != 0:
            break
    return u.shape[1] * u.shape[2] * steps, el


def cpu_baseline(target_s=10.0, nx=128, cores=None):
    """The FP64 oracle as it stands on every host core: one independent replica
    of a bounded sample per core, in spawned processes (no GPU state is
    inherited), all at once; the throughput is the sum of the replicas' rates."""
    import multiprocessing as mp
    cores = cores or _host_cores()
    with mp.get_context("spawn").Pool(cores) as pool:
        res = pool.map(_oracle_sample, [(nx, target_s, i) for i in range(cores)])
    value = sum(w / t for w, t in res)
    steps = sum(w for w, _ in res) // (nx * nx * 25)
    return {"value": value, "unit": "DOF-updates/s", "cores": cores, "kind": "oracle",
            "sample": "%d concurrent replicas (one per host core) of %dx%d elements of the same "
                      "workload recipe, %d oracle steps in total, >= %.0f s each"
                      % (cores, nx, nx, steps, target_s)}


def _oracle_one_step(job):
    nx, seed = job
    return _oracle_sample((nx, 0.0, seed))


def train_alpha_network(degree, stream, seeds=range(1000, 1008), nx=96, snaps=(0, 10, 40),
                        epochs=15, make=None, label=None):
    """Learned blending coefficient for this degree: network inputs and the
    indicator's raw alpha harvested along GPU runs of a workload recipe (by
    default the vortex-plus-Riemann recipe: shocks and smooth flow), then Adam
    on the GPU (cr_mlp_train)."""
    import torch
    from paper_2502_07517_gb300 import crkfr
    if make is None:
        make = lambda seed: wl.euler2d_vortex_riemann(nx=nx, degree=degree, seed=seed)
        label = "vortex + planar Riemann jump, %dx%d, N=%d" % (nx, nx, degree)
    X, T = [], []
    for seed in seeds:
        prob, u = make(seed)
        ctx = crkfr.cr_init_mesh(crkfr.desc_from_problem(prob, stream=stream))
        crkfr.cr_set_state(ctx, u)
        done = 0
        for s in snaps:
            if s > done:
                try:
                    crkfr.cr_step(ctx, s - done, 1e300)
                except crkfr.CrError:  # data that reach an inadmissible state: stop harvesting
                    break
                done = s
            f, a = crkfr.cr_get_features(ctx, u.shape[1], u.shape[2])
            X.append(f)
            T.append(a)
        crkfr.cr_destroy(ctx)
    X, T = np.concatenate(X), np.concatenate(T).astype(np.float32)
    nin = X.shape[1]
    rng = np.random.default_rng(0)
    p = torch.from_numpy(rng.normal(0.0, 0.2, crkfr.cr_mlp_param_count(nin)).astype(np.float32)).cuda()
    Xd, Td = torch.from_numpy(X).cuda(), torch.from_numpy(T).cuda()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    crkfr.cr_mlp_train(nin, p, Xd, Td, batch=512, epochs=epochs, lr=3e-3, seed=1)
    train_s = time.perf_counter() - t0
    g, loss = torch.empty_like(p), torch.empty(1, device="cuda")
    crkfr.cr_mlp_grad(nin, p, Xd, Td, g, loss)
    params = p.cpu().numpy()
    # served by the fused inference kernel on a held-out seed: |alpha_net - alpha_indicator|
    prob, u = make(max(seeds) + 1)
    ctx = crkfr.cr_init_mesh(crkfr.desc_from_problem(prob, stream=stream))
    crkfr.cr_set_state(ctx, u)
    crkfr.cr_step(ctx, 20, 1e300)
    _, a_ind = crkfr.cr_get_features(ctx, u.shape[1], u.shape[2])
    ctx2 = crkfr.cr_init_mesh(crkfr.desc_from_problem(prob, stream=stream, alpha_mode=crkfr.CR_ALPHA_MLP))
    crkfr.cr_mlp_load(ctx2, params)
    crkfr.cr_set_state(ctx2, crkfr.cr_get_state(ctx, shape=u.shape))
    _, a_net = crkfr.cr_get_features(ctx2, u.shape[1], u.shape[2])
    info = {"samples": int(T.size), "inputs": nin, "epochs": epochs, "train_s": train_s,
            "cross_entropy": float(loss.item()), "target_mean": float(T.mean()),
            "heldout_mean_abs_alpha_err": float(np.abs(a_net - a_ind).mean()),
            "heldout_max_abs_alpha_err": float(np.abs(a_net - a_ind).max()),
            "data": "%s, %d seeds, steps %s" % (label, len(seeds), list(snaps))}
    return params, info


def alu_roofline(prob, nodes, kms, mixed, ms_per_step):
    """ALU roofline of the dominant kernel of a 2D Euler step: algorithmic
    flops (flop_model) per launch over the kernel's CUDA-event time, against
    the FP64 or FP32 peak; kms = per-kernel ms (k_local, k_face, k_update,
    k_finish_step)."""
    names = ["k_local", "k_face", "k_update", "k_finish_step"]
    dom = int(np.argmax(kms[:3]))
    flops = flop_model(2, prob["degree"], "euler2d")
    achieved = flops[dom] * nodes / (kms[dom] * 1e-3) / 1e12
    peak = PEAK_FP32_TFLOPS if mixed else PEAK_FP64_TFLOPS
    mode = "fp32" if mixed else "fp64"
    ne = nodes // (prob["degree"] + 1) ** 2
    return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak, "kernel": names[dom],
            "traffic": (NCU_TRAFFIC_PER_ELEMENT[(mode, names[dom])] * ne
                        if (mode, names[dom]) in NCU_TRAFFIC_PER_ELEMENT else None),
            "peak_source": "derived: 152 SMs x %s FMA lanes x 2 x 2070 MHz"
                           % ("128 FP32" if mixed else "2 FP64"),
            "algorithmic_flops_per_point": flops[dom],
            "kernel_ms": {nm: float(x) for nm, x in zip(names, kms)},
            "step_tflops": sum(flops) * nodes / (ms_per_step * 1e-3) / 1e12}


def timed_steps(ctx, steps, warmup, stream):
    import torch
    from paper_2502_07517_gb300 import crkfr
    crkfr.cr_step_async(ctx, warmup, 1e300)
    crkfr.cr_sync(ctx)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    crkfr.cr_step_async(ctx, steps, 1e300)
    e1.record(stream)
    torch.cuda.synchronize()
    crkfr.cr_sync(ctx)
    return e0.elapsed_time(e1) / steps


def l1_rel(g, ref):
    return [float(np.abs(g[v] - ref[v]).sum() / max(np.abs(ref[v]).sum(), 1e-300))
            for v in range(ref.shape[0])]


def phys_flux(prob, u, direction):
    """Physical flux of the conserved state u [M][Ne][Np] (Euler, ten-moment):
    only used to scale differences, never on the step's path."""
    rho = u[0]
    if prob["equation"] == "euler":
        g1 = prob["gamma"] - 1.0
        if prob["dim"] == 1:
            v = u[1] / rho
            p = g1 * (u[2] - 0.5 * u[1] * v)
            return np.stack([u[1], u[1] * v + p, (u[2] + p) * v])
        v1, v2 = u[1] / rho, u[2] / rho
        p = g1 * (u[3] - 0.5 * (u[1] * v1 + u[2] * v2))
        vn = v1 if direction == 0 else v2
        return np.stack([u[1 + direction], u[1] * vn + (p if direction == 0 else 0.0),
                         u[2] * vn + (p if direction == 1 else 0.0), (u[3] + p) * vn])
    v1, v2 = u[1] / rho, u[2] / rho
    p11, p12, p22 = 2 * u[3] - u[1] * v1, 2 * u[4] - u[1] * v2, 2 * u[5] - u[2] * v2
    if direction == 0:
        return np.stack([u[1], p11 + u[1] * v1, p12 + u[1] * v2, (u[3] + p11) * v1,
                         u[4] * v1 + 0.5 * (p11 * v2 + p12 * v1), u[5] * v1 + p12 * v2])
    return np.stack([u[2], p12 + u[1] * v2, p22 + u[2] * v2, u[3] * v2 + p12 * v1,
                     u[4] * v2 + 0.5 * (p12 * v2 + p22 * v1), (u[5] + p22) * v2])


def l1_flux_scaled(prob, g, ref, steps, dt):
    """Per variable: mean |g - ref| over the points divided by the larger of
    the variable's mean magnitude and its flux increment over the run,
    steps dt (max|f_v|/dx + max|g_v|/dy).  A variable that starts at zero and
    moves only through O(1) fluxes (a transverse momentum) is then measured
    against the size of what moves it, as the parity tests do."""
    dx = (prob["x1"] - prob["x0"]) / prob["nx"]
    inc = np.abs(phys_flux(prob, ref, 0)).max(axis=(1, 2)) / dx
    if prob["dim"] == 2:
        inc = inc + np.abs(phys_flux(prob, ref, 1)).max(axis=(1, 2)) / ((prob["y1"] - prob["y0"]) / prob["ny"])
    inc = inc * steps * dt
    return [float(np.abs(g[v] - ref[v]).mean() / max(np.abs(ref[v]).mean(), inc[v], 1e-300))
            for v in range(ref.shape[0])]


def alpha_agreement(prob, state, params, stream):
    """Raw blending coefficients of the network and of the indicator on the
    same state (FP64 contexts): the fraction of elements where they differ by
    more than 0.1, the largest difference, and the fraction of elements where
    the indicator is active (alpha > 0)."""
    from paper_2502_07517_gb300 import crkfr
    ne, npn = state.shape[1], state.shape[2]
    out = {}
    for name, mode in (("indicator", crkfr.CR_ALPHA_INDICATOR), ("network", crkfr.CR_ALPHA_MLP)):
        c = crkfr.cr_init_mesh(crkfr.desc_from_problem(prob, alpha_mode=mode, stream=stream))
        if mode == crkfr.CR_ALPHA_MLP:
            crkfr.cr_mlp_load(c, params)
        crkfr.cr_set_state(c, state)
        out[name] = crkfr.cr_get_features(c, ne, npn)[1]
        crkfr.cr_destroy(c)
    d = np.abs(out["network"] - out["indicator"])
    return {"elements": int(ne), "frac_disagree_gt_0.1": float((d > 0.1).mean()),
            "max_abs_diff": float(d.max()), "mean_abs_diff": float(d.mean()),
            "frac_indicator_active": float((out["indicator"] > 0).mean()),
            "frac_network_active": float((out["network"] > 0).mean())}


def fp32_variants(prob, u, ctx64, steps, warmup, stream, fp64_ms):
    """FP32 bulk with the indicator's alpha and with the learned alpha: device
    time per step on the same workload, and the normalised L1 difference per
    variable from the FP64 path (parity-checked against the FP64 oracle) after
    the same number of steps at the same fixed dt."""
    from paper_2502_07517_gb300 import crkfr
    params, train = train_alpha_network(prob["degree"], stream.cuda_stream)
    nodes = u.shape[1] * u.shape[2]
    crkfr.cr_set_state(ctx64, u)
    dt0 = crkfr.cr_next_dt(ctx64)
    crkfr.cr_step(ctx64, steps, 1e300, dt0)
    ref = crkfr.cr_get_state(ctx64, shape=u.shape)
    out = {"alpha_network": train, "l1_reference": "FP64 path after %d steps at dt %.6g" % (steps, dt0)}
    for name, mode in (("fp32_indicator", crkfr.CR_ALPHA_INDICATOR),
                       ("fp32_learned_alpha", crkfr.CR_ALPHA_MLP)):
        d = crkfr.desc_from_problem(prob, precision=crkfr.CR_FP32_BULK, alpha_mode=mode,
                                    stream=stream.cuda_stream)
        ctx = crkfr.cr_init_mesh(d)
        if mode == crkfr.CR_ALPHA_MLP:
            crkfr.cr_mlp_load(ctx, params)
        crkfr.cr_set_state(ctx, u)
        ms = timed_steps(ctx, steps, warmup, stream)
        crkfr.cr_set_state(ctx, u)
        crkfr.cr_step(ctx, steps, 1e300, dt0)
        g = crkfr.cr_get_state(ctx, shape=u.shape)
        a = crkfr.cr_get_alpha(ctx, u.shape[1])
        crkfr.cr_set_state(ctx, u)
        kms = crkfr.cr_profile_steps(ctx, steps, 1e300) / steps
        out[name] = {"value": nodes / (ms * 1e-3), "unit": "DOF-updates/s", "ms_per_step": ms,
                     "speedup_vs_fp64": fp64_ms / ms, "l1_rel_vs_fp64": l1_rel(g, ref),
                     "l1_flux_scaled_vs_fp64": l1_flux_scaled(prob, g, ref, steps, dt0),
                     "alpha_mean": float(a.mean()), "alpha_max": float(a.max()),
                     "roofline": alu_roofline(prob, nodes, kms, True, ms)}
        crkfr.cr_destroy(ctx)
    out["alpha_agreement_after_run"] = alpha_agreement(prob, ref, params, stream.cuda_stream)
    return out


def config_legs(steps, warmup):
    """The other workloads: 1D linear advection to t = 1 (error against the
    exact solution), 1D Euler Riemann problems (4000 elements, N = 4), 2D Euler
    in a box closed by solid walls (256x256, N = 4) and 2D ten-moment with the
    Gaussian source (256x256, N = 3), each in FP64 (plain,
    indicator alpha) and FP32 bulk with the learned alpha (a network trained
    for that workload on the GPU): device time per step, DOF-updates/s and the
    normalised L1 difference from the FP64 path after the same steps at the
    same fixed dt."""
    import torch
    from paper_2502_07517_gb300 import crkfr
    stream = torch.cuda.Stream()
    sp = stream.cuda_stream
    out = {}
    # linear advection, N = 3, 64 elements, CFL step to t = 1
    prob, u = wl.linadv_sine(nx=64, degree=3, t_final=1.0)
    ctx = crkfr.cr_init_mesh(crkfr.desc_from_problem(prob, stream=sp))
    crkfr.cr_set_state(ctx, u)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    t, n = crkfr.cr_step(ctx, 10 ** 6, 1.0)
    wall = time.perf_counter() - t0
    g = crkfr.cr_get_state(ctx, shape=u.shape)
    x, _ = wl.node_coords(prob)
    _, w = wl.gl_nodes01(3)
    out["linadv1d_sine_64_N3"] = {
        "steps_to_t1": n, "t": t, "wall_s": wall, "value": u.size * n / wall, "unit": "DOF-updates/s",
        "l1_error_vs_exact": float((np.abs(g[0] - np.sin(2 * np.pi * (x - 1.0))) * w).sum() / 64),
        "note": "256 DOF: launch-bound; the value is whole-run throughput including the host loop"}

    def leg(name, prob, u, make, nin_label, seeds, snaps):
        nodes = u.shape[1] * u.shape[2]
        c64 = crkfr.cr_init_mesh(crkfr.desc_from_problem(prob, stream=sp))
        crkfr.cr_set_state(c64, u)
        ms64 = timed_steps(c64, steps, warmup, stream)
        crkfr.cr_set_state(c64, u)
        dt0 = crkfr.cr_next_dt(c64)
        crkfr.cr_step(c64, steps, 1e300, dt0)
        ref = crkfr.cr_get_state(c64, shape=u.shape)
        params, info = train_alpha_network(prob["degree"], sp, seeds=seeds, snaps=snaps, make=make,
                                           label=nin_label)
        out[name] = {"dofs": nodes, "steps": steps, "dt": dt0,
                     "fp64": {"value": nodes / (ms64 * 1e-3), "ms_per_step": ms64},
                     "alpha_network": info, "unit": "DOF-updates/s",
                     "l1_reference": "FP64 path (indicator alpha) after the same steps at the same dt"}
        for label, mode in (("fp32_indicator", crkfr.CR_ALPHA_INDICATOR),
                            ("fp32_learned_alpha", crkfr.CR_ALPHA_MLP)):
            c32 = crkfr.cr_init_mesh(crkfr.desc_from_problem(prob, precision=crkfr.CR_FP32_BULK,
                                                             alpha_mode=mode, stream=sp))
            if mode == crkfr.CR_ALPHA_MLP:
                crkfr.cr_mlp_load(c32, params)
            crkfr.cr_set_state(c32, u)
            ms32 = timed_steps(c32, steps, warmup, stream)
            crkfr.cr_set_state(c32, u)
            crkfr.cr_step(c32, steps, 1e300, dt0)
            g = crkfr.cr_get_state(c32, shape=u.shape)
            a = crkfr.cr_get_alpha(c32, u.shape[1])
            out[name][label] = {"value": nodes / (ms32 * 1e-3), "ms_per_step": ms32,
                                "speedup_vs_fp64": ms64 / ms32, "l1_rel_vs_fp64": l1_rel(g, ref),
                                "l1_flux_scaled_vs_fp64": l1_flux_scaled(prob, g, ref, steps, dt0),
                                "alpha_mean": float(a.mean()), "alpha_frac_nonzero": float((a > 0).mean())}
            crkfr.cr_destroy(c32)
        li, ll = out[name]["fp32_indicator"], out[name]["fp32_learned_alpha"]
        out[name]["learned_vs_indicator"] = {
            "time_ratio": ll["ms_per_step"] / li["ms_per_step"],
            "l1_flux_scaled_ratio_max_over_vars": max(
                a / max(b, 1e-300) for a, b in zip(ll["l1_flux_scaled_vs_fp64"], li["l1_flux_scaled_vs_fp64"])),
            "alpha_agreement_on_initial_state": alpha_agreement(prob, u, params, sp),
            "alpha_agreement_after_run": alpha_agreement(prob, ref, params, sp)}
        crkfr.cr_destroy(c64)

    prob, u = wl.euler1d_riemann(nx=4000, degree=4, seed=0)
    leg("euler1d_riemann_4000_N4", prob, u,
        lambda seed: wl.euler1d_riemann(nx=4000, degree=4, seed=seed),
        "1D Euler Riemann problems, 4000 elements, N=4", range(1000, 1024), (0, 50, 200, 800))
    prob, u = wl.euler2d_vortex_riemann(nx=256, degree=4, seed=0)
    box = lambda pr: dict(pr, bc_x="wall", bc_y="wall")
    leg("euler2d_closed_box_walls_256x256_N4", box(prob), u,
        lambda seed: (lambda pu: (box(pu[0]), pu[1]))(wl.euler2d_vortex_riemann(nx=96, degree=4, seed=seed)),
        "vortex + planar Riemann jump in a box closed by walls, 96x96, N=4", range(1000, 1008),
        (0, 10, 40))
    # dissipation models and central fluxes of Sec. 3.1 on the 2D Euler recipe (FP64)
    prob, u = wl.euler2d_vortex(nx=256, degree=4, seed=0)
    var = {}
    for name, diss, cen in (("D2-EA", 0, 0), ("D1-EA", 1, 0), ("DCSX-EA", 2, 0), ("D2-AE", 0, 1),
                            ("DCSX-AE", 2, 1)):
        c = crkfr.cr_init_mesh(crkfr.desc_from_problem(prob, stream=sp, dissipation=diss, central=cen))
        crkfr.cr_set_state(c, u)
        ms = timed_steps(c, steps, warmup, stream)
        var[name] = {"ms_per_step": ms, "value": u.shape[1] * u.shape[2] / (ms * 1e-3)}
        crkfr.cr_destroy(c)
    out["euler2d_vortex_256x256_N4_dissipation_central"] = {"unit": "DOF-updates/s", "fp64": var}
    prob, u = wl.tenmoment2d_voronoi(nx=256, degree=3, seed=0)
    leg("tenmoment2d_voronoi_256x256_N3", prob, u,
        lambda seed: wl.tenmoment2d_voronoi(nx=128, degree=3, seed=seed),
        "ten-moment Voronoi states with source, 128x128, N=3", range(1000, 1020), (0, 5, 20))
    out.update(widened_legs(steps, warmup, stream))
    return out


def widened_legs(steps, warmup, stream):
    """Workloads of the further rows: the Rayleigh-Taylor instability (walls,
    given-state boundaries, gravity; 64x256, N = 3), the periodic 2D Sedov
    blast (64x64, N = 3) and the 1D Sedov blast between walls (201, N = 3),
    per step in FP64 and FP32 bulk (indicator alpha, normalised L1 from FP64
    after the same steps at the same dt); Gauss-Lobatto points (scaling
    limiter only) against Gauss-Legendre points on the 2D Euler recipe
    (256x256, N = 4, FP64); Burgers (Sec. 5.1, 128 elements, N = 3, to
    t = 2) with the EA and AE fluxes on both point sets, and variable
    advection (a = x^2, 128 elements, N = 3, to t = 1) with EA and AE: whole-run
    time and L2 error against the exact solution."""
    import torch
    from paper_2502_07517_gb300 import crkfr
    sp = stream.cuda_stream
    out = {}

    def per_step(prob, u, precision=crkfr.CR_FP64, dt=None, **over):
        c = crkfr.cr_init_mesh(crkfr.desc_from_problem(prob, precision=precision, stream=sp, **over))
        crkfr.cr_set_state(c, u)
        ms = timed_steps(c, steps, warmup, stream)
        crkfr.cr_set_state(c, u)
        dt0 = crkfr.cr_next_dt(c) if dt is None else dt
        crkfr.cr_step(c, steps, 1e300, dt0)
        g = crkfr.cr_get_state(c, shape=u.shape)
        crkfr.cr_destroy(c)
        return ms, g, dt0

    for name, (prob, u) in (("rayleigh_taylor_64x256_N3", wl.rayleigh_taylor()),
                            ("sedov2d_periodic_64x64_N3", wl.sedov2d_periodic()),
                            ("sedov1d_walls_201_N3", wl.sedov1d())):
        nodes = u.shape[1] * u.shape[2]
        ms64, ref, dt0 = per_step(prob, u)
        ms32, g, _ = per_step(prob, u, crkfr.CR_FP32_BULK, dt=dt0)
        out[name] = {"dofs": nodes, "steps": steps, "unit": "DOF-updates/s",
                     "fp64": {"ms_per_step": ms64, "value": nodes / (ms64 * 1e-3)},
                     "fp32_indicator": {"ms_per_step": ms32, "value": nodes / (ms32 * 1e-3),
                                        "speedup_vs_fp64": ms64 / ms32, "l1_rel_vs_fp64": l1_rel(g, ref),
                                        "l1_flux_scaled_vs_fp64": l1_flux_scaled(prob, g, ref, steps, dt0)}}
    prob, u = wl.euler2d_vortex(nx=256, degree=4, seed=0, limiter=("scaling", "traces"))
    pts = {}
    for label in ("gl", "gll"):
        pr = dict(prob, points=label)
        x, y = wl.node_coords(pr)
        rho, v1, v2, p = wl.isentropic_vortex(x, y, pr["gamma"])
        uu = wl.euler_conservative(rho, v1, v2, p, pr["gamma"], 2)
        ms, _, dt0 = per_step(pr, uu)
        pts[label] = {"ms_per_step": ms, "value": uu.shape[1] * uu.shape[2] / (ms * 1e-3), "dt": dt0}
    out["euler2d_vortex_256x256_N4_points"] = {
        "unit": "DOF-updates/s", "limiters": "scaling", "fp64": pts,
        "note": "the Gauss-Lobatto scheme takes a larger step (CFL 0.104 against 0.070)"}
    burg = {}
    for label in ("gl", "gll"):
        for cname, cen in (("EA", crkfr.CR_CENTRAL_EA), ("AE", crkfr.CR_CENTRAL_AE)):
            prob, u = wl.burgers_sine(nx=128, degree=3, points=label)
            c = crkfr.cr_init_mesh(crkfr.desc_from_problem(prob, stream=sp, central=cen))
            crkfr.cr_set_state(c, u)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            t, n = crkfr.cr_step(c, 10 ** 6, 2.0)
            wall = time.perf_counter() - t0
            g = crkfr.cr_get_state(c, shape=u.shape)
            crkfr.cr_destroy(c)
            x, _ = wl.node_coords(prob)
            _, w = wl.nodes01(prob)
            ex = 0.2 * np.sin(x)
            for _ in range(100):
                ex = ex - (ex - 0.2 * np.sin(x - 2.0 * ex)) / (1.0 + 0.4 * np.cos(x - 2.0 * ex))
            err = float(np.sqrt(((g[0] - ex) ** 2 * w * 2 * np.pi / 128).sum()))
            burg["%s-%s" % (label, cname)] = {"steps": n, "wall_s": wall, "l2_error_vs_exact": err,
                                             "value": u.size * n / wall}
    out["burgers1d_sine_128_N3_t2"] = {"unit": "DOF-updates/s", "fp64": burg,
                                       "note": "512 DOF: launch-bound whole runs incl. the host loop"}
    var = {}
    for cname, cen in (("EA", crkfr.CR_CENTRAL_EA), ("AE", crkfr.CR_CENTRAL_AE)):
        prob, u = wl.varadv_x2(nx=128, degree=3)
        c = crkfr.cr_init_mesh(crkfr.desc_from_problem(prob, stream=sp, central=cen))
        crkfr.cr_set_state(c, u)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        t, n = crkfr.cr_step(c, 10 ** 6, 1.0)
        wall = time.perf_counter() - t0
        g = crkfr.cr_get_state(c, shape=u.shape)
        crkfr.cr_destroy(c)
        x, _ = wl.node_coords(prob)
        _, w = wl.nodes01(prob)
        err = float(np.sqrt(((g[0] - wl.varadv_exact(x, 1.0)) ** 2 * w * 0.9 / 128).sum()))
        var[cname] = {"steps": n, "wall_s": wall, "l2_error_vs_exact": err, "value": u.size * n / wall}
    out["varadv1d_x2_128_N3_t1"] = {"unit": "DOF-updates/s", "fp64": var,
                                    "note": "a(x) = x^2, exact inflow; 512 DOF: launch-bound whole runs"}
    return out


def _finite_min(xs):
    """Smallest finite value, or None (JSON has no NaN)."""
    xs = [float(x) for x in xs if np.isfinite(x)]
    return min(xs) if xs else None


def ensemble_leg(steps, warmup, nprob=96, seed=0, config=None, learned=True, nmin=32, nmax=512):
    """Batched ensemble: nprob independent 2D Euler problems (sides uniform in
    32..512, N in {3, 4}, vortex plus planar Riemann jump), FP32 bulk with the
    learned alpha, advanced by one batch (autotuned threads per block and
    mode, CUDA graphs); against the same problems stepped one at a time."""
    import torch
    from paper_2502_07517_gb300 import crkfr
    t0 = time.perf_counter()
    probs = wl.euler2d_ensemble(nprob=nprob, seed=seed, nmin=nmin, nmax=nmax)
    gen_s = time.perf_counter() - t0
    stream = torch.cuda.Stream()
    nets = {N: train_alpha_network(N, stream.cuda_stream) for N in (3, 4)} if learned else None
    ctxs = []
    for prob, u in probs:
        d = crkfr.desc_from_problem(prob, precision=crkfr.CR_FP32_BULK,
                                    alpha_mode=crkfr.CR_ALPHA_MLP if learned else crkfr.CR_ALPHA_INDICATOR,
                                    stream=stream.cuda_stream)
        c = crkfr.cr_init_mesh(d)
        if learned:
            crkfr.cr_mlp_load(c, nets[prob["degree"]][0])
        crkfr.cr_set_state(c, u)
        ctxs.append(c)
    nodes = sum(u.shape[1] * u.shape[2] for _, u in probs)
    b = crkfr.cr_batch_init(ctxs)
    if config:  # "threads/mode[/tiles]", e.g. "256/fused/2": fixed instead of tuned
        parts = config.split("/")
        threads, mode = int(parts[0]), int(parts[1] == "fused")
        tiles = int(parts[2]) if len(parts) > 2 else 1
        crkfr.cr_batch_config(b, threads, mode, tiles)
        cand = np.full(len(crkfr.BATCH_CANDIDATES), np.nan)
    else:
        threads, mode, tiles, cand = crkfr.cr_batch_autotune(b, 2)

    def reset():
        for (prob, u), c in zip(probs, ctxs):
            crkfr.cr_set_state(c, u)
        torch.cuda.synchronize()

    reset()
    crkfr.cr_batch_step(b, warmup)
    reset()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    crkfr.cr_batch_step_async(b, steps)
    e1.record(stream)
    crkfr.cr_batch_sync(b)
    batch_ms = e0.elapsed_time(e1)
    # the same problems, one problem's steps at a time (its own launches, then the next)
    reset()
    for c in ctxs:
        crkfr.cr_step(c, warmup, 1e300)
    reset()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for c in ctxs:
        crkfr.cr_step(c, steps, 1e300)
    seq_s = time.perf_counter() - t0
    a = np.concatenate([crkfr.cr_get_alpha(c, u.shape[1]) for (prob, u), c in zip(probs, ctxs)])
    names = ["%d/%s/%d" % (t, "fused" if m else "phases", k) for t, m, k in crkfr.BATCH_CANDIDATES]
    return {"problems": nprob, "sides": [nmin, nmax],
            "elements": int(sum(u.shape[1] for _, u in probs)), "dofs": int(nodes),
            "degrees": {"3": sum(p["degree"] == 3 for p, _ in probs), "4": sum(p["degree"] == 4 for p, _ in probs)},
            "steps": steps, "value": nodes * steps / (batch_ms * 1e-3), "unit": "DOF-updates/s",
            "ms_per_step": batch_ms / steps,
            "sequential_value": nodes * steps / seq_s, "sequential_ms_per_step": seq_s * 1e3 / steps,
            "speedup_vs_sequential": seq_s * 1e3 / batch_ms,
            "autotune": {"chosen": "%d/%s/%d" % (threads, "fused" if mode else "phases", tiles),
                         "candidates": "threads/mode/tiles: threads per block (elements per tile = threads / "
                                       "(N+1)^2); fused: 8 x tiles tiles per queue claim",
                         "best_phases_ms": _finite_min(x for (t, m, k), x in zip(crkfr.BATCH_CANDIDATES, cand)
                                                       if m == crkfr.CR_BATCH_PHASES),
                         "best_fused_ms": _finite_min(x for (t, m, k), x in zip(crkfr.BATCH_CANDIDATES, cand)
                                                      if m == crkfr.CR_BATCH_FUSED),
                         "ms_per_step": {nm: (float(x) if np.isfinite(x) else None) for nm, x in zip(names, cand)}},
            "alpha_networks": {str(N): nets[N][1] for N in (3, 4)} if learned else None,
            "alpha_mean": float(a.mean()), "generate_s": gen_s,
            "precision": "FP32 bulk + FP64 means/limiter theta, " +
                         ("learned alpha (BF16 weights)" if learned else "indicator alpha")}


def run_reference(args):
    """The reference arm: the FP64 oracle as it stands on the host cores (this
    paper has no reference implementation to install).  Each bench step is one
    oracle step of a 128x128-element sample of the workload recipe on every
    core at once; throughput = all cores' point updates / the step's wall time."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import multiprocessing as mp
    cores, nx = _host_cores(), 128
    times = []
    with mp.get_context("spawn").Pool(cores) as pool:
        pool.map(_oracle_sample, [(nx, -1.0, i) for i in range(cores)], chunksize=1)  # load, generate
        for it in range(args.warmup + args.steps):
            t0 = time.perf_counter()
            res = pool.map(_oracle_one_step, [(nx, i) for i in range(cores)])
            if it >= args.warmup:
                times.append(time.perf_counter() - t0)
    points = sum(w for w, _ in res)
    val = points / statistics.median(times)
    line = {"impl": "reference", "metric": "DOF-updates/s", "value": val, "unit": "DOF-updates/s",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": statistics.median(times) * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD["name"],
                       "sample": "%d concurrent %dx%d-element samples per step" % (cores, nx, nx)},
            "cpu_baseline": {"value": val, "unit": "DOF-updates/s", "cores": cores, "kind": "oracle",
                             "sample": "one oracle step of a %dx%d-element sample of the workload "
                                       "recipe on each of %d host cores per bench step" % (nx, nx, cores)},
            "e2e": {"value": val, "unit": "DOF-updates/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def run_ours(args):
    import torch
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as tdist
        tdist.init_process_group("nccl")
    from paper_2502_07517_gb300 import build as lib_build
    if rank == 0:
        lib_build.build()
    if world > 1:
        tdist.barrier()
    from paper_2502_07517_gb300 import crkfr

    mixed = args.mode == "fp32"
    prob, u = make_workload(seed=rank, nx=args.nx, degree=args.degree)
    M, ne, npn = u.shape
    nodes = ne * npn
    stream = torch.cuda.Stream()
    desc = crkfr.desc_from_problem(prob, precision=crkfr.CR_FP32_BULK if mixed else crkfr.CR_FP64,
                                   stream=stream.cuda_stream)
    ctx = crkfr.cr_init_mesh(desc)
    crkfr.cr_set_state(ctx, u)
    launches = crkfr.cr_launches_per_step(ctx)
    crkfr.cr_step_async(ctx, args.warmup, 1e300)
    crkfr.cr_sync(ctx)

    # ---- timed region: K steps, CUDA events on the library's stream ----
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if world > 1:
        tdist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        e0.record(stream)
        crkfr.cr_step_async(ctx, args.steps, 1e300)
        e1.record(stream)
        torch.cuda.synchronize()
    t_s, n_s = crkfr.cr_sync(ctx)
    if world > 1:
        tdist.barrier()
    ms = e0.elapsed_time(e1)
    ms, value = aggregate_timing(ms, nodes, args.steps, world, tdist if world > 1 else None, "cuda")
    ms_per_step = ms / args.steps

    # ---- per-kernel device times (same workload, every kernel between events) ----
    kms = crkfr.cr_profile_steps(ctx, args.steps, 1e300) / args.steps
    roofline = alu_roofline(prob, nodes, kms, mixed, ms_per_step)

    # ---- HBM view: the method's own bytes (read u^n, write u^{n+1}) per step ----
    state_bytes = u.size * (4 if mixed else 8) + (2 * M * ne * 8 if mixed else 0)
    hbm_peak = json.load(open(MEASURED_PEAKS))["hbm_gbs"] if os.path.exists(MEASURED_PEAKS) else 6800.0
    hbm = {"algorithmic_bytes_per_step": 2 * state_bytes,
           "achieved_GBs": 2 * state_bytes / (ms_per_step * 1e-3) / 1e9, "peak_GBs": hbm_peak}
    hbm["frac"] = hbm["achieved_GBs"] / hbm_peak

    variants = None
    if not mixed and not args.quick and not args.no_variants:
        variants = fp32_variants(prob, u, ctx, args.steps, args.warmup, stream, ms_per_step)
    ensemble = None
    if not args.quick and not args.no_ensemble:
        ensemble = ensemble_leg(args.steps, args.warmup, seed=rank)
        # many small meshes (sides 32..128): where one launch per problem is launch bound
        ensemble["small_meshes"] = ensemble_leg(args.steps, args.warmup, seed=rank, nmin=32, nmax=128)
    configs = None
    if not args.quick and not args.no_configs:
        configs = config_legs(args.steps, args.warmup)

    # ---- end to end through the public API with host buffers ----
    if args.quick:
        print(json.dumps({"quick": True, "mode": args.mode, "nx": args.nx, "ms_per_step": ms_per_step,
                          "value": value, "roofline": roofline}))
        return
    host_in = torch.from_numpy(u).pin_memory()
    host_out = torch.empty(u.shape, dtype=torch.float64).pin_memory()
    e2e_steps = max(1, min(args.steps, 5))
    parts = np.zeros(2)

    def e2e_step():
        # cr_set_state reads the pinned input in its checking kernel; cr_step_get's
        # update kernel writes the new state into the pinned output while it runs
        ta = time.perf_counter()
        crkfr.lib().cr_set_state(ctx.handle, host_in.data_ptr(), 0)
        tb = time.perf_counter()
        crkfr.cr_step_get(ctx, 1, 1e300, host_out)
        return np.array([tb - ta, time.perf_counter() - tb])

    e2e_step()  # untimed: first use of the pinned buffers
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        parts += e2e_step()
    e2e_s = (time.perf_counter() - t0) / e2e_steps
    nbytes = u.size * 8
    e2e = {"value": world * nodes / e2e_s, "unit": "DOF-updates/s", "h2d_bytes_per_step": nbytes,
           "d2h_bytes_per_step": nbytes, "ms_per_step": e2e_s * 1e3,
           "ms_set_and_step_get": [float(x) for x in parts / e2e_steps * 1e3]}

    if rank != 0:
        if world > 1:
            tdist.barrier()
            tdist.destroy_process_group()
        return
    cb = cpu_baseline() if world == 1 else None
    clocks = clk.summary()
    line = {
        "metric": "DOF-updates/s", "value": value, "unit": "DOF-updates/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32+f64" if mixed else "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD["name"] if (args.nx, args.degree) == (WORKLOAD["nx"], WORKLOAD["degree"])
                   else "euler2d_vortex_%dx%d_N%d" % (args.nx, args.nx, args.degree),
                   "elements": ne, "points_per_element": npn,
                   "variables": M, "mode": args.mode,
                   "limiters": "blend+MUSCL-Hancock+flux+scaling",
                   "l2": "inputs larger than L2 (state %.0f MB)" % (u.size * (4 if mixed else 8) / 1e6),
                   "parallelism": "replicas" if world > 1 else "single"},
        "roofline": roofline, "hbm_roofline": hbm, "variants": variants, "ensemble": ensemble,
        "other_workloads": configs,
        "cpu_baseline": cb, "e2e": e2e, "clocks": clocks,
        "gpu_launches": launches * args.steps, "t_reached": t_s, "steps_run": n_s,
    }
    print(json.dumps(line))
    if world > 1:
        tdist.barrier()
        tdist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--mode", choices=("fp64", "fp32"), default="fp64")
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--nx", type=int, default=WORKLOAD["nx"],
                    help="elements per direction (smaller meshes of the same recipe for profiling)")
    ap.add_argument("--no-ensemble", action="store_true",
                    help="skip the batched-ensemble leg (96 problems in one batch)")
    ap.add_argument("--ensemble-only", action="store_true",
                    help="run only the batched-ensemble leg and print it")
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the legs of the other workloads (1D linear advection, 1D Euler, ten-moment)")
    ap.add_argument("--configs-only", action="store_true", help="run only those legs and print them")
    ap.add_argument("--widened-only", action="store_true",
                    help="run only the legs of the further rows (boundaries, sources, points, Burgers)")
    ap.add_argument("--ens-problems", type=int, default=96, help="problems in the ensemble leg")
    ap.add_argument("--ens-config", default=None,
                    help="fixed batch configuration threads/mode[/tiles] (128|256 / phases|fused / 1|2|4) "
                         "instead of autotuning")
    ap.add_argument("--ens-indicator", action="store_true",
                    help="ensemble leg with the indicator's alpha (no network training)")
    ap.add_argument("--no-variants", action="store_true",
                    help="skip the FP32 bulk / learned-alpha comparison legs")
    ap.add_argument("--degree", type=int, default=WORKLOAD["degree"],
                    help="degree N of the same recipe (profiling; the bench workload is N = 4)")
    ap.add_argument("--quick", action="store_true",
                    help="device timing only (no CPU baseline, no end-to-end leg)")
    args = ap.parse_args()
    if args.configs_only:
        import torch
        from paper_2502_07517_gb300 import build as lib_build
        lib_build.build()
        torch.cuda.set_device(0)
        print(json.dumps(config_legs(args.steps, args.warmup)))
    elif args.widened_only:
        import torch
        from paper_2502_07517_gb300 import build as lib_build
        lib_build.build()
        torch.cuda.set_device(0)
        print(json.dumps(widened_legs(args.steps, args.warmup, torch.cuda.Stream())))
    elif args.ensemble_only:
        import torch
        from paper_2502_07517_gb300 import build as lib_build
        lib_build.build()
        torch.cuda.set_device(0)
        print(json.dumps(ensemble_leg(args.steps, args.warmup, nprob=args.ens_problems,
                                      config=args.ens_config, learned=not args.ens_indicator)))
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
