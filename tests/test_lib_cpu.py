"""CPU checks of the CUDA library: it loads without a GPU, exports every symbol
include/cr.h declares, and its host-only routines (no device work) agree with
the oracle's independently written ones."""
import os
import re

import numpy as np
import pytest

from paper_2502_07517_gb300 import build as lib_build
from paper_2502_07517_gb300 import crkfr
from paper_2502_07517_gb300 import workloads as wl

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def built():
    lib_build.build()
    return crkfr.lib()


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "cr.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(cr_[a-z_0-9]+)\s*\(", text)))


def test_exports_every_declared_symbol(built):
    syms = declared_symbols()
    assert len(syms) >= 14
    for s in syms:
        assert hasattr(built, s), s
    assert set(syms) == set(crkfr.SYMBOLS)


@pytest.mark.parametrize("N", [1, 2, 3, 4])
def test_library_cfl_matches_oracle(built, N):
    from oracle.cfl import cfl_number
    assert abs(crkfr.cr_cfl_number(N) - cfl_number(N)) < 1e-6


@pytest.mark.parametrize("N", [1, 2, 3, 4])
def test_library_tables_match_numpy(built, N):
    xi, w, D = crkfr.cr_reference_tables(N)
    x, ww = np.polynomial.legendre.leggauss(N + 1)
    np.testing.assert_allclose(xi, 0.5 * (x + 1), atol=1e-15)
    np.testing.assert_allclose(w, 0.5 * ww, atol=1e-15)
    for m in range(N + 1):
        np.testing.assert_allclose(D @ xi ** m, m * xi ** max(m - 1, 0) * (m > 0), atol=1e-12)


def test_invalid_descriptor_rejected(built):
    from paper_2502_07517_gb300 import workloads as wl
    prob, _ = wl.linadv_sine(nx=8, degree=3)
    d = crkfr.desc_from_problem(prob)
    d.degree = 7
    with pytest.raises(crkfr.CrError) as ei:
        crkfr.cr_workspace_bytes(d)
    assert ei.value.status == -1
    d.degree = 3
    assert crkfr.cr_workspace_bytes(d) > 0


def test_static_step_wrapper_refuses_bad_tensors(built):
    """The cr_step_static binding hands the library no pointer it cannot use:
    host tensors, a wrong dtype or size, or a non-contiguous layout are refused
    with CR_E_INVALID_ARG before the library is called."""
    import torch
    prob, u = wl.euler2d_vortex(nx=4, ny=3, degree=3, seed=0)
    d = crkfr.desc_from_problem(prob)
    good = torch.from_numpy(u)
    bad = [good, good.float(), good[:, :, :-1], good.transpose(1, 2), np.asarray(u)]
    for t in bad:
        with pytest.raises(crkfr.CrError) as ei:
            crkfr.cr_step_static(d, t, t, 1e-3)
        assert ei.value.status == -1
    assert crkfr._state_numel(d) == u.size
    prob1, u1 = wl.euler1d_riemann(nx=7, degree=4, seed=0)
    assert crkfr._state_numel(crkfr.desc_from_problem(prob1)) == u1.size
    prob2, u2 = wl.tenmoment2d_voronoi(nx=5, ny=4, degree=2, seed=0)
    assert crkfr._state_numel(crkfr.desc_from_problem(prob2)) == u2.size


def test_step_get_wrapper_refuses_bad_output(built):
    """The cr_step_get binding writes only into contiguous float64 host memory of
    the state's size: a wrong dtype or size, a non-contiguous array or tensor are
    refused with CR_E_INVALID_ARG before the library is called (the context is
    never touched, so a stand-in with the description serves)."""
    import torch

    class _Ctx:
        handle = None

    prob, u = wl.euler2d_vortex(nx=4, ny=3, degree=3, seed=0)
    ctx = _Ctx()
    ctx.desc = crkfr.desc_from_problem(prob)
    t = torch.from_numpy(u.copy())
    bad = [u.astype(np.float32), u[:, :, :-1].copy(), np.asfortranarray(u), u.reshape(-1)[::2],
           t.float(), t.transpose(1, 2), t[:, :, :-1]]
    for out in bad:
        with pytest.raises(crkfr.CrError) as ei:
            crkfr.cr_step_get(ctx, 1, 1.0, out)
        assert ei.value.status == -1


@pytest.mark.parametrize("N", [1, 2, 3, 4])
def test_library_cfl_for_dissipation_models_matches_oracle(N):
    from oracle.cfl import cfl_number
    assert abs(crkfr.cr_cfl_number_for(N, crkfr.CR_DISS_D1) - cfl_number(N, True)) < 1e-6
    assert crkfr.cr_cfl_number_for(N, crkfr.CR_DISS_DCSX) == crkfr.cr_cfl_number(N)
    assert crkfr.cr_cfl_number_for(N, crkfr.CR_DISS_D1) < crkfr.cr_cfl_number(N)


def _rejected(d):
    with pytest.raises(crkfr.CrError) as ei:
        crkfr.cr_workspace_bytes(d)
    return ei.value.status == -1


def test_boundary_and_source_descriptors_checked(built):
    """Host checks of the per-side boundaries, ghost states and sources (no
    device work): what is accepted and what is refused."""
    from paper_2502_07517_gb300 import workloads as wl
    prob, _ = wl.rayleigh_taylor(nx=8, ny=32)
    d = crkfr.desc_from_problem(prob)
    assert crkfr.cr_workspace_bytes(d) > 0
    d.bc_state[2][3] = 0.0                       # bottom ghost state: E = 0, p < 0
    assert _rejected(d)
    d = crkfr.desc_from_problem(prob)
    d.bc_state[3][0] = float("nan")
    assert _rejected(d)
    d = crkfr.desc_from_problem(prob)
    d.bc_side[0] = 5                             # unknown code
    assert _rejected(d)
    d = crkfr.desc_from_problem(prob)
    d.gravity[1] = float("inf")
    assert _rejected(d)
    d = crkfr.desc_from_problem(prob)
    d.bc_side[1] = crkfr.CR_BC_INFLOW            # x+ becomes inflow of the zero state
    assert _rejected(d)
    d.bc_state[1][0], d.bc_state[1][3] = 1.0, 2.0
    assert crkfr.cr_workspace_bytes(d) > 0
    # a periodic direction takes no per-side override
    pv, _ = wl.euler2d_vortex(nx=8, degree=3)
    d = crkfr.desc_from_problem(pv)
    d.bc_side[2] = crkfr.CR_BC_OUTFLOW
    assert _rejected(d)
    # gravity is an Euler source; walls stay Euler only, also per side
    pl, _ = wl.linadv_random(nx=8, degree=3, bc="outflow")
    d = crkfr.desc_from_problem(pl)
    d.source, d.gravity[0] = crkfr.CR_SRC_GRAVITY, 1.0
    assert _rejected(d)
    d = crkfr.desc_from_problem(pl)
    d.bc_side[1] = crkfr.CR_BC_WALL
    assert _rejected(d)
    d.bc_side[1] = crkfr.CR_BC_DIRICHLET          # a scalar ghost state needs only finiteness
    assert crkfr.cr_workspace_bytes(d) > 0


@pytest.mark.parametrize("N", [1, 2, 3, 4])
def test_gauss_lobatto_tables_and_cfl(built, N):
    """The library's Gauss-Lobatto tables against numpy's Legendre class, and
    its CFL numbers for both point sets against the oracle's analysis."""
    import oracle
    from oracle.cfl import cfl_number
    xi, w, D = crkfr.cr_reference_tables_points(N, crkfr.CR_POINTS_GLL)
    Leg = np.polynomial.legendre.Legendre
    inner = np.sort(Leg.basis(N).deriv().roots().real) if N > 1 else np.zeros(0)
    x = np.concatenate([[-1.0], inner, [1.0]])
    np.testing.assert_allclose(xi, 0.5 * (x + 1.0), rtol=0, atol=1e-15)
    np.testing.assert_allclose(w, 1.0 / (N * (N + 1) * Leg.basis(N)(x) ** 2), rtol=1e-14)
    for m in range(N + 1):
        np.testing.assert_allclose(D @ xi ** m, m * xi ** max(m - 1, 0) * (m > 0), atol=1e-12)
    g = crkfr.cr_reference_tables_points(N, crkfr.CR_POINTS_GL)
    np.testing.assert_array_equal(g[0], crkfr.cr_reference_tables(N)[0])
    for diss in (crkfr.CR_DISS_D2, crkfr.CR_DISS_D1):
        got = crkfr.cr_cfl_number_points(N, diss, crkfr.CR_POINTS_GLL)
        assert abs(got - cfl_number(N, diss == crkfr.CR_DISS_D1, points=oracle.POINTS_GLL)) < 1e-6


def test_gauss_lobatto_refusals(built):
    from paper_2502_07517_gb300 import workloads as wl
    prob, _ = wl.burgers_sine(nx=16, degree=3, points="gll")
    d = crkfr.desc_from_problem(prob)
    assert crkfr.cr_workspace_bytes(d) > 0
    for lim in (crkfr.CR_LIM_BLEND, crkfr.CR_LIM_MH, crkfr.CR_LIM_FLUX):
        d.limiter = lim
        assert _rejected(d)
    d.limiter = crkfr.CR_LIM_SCALING | crkfr.CR_LIM_TRACES
    assert crkfr.cr_workspace_bytes(d) > 0
    d.limiter, d.alpha_mode = 0, crkfr.CR_ALPHA_FIXED
    assert _rejected(d)
    d.alpha_mode, d.points = crkfr.CR_ALPHA_INDICATOR, 2
    assert _rejected(d)


def test_time_dependent_boundary_descriptors(built):
    from paper_2502_07517_gb300 import workloads as wl
    prob, _ = wl.varadv_x2(nx=8, degree=3)
    d = crkfr.desc_from_problem(prob)
    assert d.bc_time_terms == 16 and crkfr.cr_workspace_bytes(d) > 0
    d.bc_time_span[1] = d.bc_time_span[0]
    assert _rejected(d)
    d = crkfr.desc_from_problem(prob)
    d.bc_time_coef[0][3] = float("inf")
    assert _rejected(d)
    d = crkfr.desc_from_problem(prob)
    d.bc_time_terms = 17
    assert _rejected(d)
    d = crkfr.desc_from_problem(prob)
    d.adv_poly[2] = float("nan")
    assert _rejected(d)
    # time-dependent states are for scalar equations
    pe, _ = wl.euler1d_riemann(nx=8, degree=3)
    d = crkfr.desc_from_problem(pe)
    d.bc_time_terms, d.bc_time_span[1] = 4, 1.0
    assert _rejected(d)


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    """Without the compiled library every entry point raises: there is no
    fallback that computes anything elsewhere."""
    monkeypatch.setattr(crkfr, "_lib", None)
    monkeypatch.setattr(crkfr, "LIB_PATH", str(tmp_path / "libcrkfr.so"))
    with pytest.raises(RuntimeError, match="libcrkfr.so is missing"):
        crkfr.lib()
    with pytest.raises(RuntimeError, match="libcrkfr.so is missing"):
        crkfr.cr_cfl_number(3)
    prob, _ = wl.euler2d_vortex(nx=4, ny=4, degree=3)
    with pytest.raises(RuntimeError, match="libcrkfr.so is missing"):
        crkfr.cr_init_mesh(crkfr.desc_from_problem(prob))
