"""The library's smoothness indicator (Sec. 4, the Hennemann et al. form the
paper cites) against closed forms, independent of the oracle: meshes whose
elements hold an indicator variable made of chosen Legendre modes, so that the
energy ratio equals T(N) (1 + delta) through the top ratio, the next-to-top
ratio or both (1D and 2D, N = 2, 3, 4; scalar, Euler and ten-moment
variables).  The raw alpha the library computes (before the neighbour
smoothing) must be 1 / (1 + exp(-s delta)) in FP64 and in FP32 bulk."""
import numpy as np
import pytest

from paper_2502_07517_gb300 import crkfr
from paper_2502_07517_gb300 import workloads as wl
from tests.test_oracle_indicator import (DELTAS, _state, cases_1d, cases_2d, eps_1d, eps_2d,
                                         expected_alpha)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2502_07517_gb300 import build
    build.build()


def _mesh(equation, dim, N):
    """One element per (delta, case); returns the problem, the state and the
    expected raw alpha per element."""
    cols, want = [], []
    for delta in DELTAS:
        cs = cases_1d(N, delta) if dim == 1 else cases_2d(N, delta)
        for c in cs.values():
            eps = eps_1d(c, N) if dim == 1 else eps_2d(c, N)
            cols.append(_state(equation, dim, eps))
            want.append(expected_alpha(delta))
    u = np.stack(cols, axis=1)  # [M][Ne][Np]
    prob = wl.base_problem(dim=dim, nx=u.shape[1], ny=1, degree=N, equation=equation,
                           limiter=frozenset({"blend", "mh", "flux", "scaling"}))
    return prob, u, np.array(want)


FP32_BUILT = {("euler", 1, 4), ("euler", 2, 3), ("euler", 2, 4), ("tenmoment", 2, 3)}


@pytest.mark.parametrize("precision", [crkfr.CR_FP64, crkfr.CR_FP32_BULK], ids=["fp64", "fp32"])
@pytest.mark.parametrize("equation,dim,N", [("linadv", 1, 2), ("linadv", 1, 3), ("linadv", 1, 4),
                                            ("linadv", 2, 3), ("linadv", 2, 4), ("euler", 1, 4),
                                            ("euler", 2, 2), ("euler", 2, 3), ("euler", 2, 4),
                                            ("tenmoment", 2, 3)])
def test_raw_alpha_closed_form(equation, dim, N, precision):
    prob, u, want = _mesh(equation, dim, N)
    if precision == crkfr.CR_FP32_BULK and (equation, dim, N) not in FP32_BUILT:
        pytest.skip("FP32 bulk is not built for this equation and degree")
    ctx = crkfr.cr_init_mesh(crkfr.desc_from_problem(prob, precision=precision))
    crkfr.cr_set_state(ctx, u)
    _, a = crkfr.cr_get_features(ctx, u.shape[1], u.shape[2])
    # FP64: rounding only.  FP32 bulk: FP32 fluctuations about an FP64 mean; the
    # logistic's slope at E = T is s/(4T), about 2e3 per unit of E, so an FP32
    # rounding of E (~1e-9 here) moves alpha by a few 1e-6.
    tol = 1e-9 if precision == crkfr.CR_FP64 else 1e-4
    print("\nmax |alpha - closed form| = %.2e" % np.abs(a - want).max())
    np.testing.assert_allclose(a, want, rtol=0, atol=tol)
