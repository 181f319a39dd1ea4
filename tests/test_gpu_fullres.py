"""Full residual ||M - C U R||_F / ||M||_F on the tensor cores (stored FP32
M), against FP64 from the factors the GPU returned, and the error bar
against the FP64 oracle's own solution."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from tests._parity import error_ok, rel_fro_error

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1611_01391_gb300 as L  # noqa: E402

DEV = "cuda:0"


@pytest.fixture(scope="module")
def ctx():
    c = L.Context(0)
    yield c
    c.close()


def _solve_full(ctx, A, J0, k, l, sweeps):
    m, n = A.shape
    params, keep = L.make_params(k, l, sweeps, J0, full_residual=True)
    res = ctx.solve(L.make_source("dense", a=torch.from_numpy(A).to(DEV)), params, l, m, n,
                    want_strips=True, device=DEV)
    assert res.info.status == 0, L.lra_status_str(res.info.status)
    return res


# ragged in both tile directions (128 rows, 64 columns), K padded to 64 / 128
@pytest.mark.parametrize("m,n,r,k,l,noise", [
    (256, 192, 6, 8, 8, 1e-3),
    (1000, 900, 10, 16, 24, 1e-3),
    (1024, 1024, 40, 48, 64, 1e-4),
    (3000, 2500, 64, 64, 96, 1e-4),
])
def test_full_residual_matches_fp64(ctx, m, n, r, k, l, noise):
    A = W.factor_gaussian(m + n + l, m, n, r, noise)
    J0 = W.draw_indices(m - n + 7, n, l)
    res = _solve_full(ctx, A, J0, k, l, 3)
    ref = rel_fro_error(A.astype(np.float64), res.C.cpu().numpy(), res.U, res.R.cpu().numpy())
    assert res.info.full_rel_err == pytest.approx(ref, rel=2e-3, abs=1e-7), (res.info.full_rel_err, ref)
    # error bar against the FP64 oracle's own C-A solution
    o = O.cross_approximation(O.Dense(A), J0, k=k, sweeps=3)
    err_o = O.full_residual(O.Dense(A.astype(np.float64)), o.C, o.U, o.R)[0]
    assert error_ok(res.info.full_rel_err, err_o)


def test_full_residual_rejects_unsupported_sources(ctx):
    A = torch.zeros((100, 90), dtype=torch.float64, device=DEV)
    params, keep = L.make_params(4, 4, 1, [0, 1, 2, 3], full_residual=True)
    with pytest.raises(L.LraError) as e:
        ctx.submit(L.make_source("dense", a=A), params)
    assert e.value.code == L.LRA_EINVAL
