"""The cluster forms of the cross inverse and of the nucleus against the
one-SM kernels.  A context with one stream runs them on clusters of 8 CTAs;
a context with several streams keeps them on one SM each (the other SMs
belong to the other jobs).  Every entry takes the same operations in the
same order in both forms, so the two solves agree bit for bit: index sets,
nucleus and singular values."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1611_01391_gb300 as L  # noqa: E402


def _stored(seed, m, n, r, noise):
    """Stored FP32 rank-r + noise matrix, made on the device."""
    g = torch.Generator(device="cuda")
    g.manual_seed(seed)
    a = torch.randn((m, r), device="cuda", generator=g) @ torch.randn((r, n), device="cuda", generator=g)
    a.mul_(1.0 / np.sqrt(r)).add_(torch.randn((m, n), device="cuda", generator=g), alpha=noise)
    torch.cuda.synchronize()   # the library's streams do not wait for torch's
    return a


@pytest.mark.parametrize("l,k", [(96, 64), (48, 32)])
def test_cluster_kernels_match_the_one_sm_kernels(l, k):
    # 32768 rows: the vertical strip's inverse does not fit beside the strip
    # in the maxvol launch, so the separate inverse kernel runs every sweep
    m, n = 32768, 4096
    a = _stored(W.BASE_SEED + 900 + l, m, n, k, 1e-4)
    src = L.make_source("dense", a=a)
    J0 = W.draw_indices(W.BASE_SEED + 901 + l, n, l)
    p, keep = L.make_params(k, l, 3, J0)
    with L.Context(0, n_streams=1) as c1:
        one = c1.solve(src, p, l)
    with L.Context(0, n_streams=2) as c2:
        many = c2.solve(src, p, l)
    assert one.info.status == 0 and many.info.status == 0
    np.testing.assert_array_equal(one.I, many.I)
    np.testing.assert_array_equal(one.J, many.J)
    np.testing.assert_array_equal(one.U, many.U)
    np.testing.assert_array_equal(one.sigma, many.sigma)
    assert one.info.k_eff == many.info.k_eff
    assert one.info.swaps_total > 0
