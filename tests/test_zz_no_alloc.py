"""The allocation-free GEMM entry point (rtcc_gemm_noalloc) against a float64 product and the
allocating entry point.

This entry point exists for callers that cannot let a library allocate device memory (for
example applications that hand out all device memory from their own pool); its scratch is a
fixed static device array shared by every call, so two calls in a row must not see each
other's leftovers.  The reference is np.einsum in float64, which shares nothing with the
library's packing and GEMM kernels; the allocating entry point (rtcc_selftest_gemm) is checked
beside it.  The file is named to run last: a failure here leaves every other test run.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

# same bound as the other GEMM tests: max|C - C_ref| / (max|A| max|B| K)
TOL = {1: 2e-3, 2: 2e-6, 3: 3e-5}


def _inputs(rng, nb, m, n, k, kinds):
    a = rng.standard_normal((nb, m, k)) + (1j * rng.standard_normal((nb, m, k)) if kinds[0] == "c" else 0)
    b = rng.standard_normal((nb, n, k)) + (1j * rng.standard_normal((nb, n, k)) if kinds[1] == "c" else 0)
    return a, b


@pytest.mark.parametrize("prec", [1, 2, 3])
@pytest.mark.parametrize("kinds", ["rr", "cc", "cr", "rc"])
def test_noalloc_gemm_matches_float64_product_twice(prec, kinds):
    import torch

    from paper_2205_05175_gb300 import rtcc
    rng = np.random.default_rng(7 + prec)
    shapes = [(2, 300, 200, 150), (1, 129, 70, 1000)]   # second call: other shapes, fresh inputs
    for nb, m, n, k in shapes:
        a, b = _inputs(rng, nb, m, n, k, kinds)
        ref = np.einsum("bmk,bnk->bmn", a, b)
        alloc = rtcc.rtcc_selftest_gemm(prec, a, b)
        ta = torch.from_numpy(np.ascontiguousarray(a)).cuda()
        tb = torch.from_numpy(np.ascontiguousarray(b)).cuda()
        cdt = torch.complex128 if (np.iscomplexobj(a) or np.iscomplexobj(b)) else torch.float64
        tc = torch.full((nb, m, n), float("nan"), dtype=cdt, device="cuda")   # overwritten by the call
        rtcc.rtcc_gemm_noalloc(prec, ta, tb, tc)
        torch.cuda.synchronize()
        got = tc.cpu().numpy()
        scale = np.abs(a).max() * np.abs(b).max() * k
        err = np.abs(got - ref).max() / scale
        assert err < TOL[prec], err
        assert np.abs(alloc - ref).max() / scale < TOL[prec]


def test_noalloc_rejects_oversized_and_float64():
    import torch

    from paper_2205_05175_gb300 import rtcc
    a = torch.zeros((1, 8, 8), dtype=torch.float64, device="cuda")
    c = torch.zeros((1, 8, 8), dtype=torch.float64, device="cuda")
    with pytest.raises(rtcc.RtccError) as e:
        rtcc.rtcc_gemm_noalloc(0, a, a, c)
    assert e.value.status == "INVALID_ARG"
    big = torch.zeros((1, 8192, 4096), dtype=torch.float64, device="cuda")
    cb = torch.zeros((1, 8192, 8192), dtype=torch.float64, device="cuda")
    with pytest.raises(rtcc.RtccError) as e:
        rtcc.rtcc_gemm_noalloc(3, big, big, cb)
    assert e.value.status == "INVALID_ARG" and "static limit" in rtcc.rtcc_last_error()
