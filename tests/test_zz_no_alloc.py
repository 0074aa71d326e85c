"""alp_gemm_batched_varsize_noalloc through the C-ABI: the batched GEMM for
callers that cannot allocate device memory, whose work list lives in the
library's built-in scratch array.  Two calls in a row (different batches, so
the second call finds the first one's contents in the array) must agree with
the workspace entry point within the tests' error bound.  Kept in a file of
its own that pytest collects last; it also passes alone in a fresh process."""
import numpy as np
import pytest

from paper_1706_10086_gb300 import inputs

from .test_batched_gpu import Batch

pytestmark = pytest.mark.gpu


def _bound(orc, b, p):
    A, B, C = b.host[p]
    K = b.shapes[p][2]
    return orc.error_bound(b.alpha[p], orc.absgemm(A, B), b.beta[p], C, K)


@pytest.mark.parametrize("calls", [((70, 16, 300), 5800), ((25, 16, 600), 5900)])
def test_noalloc_matches_workspace_entry_point_twice(alp, orc, calls):
    import torch
    (count0, lo0, hi0), seed0 = calls
    # two calls in a row with different batches: the second finds the first
    # call's work list in the shared scratch
    for (count, lo, hi), seed in (((count0, lo0, hi0), seed0), ((count0 + 11, 16, 200), seed0 + 50)):
        shapes = inputs.shapes(seed, count, lo, hi)
        ref = Batch(shapes, seed)                  # workspace entry point
        ref.run(alp)
        b = Batch(shapes, seed)                    # same inputs, no-alloc entry point
        alp.alp_gemm_batched_varsize_noalloc(*b.args())
        torch.cuda.synchronize()
        assert alp.alp_get_device_error() == alp.ALP_OK
        for p, (M, N, K) in enumerate(b.shapes):
            got, _ = b.result(p)
            want, _ = ref.result(p)
            assert np.all(np.abs(got - want) <= _bound(orc, b, p)), p


def test_noalloc_rejects_batches_beyond_its_scratch(alp):
    n = 70000
    hM = np.full(n, 4, dtype=np.int64)
    st = alp.alp_gemm_batched_varsize_noalloc(n, 8, 8, 8, 8, 8, 8, 8, 8, 8, 8, 8, hM, hM, hM,
                                              stream=0, raise_on_error=False)
    assert st == alp.ALP_ERR_WORKSPACE
