"""alp_gemm_batched_varsize_noalloc through the C-ABI: the batched GEMM for
callers that cannot allocate device memory (frameworks whose device memory
belongs to their own pool allocator, loops that must stay out of the
allocator), whose work list lives in the library's built-in scratch array.

Two calls in a row, on different batches, so that the second call finds the
first one's work list in the shared array: each result must be bit-identical
to the workspace entry point's (both run the same plan and persistent kernels
with the same class table, so any difference would be stale scratch) and
within the tests' error bound of the oracle.  Kept in a file of its own that
pytest collects last; it also passes alone in a fresh process."""
import numpy as np
import pytest

from paper_1706_10086_gb300 import inputs

from .test_batched_gpu import Batch

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("calls", [((70, 16, 300), 5800), ((25, 16, 600), 5900)])
def test_noalloc_matches_workspace_entry_point_twice(alp, orc, calls):
    import torch
    (count0, lo0, hi0), seed0 = calls
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
            assert np.array_equal(got, want), p
            if M == 0 or N == 0:
                continue
            A, B, C = b.host[p]
            oracle_c = orc.gemm(b.alpha[p], A, B, b.beta[p], C)
            bound = orc.error_bound(b.alpha[p], orc.absgemm(A, B), b.beta[p], C, K)
            assert np.all(np.abs(got - oracle_c) <= bound), p


def test_noalloc_rejects_batches_beyond_its_scratch(alp):
    """70,000 problems need more than the 1 MiB array: ALP_ERR_WORKSPACE.  The
    device pointers are NULL, which the library also rejects before any
    launch, so this call can launch nothing whatever order the checks take."""
    n = 70000
    hM = np.full(n, 4, dtype=np.int64)
    st = alp.alp_gemm_batched_varsize_noalloc(n, None, None, None, None, None, None, None, None,
                                              None, None, None, hM, hM, hM, stream=0,
                                              raise_on_error=False)
    assert st == alp.ALP_ERR_WORKSPACE
