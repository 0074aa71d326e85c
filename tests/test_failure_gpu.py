"""Failure detection without a GPU fault: a device wait that runs out of time
is reported as ALP_ERR_TIMEOUT through the device error word, the kernel
returns, and the context stays usable.  The failure is made on the host: the
test hook makes block 0's producer arm one pipeline stage without issuing its
copy, so its consumers' wait (limit lowered to 200 ms) runs out."""
import numpy as np
import pytest

from paper_1706_10086_gb300 import inputs

pytestmark = pytest.mark.gpu


def test_wait_timeout_reported_and_context_usable(alp, orc):
    import torch
    M = N = K = 512
    A, B, _ = inputs.gemm_operands(7100, M, N, K, kind="int", with_c=False)
    dA = torch.from_numpy(A).cuda()
    dB = torch.from_numpy(B).cuda()
    dC = torch.zeros(M, N, dtype=torch.float64, device="cuda")
    assert alp.alp_get_device_error() == alp.ALP_OK
    alp.alp_set_wait_timeout_ms(200)
    alp.alp_debug_inject_skip(3)
    try:
        alp.alp_gemm_f64(M, N, K, 1.0, dA, K, dB, N, 0.0, dC, N)
        torch.cuda.synchronize()
        assert alp.alp_get_device_error() == alp.ALP_ERR_TIMEOUT
    finally:
        alp.alp_debug_inject_skip(-1)
        alp.alp_set_wait_timeout_ms(4000)
    # the error word was read and cleared; the next call is correct
    alp.alp_gemm_f64(M, N, K, 1.0, dA, K, dB, N, 0.0, dC, N)
    torch.cuda.synchronize()
    assert alp.alp_get_device_error() == alp.ALP_OK
    assert np.array_equal(dC.cpu().numpy(), orc.gemm(1.0, A, B, 0.0))
