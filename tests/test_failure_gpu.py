"""Failure detection without a GPU fault: a device wait that runs out of time
is reported as ALP_ERR_TIMEOUT through the device error word, the kernel
returns, and the context stays usable.  The failure is made on the host: the
test hook makes block 0's producer arm one pipeline stage without issuing its
copy, so its consumers' wait (limit lowered to 200 ms) runs out."""
import numpy as np
import pytest

from paper_1706_10086_gb300 import inputs

from .test_emul_crt_gpu import crt_k

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


@pytest.mark.parametrize("cfg", [(128, 256, 64, 1, 0, 8), (256, 256, 64, 2, 0, 8)],
                         ids=["one_block", "cta_pair"])
def test_emulated_wait_timeout_reported_and_context_usable(alp, orc, cfg):
    """The emulated path's tensor-core kernel, one block per tile and CTA
    pairs (for the modular scheme's GEMM call the fused launch, with its
    schedule and reconstruction waits): block 0's producer arms its fourth pipeline stage without issuing
    the copies, the MMA thread's wait on that stage runs out (limit 200 ms),
    ALP_ERR_TIMEOUT is recorded, every block of the launch leaves (its own
    copies landed, its TMEM freed), and the next call on the same context is
    bit-exact against the oracle's definition of the modular scheme."""
    import time

    import torch
    M, N, K, n = 512, 768, 2048, 4
    CRT = alp.ALP_SLICE_BF16_CRT
    A, B, C = inputs.gemm_operands(7200 + cfg[0], M, N, K, kind="scaled", phi=2)
    dA, dB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    dC = torch.from_numpy(C).cuda()
    ws = alp.alp_gemm_f64_emul_workspace(M, N, K, n, CRT)
    work = torch.empty(ws, dtype=torch.uint8, device="cuda")
    assert alp.alp_get_device_error() == alp.ALP_OK
    alp.alp_tune_set_cached(M, N, K, alp.ALP_PATH_EMUL, cfg)
    alp.alp_set_wait_timeout_ms(200)
    alp.alp_debug_inject_skip(3)
    try:
        t0 = time.perf_counter()
        alp.alp_gemm_f64_emul(M, N, K, 1.5, dA, K, dB, N, 0.5, dC, N, n, CRT, work, ws)
        torch.cuda.synchronize()
        elapsed = time.perf_counter() - t0
        assert alp.alp_get_device_error() == alp.ALP_ERR_TIMEOUT
        assert elapsed < 5.0, elapsed       # one limit, not one per stage or block
    finally:
        alp.alp_debug_inject_skip(-1)
        alp.alp_set_wait_timeout_ms(4000)
    try:
        dC = torch.from_numpy(C).cuda()
        alp.alp_gemm_f64_emul(M, N, K, 1.5, dA, K, dB, N, 0.5, dC, N, n, CRT, work, ws)
        torch.cuda.synchronize()
        assert alp.alp_get_device_error() == alp.ALP_OK
    finally:
        alp.alp_tune_clear_cache()
    want, rc = orc.crt_gemm(1.5, A, B, 0.5, C, crt_k(K, n))
    assert rc == 0 and np.array_equal(dC.cpu().numpy(), want)


@pytest.mark.parametrize("kind", [4, 3], ids=["modular", "digits_b8_trim"])
def test_slice_products_wait_timeout_reported_and_context_usable(alp, kind):
    """The two-launch product kernel on CTA pairs (alp_emul_slice_products:
    what the digit schemes and ALP_EMUL_CRT_FUSE=0 run): the armed stage's
    wait runs out (limit 200 ms), ALP_ERR_TIMEOUT is recorded within one
    limit, and the same stage call then writes the same sums as it did before
    the fault."""
    import time

    import torch
    M, N, K, n = 512, 768, 2048, 4
    A, B, _ = inputs.gemm_operands(7300 + kind, M, N, K, kind="scaled", phi=2, with_c=False)
    kpad, ldg = K, (N + 255) // 256 * 256
    dA, dB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    de = torch.empty(M, dtype=torch.int32, device="cuda")
    df = torch.empty(N, dtype=torch.int32, device="cuda")
    alp.alp_emul_exponents(M, K, dA, K, 0, de)
    alp.alp_emul_exponents(N, K, dB, N, 1, df)
    da = torch.empty((n, M, kpad), dtype=torch.bfloat16, device="cuda")
    db = torch.empty((n, N, kpad), dtype=torch.bfloat16, device="cuda")
    alp.alp_emul_split(M, K, dA, K, 0, de, n, kind, da, kpad)
    alp.alp_emul_split(N, K, dB, N, 1, df, n, kind, db, kpad)
    gbytes = 1 if kind == 4 else 4   # modular: n byte planes; digits: s int32 group planes
    G0 = torch.zeros(n * M * ldg * gbytes, dtype=torch.uint8, device="cuda")
    alp.alp_emul_slice_products(M, N, K, n, kind, da, db, kpad, G0, ldg)
    torch.cuda.synchronize()
    assert alp.alp_get_device_error() == alp.ALP_OK
    G = torch.zeros_like(G0)
    alp.alp_set_wait_timeout_ms(200)
    alp.alp_debug_inject_skip(3)
    try:
        t0 = time.perf_counter()
        alp.alp_emul_slice_products(M, N, K, n, kind, da, db, kpad, G, ldg)
        torch.cuda.synchronize()
        elapsed = time.perf_counter() - t0
        assert alp.alp_get_device_error() == alp.ALP_ERR_TIMEOUT
        assert elapsed < 5.0, elapsed
    finally:
        alp.alp_debug_inject_skip(-1)
        alp.alp_set_wait_timeout_ms(4000)
    G.zero_()
    alp.alp_emul_slice_products(M, N, K, n, kind, da, db, kpad, G, ldg)
    torch.cuda.synchronize()
    assert alp.alp_get_device_error() == alp.ALP_OK
    assert torch.equal(G, G0)

