"""Parity of the native FP64 GEMM (alp_gemm_f64, through the C-ABI) with the
CPU oracle: bit-exact on integer inputs, elementwise within
2 K u |alpha| (|A||B|) + u |beta C| on random inputs, NaN sentinels around
every operand, every valid tile config, both the TMA and the cp.async path."""
import numpy as np
import pytest

from paper_1706_10086_gb300 import inputs

from .gpu_util import assert_within_bound, dev, host

pytestmark = pytest.mark.gpu


def run_gemm(alp, A, B, C, alpha, beta, cfg=None, lda=None, ldb=None, ldc=None, stream=None):
    import torch
    M, K = A.shape
    N = B.shape[1]
    dA, lda = dev(A, lda)
    dB, ldb = dev(B, ldb)
    dC, ldc = dev(C if C is not None else np.full((M, N), np.nan), ldc)
    alp.alp_gemm_f64(M, N, K, alpha, dA, lda, dB, ldb, beta, dC, ldc, cfg=cfg, stream=stream)
    torch.cuda.synchronize()
    assert alp.alp_get_device_error() == alp.ALP_OK
    full = dC.cpu().numpy()
    return full[:M, :N], full


def test_dgemm_512_integer_bit_exact(alp, orc):
    """Integer entries in {-8..8}: all partial sums exact in FP64, so GPU ==
    oracle bit for bit (alpha = 1, beta = 0, C never read)."""
    M = N = K = 512
    A, B, _ = inputs.gemm_operands(inputs.workload_seed("dgemm_512"), M, N, K, kind="int",
                                   with_c=False)
    got, _ = run_gemm(alp, A, B, None, 1.0, 0.0)
    ref = orc.gemm(1.0, A, B, 0.0)
    assert np.array_equal(got, ref)


def test_dgemm_512_uniform_bound(alp, orc):
    M = N = K = 512
    A, B, _ = inputs.gemm_operands(inputs.workload_seed("dgemm_512"), M, N, K, with_c=False)
    got, _ = run_gemm(alp, A, B, None, 1.0, 0.0)
    ref = orc.gemm(1.0, A, B, 0.0)
    assert_within_bound(got, ref, orc.absgemm(A, B), 1.0, 0.0, None, K)


@pytest.mark.parametrize("shape", [(200, 136, 100), (1, 1, 1), (67, 300, 257), (129, 65, 3),
                                   (256, 256, 1031)])
def test_ragged_shapes_alpha_beta(alp, orc, shape):
    M, N, K = shape
    A, B, C = inputs.gemm_operands(900 + M + N + K, M, N, K)
    got, _ = run_gemm(alp, A, B, C, 1.5, 0.5)
    ref = orc.gemm(1.5, A, B, 0.5, C)
    assert_within_bound(got, ref, orc.absgemm(A, B), 1.5, 0.5, C, K)


@pytest.mark.parametrize("pads", [(2, 2, 2), (3, 5, 1), (0, 0, 1)])
def test_sentinel_padding(alp, orc, pads):
    """lda > K, ldb > N, ldc > N with NaN padding: padding never read (no NaN
    in C) and never written (still NaN).  Odd leading dims take the cp.async path."""
    M, N, K = 77, 90, 133
    A, B, C = inputs.gemm_operands(950, M, N, K)
    got, full = run_gemm(alp, A, B, C, 1.5, 0.5, lda=K + pads[0], ldb=N + pads[1],
                         ldc=N + pads[2])
    assert np.isnan(full[:M, N:]).all()
    ref = orc.gemm(1.5, A, B, 0.5, C)
    assert_within_bound(got, ref, orc.absgemm(A, B), 1.5, 0.5, C, K)


def test_alpha_zero_and_beta_zero_read_nothing(alp, orc):
    import torch
    M, N, K = 64, 48, 32
    A, B, C = inputs.gemm_operands(960, M, N, K)
    An = np.full_like(A, np.nan)
    got, _ = run_gemm(alp, An, np.full_like(B, np.nan), C, 0.0, 0.5)
    assert np.array_equal(got, 0.5 * C)
    got, _ = run_gemm(alp, A, B, np.full_like(C, np.nan), 1.0, 0.0)
    assert not np.isnan(got).any()
    got, _ = run_gemm(alp, np.zeros((M, 0)), np.zeros((0, N)), C, 1.0, 2.0)
    assert np.array_equal(got, 2.0 * C)


def test_integer_powers_of_two_scalars_bit_exact(alp, orc):
    M, N, K = 130, 70, 300
    A, B, C = inputs.gemm_operands(970, M, N, K, kind="int")
    got, _ = run_gemm(alp, A, B, C, 2.0, 0.5)
    ref = orc.gemm(2.0, A, B, 0.5, C)
    assert np.array_equal(got, ref)


def test_every_valid_config(alp, orc):
    """Each tile config of the sweep gives the right answer on a shape that
    spans several tiles with ragged edges in M, N and K."""
    M, N, K = 300, 280, 200
    A, B, C = inputs.gemm_operands(980, M, N, K, kind="int")
    ref = orc.gemm(1.0, A, B, -1.0, C)
    P = alp.ALP_PATH_NATIVE
    for i in range(alp.alp_config_count(P)):
        cfg = alp.alp_config_at(P, i)
        got, _ = run_gemm(alp, A, B, C, 1.0, -1.0, cfg=cfg)
        assert np.array_equal(got, ref), cfg
        # and the cp.async variant of the same config (odd lda)
        got, _ = run_gemm(alp, A, B, C, 1.0, -1.0, cfg=cfg, lda=K + 1)
        assert np.array_equal(got, ref), ("ldg", cfg)


def test_full_size_sampled_rows(alp, orc):
    """N = 8192, alpha = 1.5, beta = 0.5, in the bench's launch configuration:
    sampled rows against the oracle."""
    import torch
    M = N = K = 8192
    seed = inputs.workload_seed("dgemm_scan")
    A, B, C = inputs.gemm_operands(seed, M, N, K)
    got, _ = run_gemm(alp, A, B, C, 1.5, 0.5)
    rows = np.array([0, 1, 4095, 8191, 1234, 7777])
    ref = orc.gemm(1.5, A, B, 0.5, C, rows=rows)
    absAB = orc.absgemm(A, B, rows=rows)
    assert_within_bound(got[rows], ref, absAB, 1.5, 0.5, C[rows], K)


def test_stream_ordering_and_error_word(alp, orc):
    import torch
    s = torch.cuda.Stream()
    M, N, K = 96, 96, 64
    A, B, C = inputs.gemm_operands(990, M, N, K, kind="int")
    with torch.cuda.stream(s):
        got, _ = run_gemm(alp, A, B, C, 1.0, 1.0, stream=s)
    assert np.array_equal(got, orc.gemm(1.0, A, B, 1.0, C))
    assert alp.alp_get_device_error() == alp.ALP_OK


@pytest.mark.parametrize("ta,tb", [(0, 1), (1, 0), (1, 1)])
def test_native_transposed_operands(alp, orc, ta, tb):
    """alp_gemm_f64_ex: bit-identical to alp_gemm_f64 on the transposed matrices
    (same kernel, same config), within the bound of the oracle; padded leading
    dimensions; a missing workspace is refused."""
    import torch
    M, N, K = 300, 260, 270
    A, B, C = inputs.gemm_operands(5100 + 2 * ta + tb, M, N, K)
    As = np.ascontiguousarray(A.T) if ta else A
    Bs = np.ascontiguousarray(B.T) if tb else B
    lda, ldb = As.shape[1] + 2, Bs.shape[1] + 4
    dA = torch.full((As.shape[0], lda), float("nan"), dtype=torch.float64, device="cuda")
    dA[:, :As.shape[1]] = torch.from_numpy(As)
    dB = torch.full((Bs.shape[0], ldb), float("nan"), dtype=torch.float64, device="cuda")
    dB[:, :Bs.shape[1]] = torch.from_numpy(Bs)
    cfg = (64, 128, 64, 4, 4, 0)
    dC = torch.from_numpy(C).cuda()
    ws = alp.alp_gemm_f64_ex_workspace(ta, tb, M, N, K)
    assert ws >= 8 * (ta * M * K + tb * K * N)
    work = torch.empty(ws, dtype=torch.uint8, device="cuda")
    alp.alp_gemm_f64_ex(ta, tb, M, N, K, 1.5, dA, lda, dB, ldb, 0.5, dC, N, cfg=cfg,
                        workspace=work, workspace_bytes=ws)
    ref = torch.from_numpy(C).cuda()
    alp.alp_gemm_f64(M, N, K, 1.5, torch.from_numpy(A).cuda(), K, torch.from_numpy(B).cuda(), N,
                     0.5, ref, N, cfg=cfg)
    torch.cuda.synchronize()
    got = dC.cpu().numpy()
    assert np.array_equal(got, ref.cpu().numpy())
    exact = orc.gemm(1.5, A, B, 0.5, C)
    bound = orc.error_bound(1.5, orc.absgemm(A, B), 0.5, C, K)
    assert np.all(np.abs(got - exact) <= bound)
    assert alp.alp_gemm_f64_ex(ta, tb, M, N, K, 1.5, dA, lda, dB, ldb, 0.5, dC, N,
                               raise_on_error=False) == alp.ALP_ERR_WORKSPACE
    assert alp.alp_gemm_f64_ex_workspace(2, 0, M, N, K) == 0


def test_fp64_peak_probes(alp):
    """The FP64 denominators: every probe kind runs and reports a positive
    rate; the native kernel's m16n8k4 rate is within 2x of the best DMMA shape
    (a probe that measured nothing would sit far off)."""
    rates = [alp.alp_probe_fp64_peak(kind, 2000, 2, 256) for kind in range(4)]
    assert all(r > 0 for r in rates), rates
    best = max(rates[0], rates[2], rates[3])
    assert rates[0] >= 0.5 * best, rates
