"""The GEMM calls inside CUDA graph capture: each call is captured once into a
graph (torch.cuda.graph, on its capture stream), then replayed after new
operands are copied into the captured buffers.  A replay must give, bit for
bit, what a direct call on the same operands gives (every launch, memset and
kernel parameter of the call is captured; nothing is decided on the host from
the data)."""
import pytest

from paper_1706_10086_gb300 import inputs

pytestmark = pytest.mark.gpu


def _direct_and_replays(alp, launch, M, N, K, seeds, dtype=None):
    import torch
    dtype = dtype or torch.float64
    A = torch.empty(M, K, dtype=dtype, device="cuda")
    B = torch.empty(K, N, dtype=dtype, device="cuda")
    C = torch.empty(M, N, dtype=dtype, device="cuda")
    C0 = torch.empty(M, N, dtype=dtype, device="cuda")

    def load(seed):
        a, b, c = inputs.gemm_operands(seed, M, N, K, kind="scaled", phi=4)
        A.copy_(torch.from_numpy(a).to(dtype))
        B.copy_(torch.from_numpy(b).to(dtype))
        C0.copy_(torch.from_numpy(c).to(dtype))
        C.copy_(C0)

    load(seeds[0])
    launch(A, B, C, torch.cuda.current_stream())      # warm-up outside capture
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    load(seeds[0])
    with torch.cuda.graph(g):
        launch(A, B, C, torch.cuda.current_stream())
    torch.cuda.synchronize()
    out = []
    for seed in seeds:
        load(seed)
        g.replay()
        torch.cuda.synchronize()
        replay = C.clone()
        load(seed)
        launch(A, B, C, torch.cuda.current_stream())
        torch.cuda.synchronize()
        out.append((replay, C.clone()))
    assert alp.alp_get_device_error() == alp.ALP_OK
    return out


@pytest.mark.parametrize("kind,s", [(4, 15), (3, 7)])
def test_emulated_gemm_captured_in_a_graph(alp, kind, s):
    import torch
    M, N, K = 300, 520, 700
    ws = alp.alp_gemm_f64_emul_workspace(M, N, K, s, kind)
    work = torch.empty(ws, dtype=torch.uint8, device="cuda")

    def launch(A, B, C, st):
        alp.alp_gemm_f64_emul(M, N, K, 1.5, A, K, B, N, 0.5, C, N, s, kind, work, ws, stream=st)

    for replay, direct in _direct_and_replays(alp, launch, M, N, K, [7001, 7002, 7003]):
        assert torch.equal(replay, direct)


def test_emulated_fp32_gemm_captured_in_a_graph(alp):
    import torch
    M, N, K = 260, 300, 333
    kind = alp.ALP_SLICE_BF16_B8
    ws = alp.alp_gemm_f32_emul_workspace(M, N, K, 3, kind)
    work = torch.empty(ws, dtype=torch.uint8, device="cuda")

    def launch(A, B, C, st):
        alp.alp_gemm_f32_emul(M, N, K, 1.5, A, K, B, N, 0.5, C, N, 3, kind, work, ws, stream=st)

    for replay, direct in _direct_and_replays(alp, launch, M, N, K, [7101, 7102],
                                              dtype=torch.float32):
        assert torch.equal(replay, direct)


def test_native_gemm_captured_in_a_graph(alp):
    import torch
    M, N, K = 384, 257, 300

    def launch(A, B, C, st):
        alp.alp_gemm_f64(M, N, K, 1.5, A, K, B, N, 0.5, C, N, stream=st)

    for replay, direct in _direct_and_replays(alp, launch, M, N, K, [7201, 7202]):
        assert torch.equal(replay, direct)


def test_transposed_native_gemm_captured_in_a_graph(alp):
    """alp_gemm_f64_ex packs the transposed operands into its workspace inside
    the captured region as well."""
    import torch
    M, N, K = 200, 300, 150
    ws = alp.alp_gemm_f64_ex_workspace(1, 1, M, N, K)
    work = torch.empty(ws, dtype=torch.uint8, device="cuda")
    dA = torch.from_numpy(inputs.uniform(7301, 0, (K, M))).cuda()     # op(A) = A^T, M x K
    dB = torch.from_numpy(inputs.uniform(7302, 0, (N, K))).cuda()     # op(B) = B^T, K x N
    C = torch.zeros(M, N, dtype=torch.float64, device="cuda")

    def launch():
        alp.alp_gemm_f64_ex(1, 1, M, N, K, 1.5, dA, M, dB, K, 0.0, C, N, None, work, ws,
                            stream=torch.cuda.current_stream())

    launch()
    torch.cuda.synchronize()
    direct = C.clone()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        launch()
    C.zero_()
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(C, direct)
    assert alp.alp_get_device_error() == alp.ALP_OK
