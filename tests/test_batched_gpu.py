"""Parity of the batched variable-size GEMM (alp_gemm_batched_varsize and its
CUDA-graph wrapper, through the C-ABI) with the oracle applied per problem,
and bit-identity with single-problem launches of the same tile config."""
import numpy as np
import pytest

from paper_1706_10086_gb300 import inputs

pytestmark = pytest.mark.gpu


class Batch:
    """Device storage of a batch: one allocation per matrix plus the device
    arrays of sizes, scalars, pointers and leading dimensions."""

    def __init__(self, shapes, seed, kind="uniform", alphas=None, betas=None, pad=0):
        import torch
        self.shapes = np.asarray(shapes, dtype=np.int64).reshape(-1, 3)
        n = len(self.shapes)
        self.alpha = np.full(n, 1.5) if alphas is None else np.asarray(alphas, dtype=np.float64)
        self.beta = np.full(n, 0.5) if betas is None else np.asarray(betas, dtype=np.float64)
        self.host = []
        self.dev = []
        ptrA, ptrB, ptrC, lda, ldb, ldc = [], [], [], [], [], []
        for p, (M, N, K) in enumerate(self.shapes):
            A, B, C = inputs.gemm_operands(seed + p, int(M), int(N), int(K), kind=kind)
            la, lb, lc = int(K) + pad, int(N) + pad, int(N) + pad
            dA = torch.full((max(M, 1), max(la, 1)), float("nan"), dtype=torch.float64, device="cuda")
            dB = torch.full((max(K, 1), max(lb, 1)), float("nan"), dtype=torch.float64, device="cuda")
            dC = torch.full((max(M, 1), max(lc, 1)), float("nan"), dtype=torch.float64, device="cuda")
            if M and K:
                dA[:M, :K] = torch.from_numpy(A)
            if K and N:
                dB[:K, :N] = torch.from_numpy(B)
            if M and N:
                dC[:M, :N] = torch.from_numpy(C)
            self.host.append((A, B, C))
            self.dev.append((dA, dB, dC))
            ptrA.append(dA.data_ptr()); ptrB.append(dB.data_ptr()); ptrC.append(dC.data_ptr())
            lda.append(la); ldb.append(lb); ldc.append(lc)
        t = lambda a, dt=torch.int64: torch.tensor(a, dtype=dt, device="cuda")
        self.hM = np.ascontiguousarray(self.shapes[:, 0])
        self.hN = np.ascontiguousarray(self.shapes[:, 1])
        self.hK = np.ascontiguousarray(self.shapes[:, 2])
        self.dM, self.dN, self.dK = t(self.hM), t(self.hN), t(self.hK)
        self.dalpha = t(self.alpha, torch.float64)
        self.dbeta = t(self.beta, torch.float64)
        self.dA, self.dB, self.dC = t(ptrA), t(ptrB), t(ptrC)
        self.dlda, self.dldb, self.dldc = t(lda), t(ldb), t(ldc)
        self.count = n

    def args(self):
        return (self.count, self.dM, self.dN, self.dK, self.dalpha, self.dA, self.dlda, self.dB,
                self.dldb, self.dbeta, self.dC, self.dldc, self.hM, self.hN, self.hK)

    def run(self, alp):
        import torch
        ws = alp.alp_gemm_batched_workspace(self.count, self.hM, self.hN, self.hK)
        self.work = torch.empty(max(ws, 1), dtype=torch.uint8, device="cuda")
        alp.alp_gemm_batched_varsize(*self.args(), self.work, ws)
        torch.cuda.synchronize()
        assert alp.alp_get_device_error() == alp.ALP_OK

    def result(self, p):
        M, N, _ = self.shapes[p]
        return self.dev[p][2].cpu().numpy()[:M, :N], self.dev[p][2].cpu().numpy()


def check_against_oracle(orc, b, exact=False):
    for p, (M, N, K) in enumerate(b.shapes):
        if M == 0 or N == 0:
            continue
        A, B, C = b.host[p]
        got, full = b.result(p)
        ref = orc.gemm(b.alpha[p], A, B, b.beta[p], C)
        if exact:
            assert np.array_equal(got, ref), p
        else:
            bound = orc.error_bound(b.alpha[p], orc.absgemm(A, B), b.beta[p], C, K)
            assert np.all(np.abs(got - ref) <= bound), (p, (M, N, K))
        assert not np.isnan(got).any()
        assert np.isnan(full[:M, N:]).all()   # padding untouched


def test_batched_mixed_sizes_bound(alp, orc):
    shapes = inputs.shapes(inputs.workload_seed("batched_4096"), 120, 16, 300)
    b = Batch(shapes, 5000, pad=3)
    b.run(alp)
    check_against_oracle(orc, b)


def test_batched_integer_exact_and_edge_sizes(alp, orc):
    shapes = [(1, 1, 1), (0, 5, 5), (5, 0, 5), (7, 9, 0), (33, 65, 129), (64, 64, 64),
              (128, 128, 17), (200, 31, 1000), (31, 200, 3), (129, 257, 64)]
    alphas = [1.0, 1.0, 1.0, 1.0, 1.0, 0.0, 2.0, 1.0, -1.0, 1.0]
    betas = [0.0, 0.0, 0.0, 2.0, 1.0, 0.5, 0.5, 0.0, 1.0, -2.0]
    b = Batch(shapes, 5100, kind="int", alphas=alphas, betas=betas)
    b.run(alp)
    check_against_oracle(orc, b, exact=True)


def test_batched_alpha_zero_reads_no_operands(alp, orc):
    import torch
    b = Batch([(40, 50, 60), (70, 20, 10)], 5200, alphas=[0.0, 0.0], betas=[0.5, 0.0])
    for dA, dB, _ in b.dev:
        dA.fill_(float("nan"))
        dB.fill_(float("nan"))
    b.run(alp)
    got0, _ = b.result(0)
    assert np.array_equal(got0, 0.5 * b.host[0][2])
    got1, _ = b.result(1)
    assert np.array_equal(got1, np.zeros_like(got1))


def test_batched_matches_single_launches_bit_for_bit(alp, orc):
    """Problems of the 64x64 and 128x128 classes with the same tile config as
    a single alp_gemm_f64 launch: identical bits (same k order per tile)."""
    import torch
    shapes = [(100, 90, 77), (64, 120, 300), (300, 260, 129), (500, 200, 64)]
    b = Batch(shapes, 5300)
    b.run(alp)
    for p, (M, N, K) in enumerate(b.shapes):
        cls = alp.alp_batched_class_of(M, N)
        bm, bn, bk = alp.alp_batched_get_class_config(cls)
        A, B, C = b.host[p]
        dA = torch.from_numpy(A).cuda()
        dB = torch.from_numpy(B).cuda()
        dC = torch.from_numpy(C).cuda()
        cfg = (bm, bn, bk, bm // 16, bn // 16, 0)
        assert alp.alp_config_valid(cfg)
        alp.alp_gemm_f64(M, N, K, b.alpha[p], dA, K, dB, N, b.beta[p], dC, N, cfg=cfg)
        torch.cuda.synchronize()
        got, _ = b.result(p)
        assert np.array_equal(got, dC.cpu().numpy()), (p, cfg)


def test_batched_graph_replay(alp, orc):
    import torch
    shapes = inputs.shapes(inputs.workload_seed("batched_4096"), 60, 16, 200)
    b = Batch(shapes, 5400, betas=np.zeros(60))
    ws = alp.alp_gemm_batched_workspace(b.count, b.hM, b.hN, b.hK)
    work = torch.empty(ws, dtype=torch.uint8, device="cuda")
    g = alp.alp_batched_graph_create(*b.args(), work, ws)
    try:
        for _ in range(2):      # beta = 0: replays give the same result
            alp.alp_batched_graph_launch(g)
            torch.cuda.synchronize()
            check_against_oracle(orc, b)
    finally:
        alp.alp_batched_graph_destroy(g)
