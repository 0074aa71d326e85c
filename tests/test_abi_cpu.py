"""The C-ABI library builds, loads and exports every symbol its headers
declare; host-side logic (config rules, argument checks) works without a GPU."""
import glob
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(alp_[a-z0-9_]+)\s*\(", text):
            names.add(m.group(1))
    return sorted(names)


def test_headers_declare_the_boundary():
    names = declared_symbols()
    for n in ("alp_gemm_f64", "alp_gemm_f64_emul", "alp_gemm_batched_varsize", "alp_tune",
              "alp_get_device_error", "alp_status_string"):
        assert n in names


def test_library_exports_every_declared_symbol(alp):
    out = subprocess.run(["nm", "-D", "--defined-only", alp.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\bT (alp_[a-z0-9_]+)", out))
    missing = [n for n in declared_symbols() if n not in exported]
    assert not missing, missing
    # and the binding knows them all
    assert set(declared_symbols()) <= set(alp._SIGS)


def test_status_strings(alp):
    assert alp.status_string(alp.ALP_OK) == "ALP_OK"
    for s in range(1, 7):
        assert alp.status_string(s).startswith("ALP_ERR_")


def test_table4_tile_cache_model(alp):
    """alp_config_smem_bytes for bm = bn = bk = T and one stage is 2 T^2 * 8,
    the DP tile cache K(S,T) of Eq. 3; every DP row printed in Table 4 matches."""
    units = {"B": 1, "KB": 1024, "MB": 1024 ** 2}
    n = 0
    for line in open(os.path.join(ROOT, "tests", "golden", "table4_tile_cache.txt")):
        if line.startswith("#") or not line.strip():
            continue
        arch, comp, prec, S, T, val, unit = line.split()
        S, T = int(S), int(T)
        printed = int(val) * units[unit]
        assert 2 * T * T * S == printed, line
        if S == 8:
            cfg = alp.alp_config(T, T, T, 2, 2, 1)
            assert alp.alp_config_smem_bytes(cfg) == printed, line
            n += 1
    assert n == 9


def test_config_rules(alp):
    P = alp.ALP_PATH_NATIVE
    n = alp.alp_config_count(P)
    assert 20 <= n <= 243
    seen = set()
    for i in range(n):
        c = alp.alp_config_at(P, i)
        assert alp.alp_config_valid(c, P)
        t = c.astuple()
        assert t not in seen
        seen.add(t)
        bm, bn, bk, tm, tn, st = t
        assert bm in (64, 128, 256) and bn in (64, 128, 256) and bk in (16, 32, 64)
        assert tm in (2, 4, 8) and tn in (2, 4, 8)
        thr = alp.alp_config_threads(c)
        assert thr == 32 * (1 + (bm // (8 * tm)) * (bn // (4 * tn))) and thr <= 1024
        assert alp.alp_config_smem_bytes(c) <= 227 * 1024
        assert alp.alp_config_smem_bytes(c) >= 2 * (bm + bn) * bk * 8
    # independent enumeration of the rule set: count the raw sweep, then filter
    count = 0
    for bm in (64, 128, 256):
        for bn in (64, 128, 256):
            for bk in (16, 32, 64):
                for tm in (2, 4, 8):
                    for tn in (2, 4, 8):
                        if alp.alp_config_valid((bm, bn, bk, tm, tn, 0), P):
                            count += 1
    assert count == n
    assert not alp.alp_config_valid((256, 256, 64, 8, 8, 0), P)     # one stage would not fit
    assert not alp.alp_config_valid((64, 64, 16, 2, 2, 0), P)       # 33 warps
    assert not alp.alp_config_valid((96, 64, 16, 4, 4, 0), P)
    with pytest.raises(alp.AlpError):
        alp.alp_config_at(P, n)


def test_emul_config_rules(alp):
    """Emulated-path configs: one block per 128 x 256 tile (bm 128, tm 1) or
    CTA pairs on 256 x 256 (bm 256, tm 2), raster groups 1..32.  No
    arrangement shares operand tiles between blocks through multicast loads."""
    E = alp.ALP_PATH_EMUL
    n = alp.alp_config_count(E)
    got = {alp.alp_config_at(E, i).astuple() for i in range(n)}
    groups = (1, 2, 4, 8, 16, 32)
    want = {(128, 256, 64, 1, 0, g) for g in groups}
    want |= {(256, 256, 64, 2, 0, g) for g in groups}
    assert got == want and n == len(want)
    assert all(alp.alp_config_valid(c, E) for c in want)
    for bad in ((256, 256, 64, 1, 0, 8), (256, 256, 64, 3, 0, 8), (128, 256, 64, 2, 0, 3),
                (128, 256, 64, 2, 0, 8),
                (128, 128, 64, 1, 0, 8), (128, 256, 32, 1, 0, 8), (128, 256, 64, 1, 1, 8)):
        assert not alp.alp_config_valid(bad, E), bad


def test_argument_errors_return_before_launch(alp):
    """Invalid arguments are reported synchronously, no GPU work involved."""
    E = alp.ALP_ERR_INVALID_ARG
    g = lambda *a: alp.alp_gemm_f64(*a, stream=0, raise_on_error=False)
    assert g(-1, 4, 4, 1.0, 8, 4, 8, 4, 0.0, 8, 4) == E
    assert g(4, 4, 4, 1.0, 8, 3, 8, 4, 0.0, 8, 4) == E           # lda < K
    assert g(4, 4, 4, 1.0, 8, 4, 8, 3, 0.0, 8, 4) == E           # ldb < N
    assert g(4, 4, 4, 1.0, 8, 4, 8, 4, 0.0, 8, 3) == E           # ldc < N
    assert g(4, 4, 4, 1.0, None, 4, 8, 4, 0.0, 8, 4) == E        # A read but NULL
    assert g(4, 4, 4, 1.0, 8, 4, 8, 4, 0.0, None, 4) == E        # C NULL
    assert g(4, 4, 4, 1.0, 12, 4, 8, 4, 0.0, 8, 4) == E          # misaligned double
    assert alp.alp_gemm_f64(4, 4, 4, 1.0, 8, 4, 8, 4, 0.0, 8, 4, cfg=(96, 64, 16, 4, 4, 0),
                            stream=0, raise_on_error=False) == E
    # M == 0 or N == 0: nothing to do, nothing read
    assert g(0, 4, 4, 1.0, None, 4, None, 4, 0.0, None, 4) == alp.ALP_OK
    assert g(4, 0, 4, 1.0, None, 4, None, 0, 0.0, None, 0) == alp.ALP_OK


def test_batched_classes_and_config(alp):
    assert alp.alp_batched_class_of(32, 32) == 0
    assert alp.alp_batched_class_of(33, 32) == 3
    assert alp.alp_batched_class_of(64, 65) == 5
    assert alp.alp_batched_class_of(1000, 1) == 6
    assert alp.alp_batched_class_of(65, 1000) == 8
    old = alp.alp_batched_get_class_config(4)
    try:
        alp.alp_batched_set_class_config(4, 32, 128, 32)
        assert alp.alp_batched_get_class_config(4) == (32, 128, 32)
        with pytest.raises(alp.AlpError):
            alp.alp_batched_set_class_config(4, 48, 64, 16)
        with pytest.raises(alp.AlpError):
            alp.alp_batched_set_class_config(9, 64, 64, 16)
    finally:
        alp.alp_batched_set_class_config(4, *old)
    import numpy as np
    hM = np.array([4, 5], dtype=np.int64)
    assert alp.alp_gemm_batched_workspace(2, hM, hM, hM) > 0
    assert alp.alp_gemm_batched_workspace(2, np.array([4, -1], dtype=np.int64), hM, hM) == 0


def _best_cut(s, k, trim=False):
    """Smallest largest piece (in digit pairs) over every cut of groups
    t = 2..s+1 (group t holds t-1 pairs; the trimmed last group 2) into at
    most k contiguous ranges."""
    import itertools
    w = list(range(1, s + 1))
    if trim:
        w[-1] = min(w[-1], 2)
    best = sum(w)
    for n in range(1, k + 1):
        for cuts in itertools.combinations(range(1, s), n - 1):
            bounds = (0,) + cuts + (s,)
            best = min(best, max(sum(w[a:b]) for a, b in zip(bounds, bounds[1:])))
    return best


def test_emul_tail_split(alp):
    """The last partial wave of the slice-product launch is cut into pieces
    that cover the groups once, in order, with the smallest possible largest
    piece (brute force over every cut)."""
    B7, B8T = alp.ALP_SLICE_BF16, alp.ALP_SLICE_BF16_B8_TRIM
    assert alp.alp_emul_tail_split(2048, 7, B7, 152) == (1976, [(2, 6), (7, 8)])
    assert alp.alp_emul_tail_split(32, 7, B7, 152) == (0, [(2, 4), (5, 6), (7, 7), (8, 8)])
    assert alp.alp_emul_tail_split(13 * 152, 7, B7, 152) == (13 * 152, [(2, 8)])   # full wave
    assert alp.alp_emul_tail_split(100, 7, B7, 152) == (100, [(2, 8)])   # 152 // 100 = 1 piece
    assert alp.alp_emul_tail_split(0, 7, B7, 152) == (0, [(2, 8)])
    # trimmed, 7 slices: groups t = 2..8 hold 1, 2, 3, 4, 5, 6 and 2 pairs; the
    # best cut into 4 pieces has 8 pairs in its largest piece
    assert alp.alp_emul_tail_split(32, 7, B8T, 152) == (0, [(2, 4), (5, 5), (6, 6), (7, 8)])
    for s, kind in [(s, B7) for s in range(2, 9)] + [(s, B8T) for s in range(3, 8)]:
        for tiles in (1, 5, 19, 38, 50, 75, 151, 152, 153, 300, 2048):
            for sms in (1, 8, 152, 160):
                n_full, pieces = alp.alp_emul_tail_split(tiles, s, kind, sms)
                r = tiles % sms or sms
                k = min(sms // r, s, 8)
                if k < 2 or r == sms:
                    assert (n_full, pieces) == (tiles, [(2, s + 1)])
                    continue
                assert n_full == tiles - r
                assert pieces[0][0] == 2 and pieces[-1][1] == s + 1
                assert all(a <= b for a, b in pieces)
                assert all(pieces[i][1] + 1 == pieces[i + 1][0] for i in range(len(pieces) - 1))
                assert 2 <= len(pieces) <= k
                trim = kind == B8T
                w = lambda t: 2 if trim and t == s + 1 else t - 1
                largest = max(sum(w(t) for t in range(a, b + 1)) for a, b in pieces)
                assert largest == _best_cut(s, k, trim), (s, kind, tiles, sms, pieces)
    with pytest.raises(alp.AlpError):
        alp.alp_emul_tail_split(10, 9, B7, 152)
    with pytest.raises(alp.AlpError):
        alp.alp_emul_tail_split(10, 8, B8T, 152)


def test_emul_tail_split_modular_scheme(alp):
    """With the modular kind every group is one product, so the best cut of s
    moduli into at most k pieces has ceil(s / k) in its largest piece."""
    CRT = alp.ALP_SLICE_BF16_CRT
    for s in range(4, 17):
        for tiles in (5, 38, 151, 153, 300):
            n_full, pieces = alp.alp_emul_tail_split(tiles, s, CRT, 152)
            r = tiles % 152 or 152
            k = min(152 // r, s, 8)
            if k < 2:
                assert pieces == [(2, s + 1)]
                continue
            assert n_full == tiles - r and pieces[0][0] == 2 and pieces[-1][1] == s + 1
            assert max(b - a + 1 for a, b in pieces) == -(-s // k)
    with pytest.raises(alp.AlpError):
        alp.alp_emul_tail_split(10, 17, CRT, 152)


# the moduli of the modular scheme, in the order the ABI documents them
CRT_MODULI = [256, 255, 253, 251, 247, 241, 239, 233, 229, 227, 223, 217, 211, 199, 197, 193]



def test_fused_schedule_workspace_covers_every_launch(alp):
    """alp_emul_products_recombine_crt_workspace (and the GEMM's workspace)
    holds the fused launch's schedule for any number of resident CTA pairs up
    to 128: the counter and, for each pair, one entry per item plus the end
    marker, with the items the tail split makes (whole tiles, then every
    tail tile's pieces)."""
    CRT = alp.ALP_SLICE_BF16_CRT
    for M, N in [(1, 1), (256, 256), (300, 200), (2560, 2560), (8192, 8192), (4096, 4100),
                 (19456, 256), (65536, 300)]:
        pair_tiles = ((M + 255) // 256) * ((N + 255) // 256)
        need_max = 0
        for P in (1, 2, 7, 64, 74, 76, 100, 128):
            for n in (4, 13, 15, 16):
                n_full, pieces = alp.alp_emul_tail_split(pair_tiles, n, CRT, P)
                items = n_full + (pair_tiles - n_full) * len(pieces)
                clusters = min(items, P)
                need_max = max(need_max, 4 * (1 + clusters * (items + 1)))
        ws = alp.alp_emul_products_recombine_crt_workspace(M, N)
        assert ws >= need_max, (M, N, ws, need_max)
        assert alp.alp_gemm_f64_emul_workspace(M, N, 64, 15, CRT) >= ws

def test_crt_moduli_and_bits_rule(alp):
    """The documented moduli are pairwise coprime, and alp_emul_crt_bits is the
    largest k <= 60 with K 2^(2k+1) <= Mn (1 - 2^-18), Mn their product (so
    |P| <= K 2^(2k) stays below Mn / 2 by at least Mn 2^-19)."""
    import math
    for i, a in enumerate(CRT_MODULI):
        for b in CRT_MODULI[i + 1:]:
            assert math.gcd(a, b) == 1
    for n in range(4, 17):
        Mn = math.prod(CRT_MODULI[:n])
        for K in (1, 2, 63, 1000, 1024, 8192, 8193, 32768, 65472):
            k = alp.alp_emul_crt_bits(K, n)
            assert 1 <= k <= 60
            lim = Mn - (Mn >> 18)
            assert K * 2 ** (2 * k + 1) <= lim
            assert k == 60 or K * 2 ** (2 * k + 3) > lim, (K, n, k)
    assert alp.alp_emul_crt_bits(65473, 16) == 0 and alp.alp_emul_crt_bits(65472, 16) == 54
    assert alp.alp_emul_crt_bits(100, 3) == 0 and alp.alp_emul_crt_bits(100, 17) == 0
    assert alp.alp_emul_crt_bits(8192, 15) == 51 and alp.alp_emul_crt_bits(8192, 14) == 48


def _stats_of(K, phi):
    """Expected statistics of rows (and columns) of K entries u 2^e, u uniform
    in [-1, 1), e uniform in [-phi, phi], scaled by the row maximum's 2^phi:
    S1 = K E|x|, S2 = K E x^2."""
    es = range(-phi, phi + 1)
    e1 = 0.5 * sum(2.0 ** (e - phi) for e in es) / len(es)
    e2 = sum(4.0 ** (e - phi) for e in es) / (3 * len(es))
    s1, s2 = K * e1, K * e2
    return [1 / s1 ** 2, s2 / s1 ** 2, 1 / s2] * 2


def test_crt_moduli_rule(alp):
    """The automatic-count rule (host only).  For K = 8192 and entries of one
    magnitude the predicted errors at 15 moduli (k = 51) are 0.25 u
    componentwise (g/sqrt(12) 2^2 K sqrt(2 (4/K^2)(4/(3K))), g = sqrt(2 ln
    8192^2)) and 0.10 of the native kernel normwise, inside the targets (half of
    0.045 sqrt(K) = 2.04 u, and 0.5), while 14 moduli (k = 48) predict 0.80 of
    native normwise: 15 is chosen.  Wider exponent ranges need more; an
    all-zero operand needs none beyond the minimum."""
    import math
    K = 8192
    n, (comp, norm) = alp.alp_emul_crt_moduli_rule(K, K, K, _stats_of(K, 0))
    g = math.sqrt(2 * math.log(K * K))
    want_comp = g / math.sqrt(12) * 4 * K * math.sqrt(2 * (4 / K ** 2) * (4 / (3 * K)))
    want_norm = 4 / (math.sqrt(12) * 0.311) * math.sqrt(2 * 3 / K)
    assert n == 15 and abs(comp / want_comp - 1) < 1e-12 and abs(norm / want_norm - 1) < 1e-12
    assert want_norm * 8 > 0.5                   # 14 moduli (k = 48) miss the normwise target
    assert alp.alp_emul_crt_bits(K, 15) == 51 and alp.alp_emul_crt_bits(K, 14) == 48
    counts = [alp.alp_emul_crt_moduli_rule(K, K, K, _stats_of(K, phi))[0] for phi in (0, 2, 8, 32)]
    assert counts == sorted(counts) and counts[-1] == 16, counts
    assert alp.alp_emul_crt_moduli_rule(K, K, K, [0.0] * 6)[0] == 4
    # larger statistics (a worse-conditioned operand) never lower the count
    base = _stats_of(K, 0)
    for f in (1.0, 4.0, 64.0, 1e4):
        assert alp.alp_emul_crt_moduli_rule(K, K, K, [v * f for v in base])[0] >= n
    assert alp.alp_emul_crt_moduli_rule(-1, K, K, base)[0] == 0
    assert alp.alp_emul_crt_moduli_rule(K, K, 70000, base)[0] == 0
