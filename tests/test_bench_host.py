"""Host logic of bench.py (no GPU): the slice-kind table agrees with the ABI's
enum, the defaults select the modular scheme with the library's automatic
modulus count, the oracle rows and error measures, and the committed ncu
summaries parse into the roofline's traffic and tensor-activity fields."""
import glob
import os
import re
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    import bench
    return bench


def test_kinds_match_the_abi(alp):
    bench = _bench()
    assert bench.KINDS["bf16"][0] == alp.ALP_SLICE_BF16
    assert bench.KINDS["bf16_b8"][0] == alp.ALP_SLICE_BF16_B8
    assert bench.KINDS["bf16_b8_trim"][0] == alp.ALP_SLICE_BF16_B8_TRIM
    assert bench.KINDS["bf16_crt"][0] == alp.ALP_SLICE_BF16_CRT
    # tensor-core products per scheme
    assert bench.KINDS["bf16"][1](7) == 28 and bench.KINDS["bf16_b8_trim"][1](7) == 23
    assert bench.KINDS["bf16_crt"][1](15) == 15


def test_defaults(monkeypatch):
    bench = _bench()
    monkeypatch.setattr(sys, "argv", ["bench.py"])
    a = bench.parse_args()
    assert (a.kind, a.nslices, a.n, a.gpus, a.impl) == ("bf16_crt", 0, 8192, 1, "alp")
    assert a.warmup >= 3
    monkeypatch.setattr(sys, "argv", ["bench.py", "--kind", "bf16_b8_trim"])
    assert bench.parse_args().nslices == 7
    monkeypatch.setattr(sys, "argv", ["bench.py", "--profile"])
    a = bench.parse_args()
    assert a.no_native and a.no_e2e and a.no_cpu and a.no_scan and a.no_batched
    assert bench.workload_name(8192, 15, "bf16_crt", 0) == \
        "emulated_dgemm_8192_bf16_crtx15slices_phi0"


def test_committed_profiles_parse(monkeypatch):
    """Each product-kernel summary names its workload and source hash and gives
    the DRAM bytes per launch; with that hash current, the bench reads them."""
    bench = _bench()
    paths = sorted(glob.glob(os.path.join(ROOT, bench.TRAFFIC_PROFILES)))
    assert paths
    for path in paths:
        text = open(path).read()
        workload = re.search(r"- workload: `([^`]+)`", text).group(1)
        digest = re.search(r"- kernel_source_hash: `([0-9a-f]{16})`", text).group(1)
        total = int(re.search(r"- dram_bytes_per_launch_full_size: `(\d+)`", text).group(1))
        reads = int(re.search(r"- dram_bytes_read_per_launch: `(\d+)`", text).group(1))
        writes = int(re.search(r"- dram_bytes_write_per_launch: `(\d+)`", text).group(1))
        assert total == reads + writes
        monkeypatch.setattr(bench, "kernel_source_hash", lambda d=digest: d)
        assert bench.profiled_traffic(workload) == float(total)
        assert bench.profiled_traffic("no such workload") is None
        active = bench.profiled_tensor_active(workload)
        assert active is None or 0.0 < active <= 100.0
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "0" * 16)
    assert bench.profiled_traffic(workload) is None


def test_oracle_rows_and_error_measures():
    import numpy as np
    bench = _bench()
    r = bench.oracle_rows(8192, 32)
    assert len(r) == 32 and r[0] == 0 and r[-1] == 8191 and np.all(np.diff(r) > 0)
    ref = np.array([[1.0, -2.0], [4.0, 0.5]])
    absAB = np.array([[2.0, 4.0], [8.0, 1.0]])
    got = ref + np.array([[2.0 ** -52, 0.0], [0.0, -2.0 ** -53]])
    e = bench.errors_vs_oracle(got, ref, absAB)
    # |dC|/|A||B|: 2^-52/2 = 1 u and 2^-53/1 = 1 u
    assert e["max_componentwise_u"] == 1.0
    assert abs(e["normwise"] - np.linalg.norm([2.0 ** -52, 2.0 ** -53]) / np.linalg.norm(ref)) \
        < 1e-30
    nat = {"max_componentwise_u": 1.0, "normwise": e["normwise"]}
    assert bench.no_worse(e, nat)
    assert not bench.no_worse(e, {"max_componentwise_u": 0.5, "normwise": 1.0})
