"""Host logic of bench.py (no GPU): the slice-kind table agrees with the ABI's
enum, the defaults select the modular scheme with 15 moduli, and the committed
ncu summaries parse into the roofline's traffic and tensor-activity fields."""
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
    assert (a.kind, a.nslices, a.n, a.gpus, a.impl) == ("bf16_crt", 15, 8192, 1, "alp")
    assert a.warmup >= 3
    monkeypatch.setattr(sys, "argv", ["bench.py", "--kind", "bf16_b8_trim"])
    assert bench.parse_args().nslices == 7
    monkeypatch.setattr(sys, "argv", ["bench.py", "--profile"])
    a = bench.parse_args()
    assert a.no_native and a.no_e2e and a.no_cpu
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
