#!/usr/bin/env python3
"""FP64-accurate GEMM throughput on one GB300 (and N independent replicas).

Workload (default): C = alpha*A*B + beta*C with M = N = K = 8192, FP64
row-major operands u * 2^e (u uniform in [-1,1), e uniform in [-phi, phi],
phi = 0), alpha = 1, beta = 0, computed by the emulated FP64 path's modular
scheme (ALP_SLICE_BF16_CRT: the operands rounded to k-bit integers per row and
column, their exact product from residues modulo n moduli, one tensor-core
product per modulus); n is the library's automatic count for these operands
(alp_emul_crt_choose; 15 for phi = 0).
One step = one full emulated GEMM: B's column exponent scan, A's row scan and
residue split in one kernel, B's residue split, and the tensor-core residue
products with the Chinese remainder reconstruction in the same persistent
launch (the tiles of the last wave reconstructed by a small launch after it)
-- the same kernels alp_gemm_f64_emul launches, issued stage by stage so that
CUDA events can bracket each.  Inputs (1.5 GB) are larger than L2, so no flush is
needed between steps.

Beside the headline, in the same JSON line: the end-to-end call with host
buffers; the native DMMA kernel and the FP64 peak probes (with the vendor FP64
GEMM timed as a comparison); per phi in {0, 8, 32}, the errors of the native
kernel and of 13..16 moduli against the long-double oracle on sampled rows,
the smallest count no worse than native on both measures, its throughput and
the automatic count's, and the digit scheme's errors and throughput for 3..8
slices; a short native size scan (default and autotuned
config); the batched variable-size GEMM (4096 problems) against loops of
single-problem launches; and the CPU oracle's own throughput.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl alp|reference]

Under torchrun (N > 1) every rank runs the same replica on its own GPU
(the paths share nothing across GPUs); the slowest rank's time counts.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "FP64-accurate GEMM TFLOP/s (native vs emulated) and % of peak at N=8192"
UNIT = "TFLOP/s"
NOMINAL_BF16_TFLOPS = 2250.0   # dense bf16 tensor rate of one GB300 (nominal)
KERNEL_SOURCES = ("paper_1706_10086_gb300/csrc/emul_gemm.cu", "paper_1706_10086_gb300/csrc/tc.cuh",
                  "paper_1706_10086_gb300/csrc/emul.cuh", "paper_1706_10086_gb300/csrc/crt.cuh",
                  "paper_1706_10086_gb300/csrc/crt_rec.cuh",
                  "paper_1706_10086_gb300/csrc/emul_split.cuh")
TRAFFIC_PROFILES = "profiles/emul_*_8192_*.md"
# slice kinds of alp_gemm_f64_emul: name -> (enum value, digit pairs for s slices)
KINDS = {"bf16": (1, lambda s: s * (s + 1) // 2), "bf16_b8": (2, lambda s: s * (s + 1) // 2),
         "bf16_b8_trim": (3, lambda s: s * (s - 1) // 2 + 2), "bf16_crt": (4, lambda s: s)}


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("alp", "reference"), default="alp")
    ap.add_argument("--n", type=int, default=8192)
    ap.add_argument("--nslices", type=int, default=None,
                    help="moduli for bf16_crt (default 0: the library's automatic count for "
                         "the operands, 15 for the default uniform inputs), digit slices for "
                         "the other kinds (default 7)")
    ap.add_argument("--kind", choices=tuple(KINDS), default="bf16_crt",
                    help="scheme: bf16 (7-bit digits, up to 8 slices), bf16_b8 (8-bit, "
                         "up to 7), bf16_b8_trim (8-bit, last group keeps only its two "
                         "leading-digit pairs), bf16_crt (residues modulo 4..16 moduli, one "
                         "product each)")
    ap.add_argument("--phi", type=int, default=0)
    ap.add_argument("--oracle-rows", type=int, default=32,
                    help="rows of each 8192^3 product the long-double oracle computes for the "
                         "accuracy legs (also the CPU baseline's sample)")
    ap.add_argument("--no-native", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true",
                    help="skip the oracle: no accuracy legs and no CPU baseline")
    ap.add_argument("--no-scan", action="store_true", help="skip the native size scan leg")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched GEMM leg")
    ap.add_argument("--workload", choices=("emul8192", "batched", "native_scan", "sgemm8192"),
                    default="emul8192",
                    help="emul8192 (default, the headline and every leg), batched (4096 "
                         "variable-size problems alone), native_scan (native FP64 GEMM at N = "
                         "1024..16384 alone) or sgemm8192 (emulated FP32 GEMM, 3 slices of "
                         "8-bit digits, against the vendor FP32 GEMM)")
    ap.add_argument("--count", type=int, default=4096)
    ap.add_argument("--no-tune", action="store_true",
                    help="batched: keep the default class tiles instead of autotuning them")
    ap.add_argument("--profile", action="store_true",
                    help="timed steps only (no other leg): for ncu")
    a = ap.parse_args()
    if a.nslices is None:
        a.nslices = 0 if a.kind == "bf16_crt" else 7
    if a.profile:
        a.no_native = a.no_e2e = a.no_cpu = a.no_scan = a.no_batched = True
    return a


def dist_info():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def aggregate_over_ranks(local_ms: float, local_units: float, dist=None, device=None):
    """Whole-job throughput of N replicas: every rank's elapsed time is reduced
    with MAX and its work with SUM, so value = total units / slowest rank's time.
    Returns (max_ms, total_units).  Without a process group: the local values."""
    if dist is None or not dist.is_available() or not dist.is_initialized():
        return local_ms, local_units
    import torch
    t = torch.tensor([local_ms], dtype=torch.float64, device=device)
    u = torch.tensor([local_units], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, \
            "fallback"


def kernel_source_hash():
    h = hashlib.sha256()
    for p in KERNEL_SOURCES:
        with open(os.path.join(ROOT, p), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def profiled_values(workload):
    """The `- key: value` lines of the committed ncu summary taken on the
    current kernel source and this workload ({} if there is none)."""
    import glob
    for path in sorted(glob.glob(os.path.join(ROOT, TRAFFIC_PROFILES))):
        vals = {}
        for line in open(path).read().splitlines():
            if ":" in line and line.strip().startswith("- "):
                k, v = line.strip()[2:].split(":", 1)
                vals[k.strip()] = v.strip().strip("`")
        if (vals.get("kernel_source_hash") == kernel_source_hash()
                and vals.get("workload") == workload):
            return vals
    return {}


def profiled_traffic(workload):
    """DRAM bytes per launch of the tensor-core kernel from a committed ncu
    summary taken on the current kernel source and this workload; else None."""
    try:
        return float(profiled_values(workload)["dram_bytes_per_launch_full_size"])
    except (KeyError, ValueError):
        return None


def profiled_tensor_active(workload):
    """sm__pipe_tensor_cycles_active (% of the hardware peak) from the same
    summary, or None."""
    try:
        return float(profiled_values(workload)["sm__pipe_tensor_cycles_active"].split()[0])
    except (KeyError, ValueError, IndexError):
        return None


class ClockSampler:
    """nvidia-smi samples of the SM clock and throttle reasons during a region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        reasons = sorted({names[i] for _, _, r in rows for i, v in enumerate(r) if v == "Active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows),
                "sm_max_mhz": max(r[1] for r in rows), "reasons": reasons,
                "samples": len(rows)}


def oracle_rows(n, count):
    """Rows of an n x n product the oracle computes: `count` evenly spaced,
    first and last included."""
    import numpy as np
    return np.unique(np.linspace(0, n - 1, count).round().astype(np.int64))


def workload_name(n, s, kind, phi):
    return f"emulated_dgemm_{n}_{kind}x{s}slices_phi{phi}"


def make_inputs(torch, n, phi, seed, device):
    g = torch.Generator(device=device)
    g.manual_seed(seed)

    def mat():
        u = torch.rand(n, n, dtype=torch.float64, device=device, generator=g) * 2 - 1
        if phi == 0:
            return u
        e = torch.randint(-phi, phi + 1, (n, n), device=device, generator=g,
                          dtype=torch.int32).to(torch.float64)
        return torch.ldexp(u, e)
    return mat(), mat()


def product_roofline(pairs, M, N, K, s, crt, kern_ms, region_ms, clk, workload):
    """Roofline of the tensor-core product kernel: algorithmic flops per launch
    (pairs x 2MNK) over its average event-timed duration, against the measured
    bf16 peak.  For the modular scheme the timed stage is the fused launch
    (products with the reconstruction in the kernel's own warps, and the tail
    tiles' reconstruction after it), so its flops rate counts only the
    products.  The timed region lasts well under a second, so the burst figure
    is the denominator; the sustained one and the nominal rate are given
    beside it, and a clock-normalised fraction (the kernel's flops per SM clock
    over the peak's, each at its own median SM clock) separates clock from
    kernel.  DRAM traffic comes from a committed ncu summary of this kernel
    source and workload (null otherwise), next to the algorithmic bytes:
    operand slices read once (2 bytes per entry of A and B per product) and
    the per-product sums written once (4 bytes per group sum for the digit
    schemes; for the modular scheme 1 byte per entry of C per modulus, read
    back once by the reconstruction, and C written once)."""
    peaks, peak_kind = load_peaks()
    peak = float(peaks.get("bf16_tflops", 1900.0))
    sustained = float(peaks.get("bf16_tflops_sustained", peak))
    achieved = pairs * 2.0 * M * N * K / (kern_ms * 1e-3) / 1e12
    traffic = profiled_traffic(workload)
    # modular scheme: the fused launch also reads the residue bytes back and
    # writes C (8 bytes per entry; beta = 0 in the bench)
    alg_bytes = (2.0 * s * (M + N) * K + 2.0 * s * M * N + 8.0 * M * N if crt
                 else 2.0 * s * (M + N) * K + 4.0 * s * M * N)
    peak_mhz = (peaks.get("clocks_under_load") or {}).get("sm_mhz_median")
    run_mhz = clk.get("sm_mhz")
    clock_frac = (achieved / run_mhz) / (peak / peak_mhz) if peak_mhz and run_mhz else None
    kernel = ("emul_crt_fused_pair_kernel (tcgen05 bf16 residue products; C reconstructed by "
              "its own warps) + crt_tail_recombine_kernel" if crt else
              "emul_gemm_pair_kernel (tcgen05 bf16 digit-slice products)")
    return {"bound": "tensor", "kernel": kernel,
            "achieved": round(achieved, 1), "peak": peak, "unit": "TFLOP/s",
            "frac": round(achieved / peak, 4),
            "peak_source": f"bf16_tflops (burst) of MEASURED_PEAKS.json ({peak_kind}); the "
                           f"timed region is {region_ms / 1e3:.2f} s",
            "sustained_peak": sustained, "frac_of_sustained": round(achieved / sustained, 4),
            "clock_normalised_frac": round(clock_frac, 4) if clock_frac else None,
            "peak_sm_mhz": peak_mhz, "run_sm_mhz": run_mhz,
            "algorithmic_flops_per_launch": pairs * 2.0 * M * N * K,
            "kernel_ms": round(kern_ms, 3),
            "traffic": traffic, "algorithmic_bytes_per_launch": alg_bytes,
            "dram_ratio": round(traffic / alg_bytes, 3) if traffic else None,
            "nominal_peak": NOMINAL_BF16_TFLOPS,
            "frac_of_nominal": round(achieved / NOMINAL_BF16_TFLOPS, 4),
            "tensor_active_pct_ncu": profiled_tensor_active(workload)}


def errors_vs_oracle(got_rows, ref, absAB):
    """Largest componentwise error |dC| / (|A||B|) in units of 2^-53 and
    normwise ||dC||_F / ||C||_F of result rows against oracle rows."""
    import numpy as np
    d = np.abs(got_rows - ref)
    return {"max_componentwise_u": float(np.max(d / np.maximum(absAB, 1e-300)) / 2.0 ** -53),
            "normwise": float(np.linalg.norm(d) / np.linalg.norm(ref))}


def no_worse(e, nat):
    return (e["max_componentwise_u"] <= nat["max_componentwise_u"]
            and e["normwise"] <= nat["normwise"])


def time_calls(torch, stream, fn, reps):
    """Average ms of `reps` calls after one untimed call (CUDA events)."""
    fn()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def accuracy_leg(args, torch, alp, dev, stream, native_ms):
    """Per phi in {0, 8, 32}: the long-double oracle on sampled rows of the
    8192^3 product (u 2^e entries, alpha = 1, beta = 0); the native kernel's
    and 13..16 moduli's errors against it; the smallest count no worse than
    native on both measures and its throughput; the automatic count; and the
    digit scheme's (ALP_SLICE_BF16, 7-bit digits) errors and throughput for 3..8
    slices.  Returns (list of per-phi objects, CPU baseline object)."""
    import numpy as np

    import oracle
    oracle.build()
    n = args.n
    M = N = K = n
    rows = oracle_rows(n, args.oracle_rows)
    thr = os.cpu_count() or 1
    crt = alp.ALP_SLICE_BF16_CRT
    cpu_s, cpu_flops = 0.0, 0.0
    ws16 = alp.alp_gemm_f64_emul_workspace(M, N, K, 16, crt)
    work = torch.empty(ws16, dtype=torch.uint8, device=dev)
    dig = alp.ALP_SLICE_BF16
    wsd = alp.alp_gemm_f64_emul_workspace(M, N, K, 8, dig)
    workd = torch.empty(wsd, dtype=torch.uint8, device=dev)
    C = torch.empty(n, n, dtype=torch.float64, device=dev)
    out = []
    for phi in (0, 8, 32):
        A, B = make_inputs(torch, n, phi, 1706 + 2 + phi, dev)
        hA = A[torch.from_numpy(rows).to(dev)].cpu().numpy()
        hB = B.cpu().numpy()
        t0 = time.perf_counter()
        ref = oracle.gemm(1.0, hA, hB, 0.0, nthreads=thr)
        cpu_s += time.perf_counter() - t0
        cpu_flops += 2.0 * len(rows) * N * K
        # |A||B| on the sampled rows, from the native kernel on |A|, |B|
        absA = torch.from_numpy(np.abs(hA)).to(dev)
        absB = B.abs()
        absAB = torch.empty(len(rows), N, dtype=torch.float64, device=dev)
        alp.alp_gemm_f64(len(rows), N, K, 1.0, absA, K, absB, N, 0.0, absAB, N, stream=stream)
        torch.cuda.synchronize()
        absAB = absAB.cpu().numpy()
        del absA, absB
        alp.alp_gemm_f64(M, N, K, 1.0, A, K, B, N, 0.0, C, N, stream=stream)
        torch.cuda.synchronize()
        nat = errors_vs_oracle(C[torch.from_numpy(rows).to(dev)].cpu().numpy(), ref, absAB)
        emu = {}
        for nm in (13, 14, 15, 16):
            alp.alp_gemm_f64_emul(M, N, K, 1.0, A, K, B, N, 0.0, C, N, nm, crt, work, ws16,
                                  stream)
            torch.cuda.synchronize()
            emu[nm] = errors_vs_oracle(C[torch.from_numpy(rows).to(dev)].cpu().numpy(), ref,
                                       absAB)
        ok = [nm for nm in sorted(emu) if no_worse(emu[nm], nat)]
        n_min = ok[0] if ok else None
        n_auto, pred = alp.alp_emul_crt_choose(0, 0, M, N, K, A, K, B, N, work, ws16, stream)
        assert alp.alp_get_device_error(stream) == alp.ALP_OK
        flops = 2.0 * M * N * K

        def tflops(nm, kind=crt, wk=work):
            ws = alp.alp_gemm_f64_emul_workspace(M, N, K, nm, kind)
            ms = time_calls(torch, stream, lambda: alp.alp_gemm_f64_emul(
                M, N, K, 1.0, A, K, B, N, 0.0, C, N, nm, kind, wk, ws, stream), 5)
            return round(flops / (ms * 1e-3) / 1e12, 3)
        digits = {}
        for sd in range(3, 9):
            alp.alp_gemm_f64_emul(M, N, K, 1.0, A, K, B, N, 0.0, C, N, sd, dig, workd, wsd,
                                  stream)
            torch.cuda.synchronize()
            digits[sd] = errors_vs_oracle(C[torch.from_numpy(rows).to(dev)].cpu().numpy(), ref,
                                          absAB)
            digits[sd]["tflops"] = tflops(sd, dig, workd)
        ok_d = [sd for sd in sorted(digits) if no_worse(digits[sd], nat)]
        row = {"phi": phi, "rows_sampled": int(len(rows)),
               "native": nat, "native_tflops": round(flops / (native_ms * 1e-3) / 1e12, 4)
               if native_ms else None,
               "emulated": {str(k): v for k, v in emu.items()},
               "smallest_n_no_worse_than_native": n_min,
               "tflops_at_smallest_n": tflops(n_min) if n_min else None,
               "auto_n": n_auto, "auto_predicted_componentwise_u": round(pred[0], 4),
               "auto_predicted_normwise_ratio_to_native": round(pred[1], 4),
               "auto_no_worse_than_native": no_worse(emu[n_auto], nat) if n_auto in emu
               else None,
               "tflops_at_auto_n": tflops(n_auto),
               "digit_slices": {"kind": "bf16 (7-bit digits, s(s+1)/2 products)",
                                "by_slices": {str(k): v for k, v in digits.items()},
                                "smallest_s_no_worse_than_native": ok_d[0] if ok_d else None}}
        out.append(row)
        del A, B, hB
    del work, workd, C
    cpu = {"value": cpu_flops / cpu_s / 1e12, "unit": UNIT, "cores": thr, "kind": "oracle",
           "sample": f"{len(rows)} rows of each of three {n}^3 products (phi = 0, 8, 32; "
                     f"long-double triple loop, {cpu_s:.1f} s, {os.cpu_count()} host cores)"}
    return out, cpu


def native_leg(args, torch, alp, A, B, dev, stream):
    """The native DMMA kernel at alpha = 1.5, beta = 0.5 on the same operands,
    against the FP64 peak probes (every DMMA shape and DFMA); the vendor FP64
    GEMM (torch.matmul on float64) timed beside it as a comparison only."""
    n = args.n
    C2 = torch.rand(n, n, dtype=torch.float64, device=dev) * 2 - 1
    nat_ms = time_calls(torch, stream, lambda: alp.alp_gemm_f64(
        n, n, n, 1.5, A, n, B, n, 0.5, C2, n, stream=stream), 2)
    flops = 2.0 * n ** 3
    nat_tf = flops / (nat_ms * 1e-3) / 1e12
    probes = {name: round(alp.alp_probe_fp64_peak(kind, 20000, 2, 256, stream), 4)
              for kind, name in ((0, "dmma_m16n8k4"), (2, "dmma_m16n8k8"),
                                 (3, "dmma_m16n8k16"), (1, "dfma"))}
    best = max(probes["dmma_m16n8k4"], probes["dmma_m16n8k8"], probes["dmma_m16n8k16"])
    vend_ms = time_calls(torch, stream, lambda: torch.matmul(A, B, out=C2), 2)
    return {"tflops": round(nat_tf, 4), "ms": round(nat_ms, 2),
            "roofline": {"bound": "fp64_dmma", "achieved": round(nat_tf, 4), "peak": best,
                         "unit": "TFLOP/s", "frac": round(nat_tf / best, 4),
                         "peak_source": "the fastest of the FP64 MMA probes measured in this "
                                        "run (alp_probe_fp64_peak, chains on all SMs)"},
            "fp64_probes_tflops": probes,
            "vendor_fp64_gemm": {"tflops": round(flops / (vend_ms * 1e-3) / 1e12, 4),
                                 "ms": round(vend_ms, 2),
                                 "note": "torch.matmul on float64 (a comparison only)"},
            "vs_vendor": round(vend_ms / nat_ms, 4)}, nat_ms


def run_alp(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_1706_10086_gb300 import alp

    ws, rank, local = dist_info()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if ws > 1:
        dist.init_process_group("nccl", device_id=dev)
    n, s, phi = args.n, args.nslices, args.phi
    kind, pairs_of = KINDS[args.kind]
    M = N = K = n
    seed = 1706 + 2
    A, B = make_inputs(torch, n, phi, seed, dev)
    C = torch.empty(n, n, dtype=torch.float64, device=dev)
    alpha, beta = 1.0, 0.0
    stream = torch.cuda.current_stream(dev)
    auto = kind == alp.ALP_SLICE_BF16_CRT and s == 0
    if auto:
        # the library's automatic modulus count for these operands (outside
        # the timed region; the timed step then issues the stages with it)
        wsa = alp.alp_gemm_f64_emul_workspace(M, N, K, 0, kind)
        worka = torch.empty(wsa, dtype=torch.uint8, device=dev)
        s, _ = alp.alp_emul_crt_choose(0, 0, M, N, K, A, K, B, N, worka, wsa, stream)
        del worka
    # workspace carved exactly as alp_gemm_f64_emul does
    kpad = (K + 63) // 64 * 64
    ldg = (N + 255) // 256 * 256
    da = torch.empty(s * M * kpad, dtype=torch.bfloat16, device=dev)
    db = torch.empty(s * N * kpad, dtype=torch.bfloat16, device=dev)
    # int32 group sums, or one byte per residue for the modular scheme
    G = torch.empty(s * M * ldg * (1 if kind == alp.ALP_SLICE_BF16_CRT else 4),
                    dtype=torch.uint8, device=dev)
    e = torch.empty(M, dtype=torch.int32, device=dev)
    f = torch.empty(N, dtype=torch.int32, device=dev)
    crt = kind == alp.ALP_SLICE_BF16_CRT
    sched_bytes = alp.alp_emul_products_recombine_crt_workspace(M, N) if crt else 0
    sched = torch.empty(max(sched_bytes, 4), dtype=torch.uint8, device=dev)
    # the stages alp_gemm_f64_emul launches for this kind and a given count:
    # the modular scheme scans A's rows inside A's split
    if crt:
        stage_names = ("scan_cols", "scan_split_A", "split_B", "products_recombine")
        # scan cols (2), scan+split A, split B, products with the reconstruction,
        # the tail tiles' reconstruction
        launches_per_step = 6
    else:
        stage_names = ("scan_rows", "scan_cols", "split_A", "split_B", "slice_products",
                       "recombine")
        launches_per_step = 7   # scan rows, scan cols (2), split A, split B, products, recombine
    nev = len(stage_names) + 1

    def step(ev=None):
        # ev: events bracketing the stages (None: no timing)
        it = iter(ev) if ev is not None else None
        rec = (lambda: next(it).record(stream)) if ev is not None else (lambda: None)
        rec()
        if crt:
            alp.alp_emul_exponents(N, K, B, N, 1, f, stream)
            rec()
            alp.alp_emul_scan_split_rows(M, K, A, K, e, s, kind, da, kpad, stream)
            rec()
        else:
            alp.alp_emul_exponents(M, K, A, K, 0, e, stream)
            rec()
            alp.alp_emul_exponents(N, K, B, N, 1, f, stream)
            rec()
            alp.alp_emul_split(M, K, A, K, 0, e, s, kind, da, kpad, stream)
            rec()
        alp.alp_emul_split(N, K, B, N, 1, f, s, kind, db, kpad, stream)
        rec()
        if crt:
            alp.alp_emul_products_recombine_crt(M, N, K, s, da, db, kpad, G, ldg, e, f, alpha,
                                                beta, C, N, sched, sched_bytes, stream)
            rec()
        else:
            alp.alp_emul_slice_products(M, N, K, s, kind, da, db, kpad, G, ldg, stream)
            rec()
            alp.alp_emul_recombine(M, N, s, kind, G, ldg, e, f, alpha, beta, C, N, stream)
            rec()

    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()
    assert alp.alp_get_device_error(stream) == alp.ALP_OK

    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(nev)] for _ in range(args.steps)]
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    for i in range(args.steps):
        step(ev[i])
    t_end.record(stream)
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    clk = clocks.stop()
    total_ms = t_start.elapsed_time(t_end)
    step_ms = [ev[i][0].elapsed_time(ev[i][nev - 1]) for i in range(args.steps)]
    kp = stage_names.index("products_recombine" if crt else "slice_products")
    kern_ms = [ev[i][kp].elapsed_time(ev[i][kp + 1]) for i in range(args.steps)]
    stage_ms = {nm: round(statistics.median(ev[i][k].elapsed_time(ev[i][k + 1])
                                            for i in range(args.steps)), 4)
                for k, nm in enumerate(stage_names)}
    assert alp.alp_get_device_error(stream) == alp.ALP_OK
    flops_step = 2.0 * M * N * K
    total_ms, total_flops = aggregate_over_ranks(total_ms, args.steps * flops_step,
                                                 dist if ws > 1 else None, dev)
    value = total_flops / (total_ms * 1e-3) / 1e12
    pairs = pairs_of(s)
    kern_avg = statistics.mean(kern_ms)
    roofline = product_roofline(pairs, M, N, K, s, kind == alp.ALP_SLICE_BF16_CRT, kern_avg,
                                total_ms, clk, workload_name(n, s, args.kind, phi))

    out = {"metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": ws,
           "steps": args.steps, "warmup": max(3, args.warmup),
           "ms_per_step": round(total_ms / args.steps, 3), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "bf16",
           "data": "synthetic (seeded torch generator on the GPU; u*2^e, u~U[-1,1), e~U{-phi..phi})",
           "config": {"workload": workload_name(n, s, args.kind, phi), "M": M, "N": N,
                      "K": K, "nslices": s, "slice_kind": args.kind, "digit_pairs": pairs,
                      "nslices_from": "automatic count (alp_emul_crt_choose)" if auto
                      else "--nslices",
                      "phi": phi, "alpha": alpha, "beta": beta,
                      "result_dtype": "f64", "parallelism": f"replicas{ws}",
                      "l2": "inputs 1.5 GB > 129 MB L2; no flush"},
           "step_ms_median": round(statistics.median(step_ms), 3),
           "stage_ms_median": stage_ms,
           "roofline": roofline, "gpu_launches": launches_per_step * args.steps,
           "clocks": clk}

    if args.profile:
        print(json.dumps(out), flush=True)
        return
    # public single-call API on the same device buffers (same kernels, one call)
    wsb = alp.alp_gemm_f64_emul_workspace(M, N, K, s, kind)
    work = torch.empty(wsb, dtype=torch.uint8, device=dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    alp.alp_gemm_f64_emul(M, N, K, alpha, A, K, B, N, beta, C, N, s, kind, work, wsb, stream)
    e0.record(stream)
    for _ in range(3):
        alp.alp_gemm_f64_emul(M, N, K, alpha, A, K, B, N, beta, C, N, s, kind, work, wsb,
                              stream)
    e1.record(stream)
    torch.cuda.synchronize()
    out["api_call_ms"] = round(e0.elapsed_time(e1) / 3, 3)
    del da, db, G

    if not args.no_e2e:
        # end to end through the public call with host buffers: every step copies
        # A and B from pinned host memory, runs alp_gemm_f64_emul and copies C
        # back, all inside the timed region.  Uploads and downloads run on two
        # streams of their own (the link carries both directions at once) with
        # two sets of device operands, so step i+1's upload and step i-1's
        # download overlap step i's GEMM.
        hA = A.cpu().pin_memory()
        hB = B.cpu().pin_memory()
        hC = torch.empty(n, n, dtype=torch.float64).pin_memory()
        sets = [(torch.empty_like(A), torch.empty_like(B), torch.empty_like(C)) for _ in range(2)]
        up = torch.cuda.Stream(dev)
        down = torch.cuda.Stream(dev)
        # three times the timed steps, so that the pipeline's fill (the first
        # upload) and drain (the last download) weigh less in the average
        ksteps = max(6, 3 * args.steps)

        def run_e2e(k):
            ev = lambda: torch.cuda.Event(enable_timing=True)
            h2d = [ev() for _ in range(k)]
            comp = [ev() for _ in range(k)]
            d2h = [ev() for _ in range(k)]
            t0, t1 = ev(), ev()
            t0.record(up)

            def upload(i):
                dA, dB, _ = sets[i % 2]
                if i >= 2:
                    up.wait_event(comp[i - 2])       # the set's previous GEMM has read it
                with torch.cuda.stream(up):
                    dA.copy_(hA, non_blocking=True)
                    dB.copy_(hB, non_blocking=True)
                h2d[i].record(up)
            upload(0)
            for i in range(k):
                if i + 1 < k:
                    upload(i + 1)
                dA, dB, dC = sets[i % 2]
                stream.wait_event(h2d[i])
                if i >= 2:
                    stream.wait_event(d2h[i - 2])    # the set's previous C is downloaded
                alp.alp_gemm_f64_emul(M, N, K, alpha, dA, K, dB, N, beta, dC, N, s, kind, work,
                                      wsb, stream)
                comp[i].record(stream)
                down.wait_event(comp[i])
                with torch.cuda.stream(down):
                    hC.copy_(dC, non_blocking=True)
                d2h[i].record(down)
            t1.record(down)                          # after the last download
            torch.cuda.synchronize()
            return t0.elapsed_time(t1) / k
        run_e2e(2)                       # warm-up
        e2e_ms = run_e2e(ksteps)
        assert alp.alp_get_device_error(stream) == alp.ALP_OK
        out["e2e"] = {"value": round(flops_step / (e2e_ms * 1e-3) / 1e12, 3), "unit": UNIT,
                      "ms_per_step": round(e2e_ms, 3), "steps": ksteps,
                      "h2d_bytes_per_step": int(hA.numel() * 8 + hB.numel() * 8),
                      "d2h_bytes_per_step": int(hC.numel() * 8),
                      "overlap": "uploads and downloads on two streams of their own, two "
                                 "operand sets; the first upload and the last download "
                                 "inside the region"}
        del sets

    if not args.no_e2e and alp.alp_host_access()[0]:
        # end to end with the operands left in host memory: the device reads
        # A and B and writes C through the host's page tables (NVLink-C2C on a
        # Grace host); no copies, one call per step
        hA2 = A.cpu().numpy()
        hB2 = B.cpu().numpy()
        hC2 = np.empty((n, n))
        ks = max(2, args.steps)
        call = lambda: alp.alp_gemm_f64_emul(M, N, K, alpha, hA2.ctypes.data, K, hB2.ctypes.data,
                                             N, beta, hC2.ctypes.data, N, s, kind, work, wsb,
                                             stream)
        call()
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(ks):
            call()
        e1.record(stream)
        torch.cuda.synchronize()
        assert alp.alp_get_device_error(stream) == alp.ALP_OK
        hd_ms = e0.elapsed_time(e1) / ks
        out["e2e_host_resident"] = {
            "value": round(flops_step / (hd_ms * 1e-3) / 1e12, 3), "unit": UNIT,
            "ms_per_step": round(hd_ms, 3), "steps": ks,
            "note": "A, B, C in pageable host memory, read and written by the kernels in place"}
        del hA2, hB2, hC2

    native_ms = None
    if not args.no_native:
        out["native"], native_ms = native_leg(args, torch, alp, A, B, dev, stream)
        out["native"]["emulated_speedup"] = round(value / ws / out["native"]["tflops"], 2)
    del A, B, C
    torch.cuda.empty_cache()
    if rank == 0 and ws == 1 and not args.no_cpu:
        # accuracy per phi against the long-double oracle on sampled rows; the
        # oracle's time on those rows is the CPU baseline
        out["accuracy_per_phi"], out["cpu_baseline"] = accuracy_leg(args, torch, alp, dev,
                                                                    stream, native_ms)
        torch.cuda.empty_cache()
        # the headline's own scheme and count at its phi, when the leg covers them
        head = [r for r in out["accuracy_per_phi"] if r["phi"] == phi]
        if kind == alp.ALP_SLICE_BF16_CRT and head and str(s) in head[0]["emulated"]:
            r = head[0]
            out["accuracy"] = {"reference": f"long-double oracle on {r['rows_sampled']} "
                                            "evenly spaced rows",
                               "nslices": s, "emulated": r["emulated"][str(s)],
                               "native": r["native"],
                               "no_worse_than_native": no_worse(r["emulated"][str(s)],
                                                                r["native"])}
    if rank == 0 and ws == 1 and not args.no_scan:
        out["native_scan"] = native_scan_leg(torch, alp, dev, stream, (4096, 8192))
        torch.cuda.empty_cache()
    if rank == 0 and ws == 1 and not args.no_batched:
        out["batched"] = batched_leg(args, torch, alp, dev, stream)
        torch.cuda.empty_cache()
    if ws > 1:
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(out), flush=True)


def run_reference(args):
    """The CPU oracle as the reference arm: K timed steps, each a bounded
    sample of rows of the same 8192^3 product, on the host cores."""
    ws, rank, _ = dist_info()
    if rank != 0:
        return
    import numpy as np

    import oracle
    from paper_1706_10086_gb300 import inputs
    oracle.build()
    n = args.n
    thr = os.cpu_count() or 1
    seed = inputs.workload_seed("emul_8192")
    B = inputs.uniform(seed, n * n, (n, n))
    rows_per_step = max(1, thr // 2)
    A_rows = inputs.uniform(seed, 0, (rows_per_step, n))
    for _ in range(max(1, args.warmup)):
        oracle.gemm(1.0, A_rows[:1], B, 0.0, nthreads=thr)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.gemm(1.0, A_rows, B, 0.0, nthreads=thr)
    dt = time.perf_counter() - t0
    flops = 2.0 * rows_per_step * n * n * args.steps
    v = flops / dt / 1e12
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": ws,
           "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": round(dt / args.steps * 1e3, 3), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64 (long double accumulation)",
           "data": "synthetic (seeded SplitMix64, uniform [-1,1))",
           "config": {"workload": workload_name(n, args.nslices, args.kind, args.phi),
                      "M": n, "N": n,
                      "K": n, "sample_rows_per_step": rows_per_step},
           "cpu_baseline": {"value": v, "unit": UNIT, "cores": thr, "kind": "oracle",
                            "sample": f"{rows_per_step} rows of the {n}^3 product per step"},
           "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def batched_problems(torch, alp, inputs, dev, count):
    """The batched workload's storage: sizes log-uniform in [16, 1024], one
    buffer per operand with 16-byte aligned matrices, device arrays of sizes,
    scalars, pointers and leading dimensions."""
    import numpy as np
    shapes = inputs.shapes(inputs.workload_seed("batched_4096"), count, 16, 1024)
    M, N, K = (np.ascontiguousarray(shapes[:, i]) for i in range(3))
    pad = lambda x: (x + 1) // 2 * 2
    offA = np.concatenate([[0], np.cumsum(pad(M * K))])
    offB = np.concatenate([[0], np.cumsum(pad(K * N))])
    offC = np.concatenate([[0], np.cumsum(pad(M * N))])
    g = torch.Generator(device=dev)
    g.manual_seed(inputs.workload_seed("batched_4096"))
    bufA = torch.rand(int(offA[-1]), dtype=torch.float64, device=dev, generator=g) * 2 - 1
    bufB = torch.rand(int(offB[-1]), dtype=torch.float64, device=dev, generator=g) * 2 - 1
    bufC = torch.rand(int(offC[-1]), dtype=torch.float64, device=dev, generator=g) * 2 - 1
    b = {"M": M, "N": N, "K": K, "bufA": bufA, "bufB": bufB, "bufC": bufC,
         "pA": bufA.data_ptr() + 8 * offA[:-1], "pB": bufB.data_ptr() + 8 * offB[:-1],
         "pC": bufC.data_ptr() + 8 * offC[:-1]}
    t = lambda a, dt=torch.int64: torch.tensor(np.asarray(a), dtype=dt, device=dev)
    b["dev"] = (count, t(M), t(N), t(K), t(np.full(count, 1.5), torch.float64), t(b["pA"]), t(K),
                t(b["pB"]), t(N), t(np.full(count, 0.5), torch.float64), t(b["pC"]), t(N), M, N,
                K)
    b["flops"] = float(np.sum(2.0 * M * N * K))
    return b


# Native configs the fair loop baseline chooses from per size class.
LOOP_CANDIDATES = ((64, 64, 16, 4, 4, 0), (64, 64, 32, 8, 4, 0), (64, 128, 16, 4, 4, 0),
                   (128, 128, 16, 8, 8, 0))


def batched_leg(args, torch, alp, dev, stream, tune=True):
    """4096 independent problems, M, N, K log-uniform in [16, 1024], alpha =
    1.5, beta = 0.5: one replay of the persistent batched CUDA graph (class
    tiles autotuned first, outside the timed region), against loops of
    single-problem native launches: with the default config on one stream, the
    same captured in a CUDA graph, and a fairer loop whose problems take the
    best of LOOP_CANDIDATES for their size class (timed per class) and run
    round-robin on four streams."""
    import numpy as np

    from paper_1706_10086_gb300 import inputs
    n = args.count
    b = batched_problems(torch, alp, inputs, dev, n)
    M, N, K, pA, pB, pC = b["M"], b["N"], b["K"], b["pA"], b["pB"], b["pC"]
    bufC0 = b["bufC"].clone()
    flops = b["flops"]
    tuned = None
    t0 = time.perf_counter()
    if tune:
        from paper_1706_10086_gb300 import tuning
        res = tuning.tune_batched_classes(M, N, K, pA, pB, pC, runs=2)
        tuned = {int(c): list(v[0]) for c, v in res.items()}
        b["bufC"].copy_(bufC0)
    tune_s = time.perf_counter() - t0
    ws = alp.alp_gemm_batched_workspace(n, M, N, K)
    work = torch.empty(ws, dtype=torch.uint8, device=dev)
    graph = alp.alp_batched_graph_create(*b["dev"], work, ws)

    def timed(fn, steps, warm):
        for _ in range(warm):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / steps

    ms_graph = timed(lambda: alp.alp_batched_graph_launch(graph, stream), max(3, args.steps // 2),
                     3)

    def loop(st=stream, cfgs=None, streams=None):
        for p in range(n):
            s_p = streams[p % len(streams)] if streams else st
            alp.alp_gemm_f64(int(M[p]), int(N[p]), int(K[p]), 1.5, int(pA[p]), int(K[p]),
                             int(pB[p]), int(N[p]), 0.5, int(pC[p]), int(N[p]),
                             cfg=cfgs[p] if cfgs is not None else None, stream=s_p)
    ms_loop = timed(loop, 1, 1)
    side = torch.cuda.Stream(dev)
    side.wait_stream(stream)
    gl = torch.cuda.CUDAGraph()
    with torch.cuda.graph(gl, stream=side):
        loop(side)
    stream.wait_stream(side)
    ms_loop_graph = timed(gl.replay, 1, 1)
    del gl
    # fairer loop: per size class the fastest candidate config, four streams
    cls = np.array([alp.alp_batched_class_of(int(m), int(q)) for m, q in zip(M, N)])
    best = {}
    for c in sorted(set(cls.tolist())):
        idx = np.where(cls == c)[0]

        def run_class(cfg, idx=idx):
            for p in idx:
                alp.alp_gemm_f64(int(M[p]), int(N[p]), int(K[p]), 1.5, int(pA[p]), int(K[p]),
                                 int(pB[p]), int(N[p]), 0.5, int(pC[p]), int(N[p]), cfg=cfg,
                                 stream=stream)
        times = {cfg: timed(lambda cfg=cfg: run_class(cfg), 1, 1) for cfg in LOOP_CANDIDATES}
        best[c] = min(times, key=lambda k: (times[k], k))
    cfgs = [best[c] for c in cls]
    streams = [torch.cuda.Stream(dev) for _ in range(4)]

    def fair():
        for st in streams:
            st.wait_stream(stream)
        loop(cfgs=cfgs, streams=streams)
        for st in streams:
            stream.wait_stream(st)
    ms_fair = timed(fair, 1, 1)
    alp.alp_batched_graph_destroy(graph)
    assert alp.alp_get_device_error(stream) == alp.ALP_OK
    tf = lambda ms: round(flops / (ms * 1e-3) / 1e12, 4)
    fp64_peak = alp.alp_probe_fp64_peak(0, 20000, 2, 256, stream)
    return {"workload": f"batched_dgemm_{n}_loguniform_16_1024", "count": n,
            "flops_per_step": flops, "alpha": 1.5, "beta": 0.5,
            "graph_ms": round(ms_graph, 3), "tflops": tf(ms_graph),
            "frac_of_fp64_dmma_probe": round(tf(ms_graph) / fp64_peak, 4),
            "class_tiles": tuned if tuned is not None else "defaults",
            "class_tuning_s": round(tune_s, 1),
            "loop_of_launches": {"ms": round(ms_loop, 3), "tflops": tf(ms_loop)},
            "loop_of_launches_graph": {"ms": round(ms_loop_graph, 3), "tflops": tf(ms_loop_graph)},
            "loop_tuned_per_class_4_streams": {
                "ms": round(ms_fair, 3), "tflops": tf(ms_fair),
                "configs": {str(c): list(v) for c, v in best.items()}},
            "speedup_vs_loop": round(ms_loop / ms_graph, 3),
            "speedup_vs_tuned_loop_4_streams": round(ms_fair / ms_graph, 3)}


def run_batched(args):
    """The batched leg alone, as its own JSON line."""
    import torch

    from paper_1706_10086_gb300 import alp
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)
    clocks = ClockSampler(0)
    clocks.start()
    res = batched_leg(args, torch, alp, dev, stream, tune=not args.no_tune)
    clk = clocks.stop()
    out = {"metric": "batched FP64 GEMM TFLOP/s", "value": res["tflops"], "unit": UNIT,
           "n_gpus": 1, "steps": args.steps, "warmup": max(3, args.warmup),
           "ms_per_step": res["graph_ms"], "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64",
           "data": "synthetic (seeded: sizes SplitMix64 log-uniform, entries torch generator)",
           "config": {"workload": res["workload"], "l2": "operands 4.6 GB > L2; no flush"},
           "batched": res, "gpu_launches": 2 * max(3, args.steps // 2), "clocks": clk}
    print(json.dumps(out), flush=True)


def native_scan_leg(torch, alp, dev, stream, sizes):
    """Native DGEMM size scan: square N, U[-1,1), alpha = 1.5, beta = 0.5; the
    library's default config (no tuned entry yet) and the autotuner's pick
    (alp_tune, exhaustive sweep), each timed on the full problem (best of 2
    after a warm-up, CUDA events)."""
    g = torch.Generator(device=dev)
    g.manual_seed(1706 + 1)
    peak = max(alp.alp_probe_fp64_peak(k, 20000, 2, 256, stream) for k in (0, 2, 3))
    rows = []
    for n in sizes:
        A = torch.rand(n, n, dtype=torch.float64, device=dev, generator=g) * 2 - 1
        B = torch.rand(n, n, dtype=torch.float64, device=dev, generator=g) * 2 - 1
        C = torch.rand(n, n, dtype=torch.float64, device=dev, generator=g) * 2 - 1
        res = {"N": n}

        def best_ms(cfg):
            alp.alp_gemm_f64(n, n, n, 1.5, A, n, B, n, 0.5, C, n, cfg=cfg, stream=stream)
            times = []
            for _ in range(2):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                alp.alp_gemm_f64(n, n, n, 1.5, A, n, B, n, 0.5, C, n, cfg=cfg, stream=stream)
                e1.record(stream)
                e1.synchronize()
                times.append(e0.elapsed_time(e1))
            return min(times)
        for name in ("default", "tuned"):
            cfg = None
            if name == "tuned":
                t0 = time.perf_counter()
                _, tuned, _ = alp.alp_tune(n, n, n, alp.ALP_PATH_NATIVE, alp.ALP_TUNE_EXHAUSTIVE)
                res["tune_s"] = round(time.perf_counter() - t0, 2)
                res["tuned_config"] = list(tuned.astuple())
                cfg = tuned
            ms = best_ms(cfg)
            tf = 2.0 * n ** 3 / (ms * 1e-3) / 1e12
            res[name] = {"ms": round(ms, 3), "tflops": round(tf, 4),
                         "frac_of_fp64_peak": round(tf / peak, 4)}
        rows.append(res)
        del A, B, C
    return {"fp64_peak_measured": round(peak, 4), "alpha": 1.5, "beta": 0.5, "rows": rows}


def run_native_scan(args):
    """Native DGEMM size scan at N = 1024 .. 16384, as its own JSON line."""
    import torch

    from paper_1706_10086_gb300 import alp
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    res = native_scan_leg(torch, alp, dev, stream, (1024, 2048, 4096, 8192, 16384))
    print(json.dumps({"metric": "native FP64 GEMM TFLOP/s, size scan", "unit": UNIT, **res}),
          flush=True)


def run_sgemm(args):
    """Emulated FP32 GEMM, M = N = K = 8192, u in [-1,1) as float, alpha = 1,
    beta = 0: one step = the scans, splits, tensor-core slice products and FP32
    recombination (the kernels alp_gemm_f32_emul launches, stage by stage).
    Beside it, the vendor library's FP32 GEMM (TF32 off) on the same operands,
    and both results' errors against the emulated FP64 product (8 slices of
    7-bit digits) rounded nowhere (compared in double)."""
    import torch

    from paper_1706_10086_gb300 import alp
    n = args.n
    s = 3
    kind = alp.ALP_SLICE_BF16_B8
    M = N = K = n
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    A64, B64 = make_inputs(torch, n, 0, 1706 + 4, dev)
    A, B = A64.float(), B64.float()
    A64, B64 = A.double(), B.double()          # the exact values of the float operands
    C = torch.empty(n, n, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)
    kpad = (K + 63) // 64 * 64
    ldg = (N + 255) // 256 * 256
    da = torch.empty(s * M * kpad, dtype=torch.bfloat16, device=dev)
    db = torch.empty(s * N * kpad, dtype=torch.bfloat16, device=dev)
    G = torch.empty(s * M * ldg, dtype=torch.int32, device=dev)
    e = torch.empty(M, dtype=torch.int32, device=dev)
    f = torch.empty(N, dtype=torch.int32, device=dev)

    def step(ev=None):
        rec = (lambda i: ev[i].record(stream)) if ev is not None else (lambda i: None)
        rec(0)
        alp.alp_emul_exponents_f32(M, K, A, K, 0, e, stream)
        alp.alp_emul_exponents_f32(N, K, B, N, 1, f, stream)
        alp.alp_emul_split_f32(M, K, A, K, 0, e, s, kind, da, kpad, stream)
        alp.alp_emul_split_f32(N, K, B, N, 1, f, s, kind, db, kpad, stream)
        rec(1)
        alp.alp_emul_slice_products(M, N, K, s, kind, da, db, kpad, G, ldg, stream)
        rec(2)
        alp.alp_emul_recombine_f32(M, N, s, kind, G, ldg, e, f, 1.0, 0.0, C, N, stream)
        rec(3)

    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()
    assert alp.alp_get_device_error(stream) == alp.ALP_OK
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(args.steps)]
    clocks = ClockSampler(0)
    clocks.start()
    time.sleep(0.3)
    torch.cuda.synchronize()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for i in range(args.steps):
        step(ev[i])
    t1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    total_ms = t0.elapsed_time(t1)
    kern_ms = statistics.mean(ev[i][1].elapsed_time(ev[i][2]) for i in range(args.steps))
    flops = 2.0 * M * N * K
    pairs = s * (s + 1) // 2
    peaks, peak_kind = load_peaks()
    peak = float(peaks.get("bf16_tflops", 1900.0))
    achieved = pairs * flops / (kern_ms * 1e-3) / 1e12
    # the vendor FP32 GEMM on the same float operands (a comparison, not this library)
    old = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = False
    Cv = A @ B
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(3):
        Cv = A @ B
    e1.record(stream)
    torch.cuda.synchronize()
    torch.backends.cuda.matmul.allow_tf32 = old
    vend_ms = e0.elapsed_time(e1) / 3
    # accuracy over the whole result against the FP64 emulated product of the
    # same (float) values, relative to |A||B| from the native FP64 kernel
    Cref = torch.empty(n, n, dtype=torch.float64, device=dev)
    ws8 = alp.alp_gemm_f64_emul_workspace(M, N, K, 8, alp.ALP_SLICE_BF16)
    work8 = torch.empty(ws8, dtype=torch.uint8, device=dev)
    alp.alp_gemm_f64_emul(M, N, K, 1.0, A64, K, B64, N, 0.0, Cref, N, 8, alp.ALP_SLICE_BF16,
                          work8, ws8, stream)
    del work8
    absAB = torch.empty_like(Cref)
    alp.alp_gemm_f64(M, N, K, 1.0, A64.abs(), K, B64.abs(), N, 0.0, absAB, N, stream=stream)
    torch.cuda.synchronize()
    u = 2.0 ** -24

    def errs(X):
        d = (X.double() - Cref).abs()
        return {"max_componentwise_u32": float((d / absAB).max()) / u,
                "normwise": float(torch.linalg.norm(d) / torch.linalg.norm(Cref))}
    out = {"metric": "FP32-accurate GEMM TFLOP/s (emulated on BF16 tensor cores) at N=8192",
           "value": round(flops * args.steps / (total_ms * 1e-3) / 1e12, 3), "unit": UNIT,
           "n_gpus": 1, "steps": args.steps, "warmup": max(3, args.warmup),
           "ms_per_step": round(total_ms / args.steps, 3), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "bf16",
           "data": "synthetic (seeded torch generator on the GPU, u~U[-1,1) as float)",
           "config": {"workload": f"emulated_sgemm_{n}_bf16_b8x{s}slices", "M": M, "N": N,
                      "K": K, "nslices": s, "slice_kind": "bf16_b8", "digit_pairs": pairs,
                      "l2": "inputs 0.5 GB > 129 MB L2; no flush"},
           "stage_ms_median": {
               "scans_and_splits": round(statistics.median(ev[i][0].elapsed_time(ev[i][1])
                                                           for i in range(args.steps)), 4),
               "slice_products": round(statistics.median(ev[i][1].elapsed_time(ev[i][2])
                                                         for i in range(args.steps)), 4),
               "recombine": round(statistics.median(ev[i][2].elapsed_time(ev[i][3])
                                                    for i in range(args.steps)), 4)},
           "roofline": {"bound": "tensor", "kernel": "emul_gemm_pair_kernel (tcgen05 bf16)",
                        "achieved": round(achieved, 1), "peak": peak, "unit": "TFLOP/s",
                        "frac": round(achieved / peak, 4),
                        "peak_source": f"bf16_tflops (burst) of MEASURED_PEAKS.json ({peak_kind})",
                        "algorithmic_flops_per_launch": pairs * flops,
                        "kernel_ms": round(kern_ms, 3), "traffic": None},
           "vendor_fp32": {"tflops": round(flops / (vend_ms * 1e-3) / 1e12, 3),
                           "ms": round(vend_ms, 3), "note": "torch.matmul FP32, TF32 off"},
           "accuracy": {"reference": "emulated FP64 product (8 slices of 7-bit digits)",
                        "emulated_fp32": errs(C), "vendor_fp32": errs(Cv)},
           "gpu_launches": 7 * args.steps, "clocks": clk}
    print(json.dumps(out), flush=True)


def main():
    args = parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batched":
        run_batched(args)
    elif args.workload == "native_scan":
        run_native_scan(args)
    elif args.workload == "sgemm8192":
        run_sgemm(args)
    else:
        run_alp(args)


if __name__ == "__main__":
    main()
