"""Host-side helpers of bench.py (no GPU): the DRAM-traffic record keyed by the
kernel source's hash, the workload config both arms print, the fitted CPU-oracle
sample, and the NUMA CPU-list parser."""
import argparse
import hashlib
import os

import bench


def _args(**kw):
    a = dict(n=32768, gen="uniform", path="fp64", leaf=32, gpus=1, steps=3, warmup=3)
    a.update(kw)
    return argparse.Namespace(**a)


def test_traffic_needs_a_record_of_the_current_source(monkeypatch):
    root = os.path.dirname(os.path.abspath(bench.__file__))
    src = "paper_1612_07526_gb300/csrc/gemm_fp64.cu"
    with open(os.path.join(root, src), "rb") as f:
        sha = hashlib.sha256(f.read()).hexdigest()
    monkeypatch.setattr(bench, "TRAFFIC_RATIO", {"k_gemm_fp64": (1.25, ((src, sha),))})
    assert bench.measured_traffic("k_gemm_fp64", 1000.0) == 1250.0
    assert bench.measured_traffic("k_oz_gemm", 1000.0) is None
    assert bench.measured_traffic("k_gemm_fp64", 0.0) is None
    monkeypatch.setattr(bench, "TRAFFIC_RATIO", {"k_gemm_fp64": (1.25, ((src, sha), (src, "0" * 64)))})
    assert bench.measured_traffic("k_gemm_fp64", 1000.0) is None       # a kernel file changed since


def test_traffic_record_matches_the_current_kernel_sources():
    """The committed record was captured on the product kernel as it is now."""
    assert bench.measured_traffic("k_gemm_fp64", 1000.0) is not None


def test_both_arms_print_the_same_config():
    a = _args()
    c = bench.workload_config(a)
    assert c == bench.workload_config(_args())
    assert c["n"] == 32768 and c["leaf"] == 32 and "n=32768" in c["workload"]
    assert bench.workload_config(_args(leaf=16))["workload"] != c["workload"]


def test_cpu_oracle_fit_small():
    v, fit, sample, cores = bench.cpu_oracle_fit("uniform", 512, 32, sizes=(64, 128))
    assert fit["sizes"] == [64, 128] and len(fit["seconds"]) == 2
    assert v == fit["seconds"][1] * (512 / 128) ** fit["exponent"]
    assert "fitted exponent" in sample and cores >= 1


def test_cpulist():
    assert bench._cpulist("0-3,8,10-11\n") == {0, 1, 2, 3, 8, 10, 11}
    assert bench._cpulist("") == set()
