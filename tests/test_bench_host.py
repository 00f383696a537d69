"""Host-side helpers of bench.py (no GPU): the DRAM-traffic record keyed by the
kernel sources' hashes, and the NUMA CPU-list parser."""
import argparse
import hashlib
import os

import bench


def _args(**kw):
    a = dict(n=32768, gen="uniform", path="fp64")
    a.update(kw)
    return argparse.Namespace(**a)


def test_traffic_only_for_the_default_workload():
    assert bench.measured_traffic("k_gemm_fp64", _args(n=8192)) is None
    assert bench.measured_traffic("k_gemm_fp64", _args(gen="toeplitz")) is None
    assert bench.measured_traffic("k_oz_gemm", _args()) is None


def test_traffic_follows_the_source_hash():
    root = os.path.dirname(os.path.abspath(bench.__file__))
    for kernel, (per_step, launches, src, sha) in bench.TRAFFIC_U32768.items():
        with open(os.path.join(root, src), "rb") as f:
            current = hashlib.sha256(f.read()).hexdigest()
        got = bench.measured_traffic(kernel, _args())
        if current == sha:
            assert got == (per_step / launches, per_step)
        else:                                   # the kernel changed since the capture
            assert got is None


def test_cpulist():
    assert bench._cpulist("0-3,8,10-11\n") == {0, 1, 2, 3, 8, 10, 11}
    assert bench._cpulist("") == set()
