"""bench.py's host logic on CPU: the roofline's DRAM traffic is taken only
from an ncu summary line naming the kernel and the workload (or a
per-cluster figure in the kernel's own summary), never from another
kernel's figure."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _figure(name, key):
    for f in sorted(os.listdir(os.path.join(ROOT, "profiles"))):
        for line in open(os.path.join(ROOT, "profiles", f)):
            if line.startswith(key):
                return int(line.split(":")[1])
    raise AssertionError(f"no {key} line under profiles/ for {name}")


def test_traffic_of_the_named_kernel_and_workload():
    want = _figure("qr_cluster", "traffic_bytes_per_launch(qr_cluster_kernel, poisson3d_128)")
    assert bench._traffic("qr_cluster", "poisson3d_128", 16384, 474) == want


def test_traffic_of_another_workload_or_kernel_is_not_borrowed():
    # the Schur figure of the launch list predates a change of that kernel
    # and carries no kernel-and-workload line: no traffic for it
    assert bench._traffic("schur", "poisson3d_128", 16384, 596) is None
    # no summary captured this workload for the cluster QR
    assert bench._traffic("qr_cluster", "poisson3d_64", 2048, 148) is None
    # a kernel without a summary
    assert bench._traffic("gemm_fill", "poisson3d_128", 16384, 596) is None


def test_per_cluster_traffic_scales_by_clusters_per_launch():
    per = _figure("prep", "traffic_bytes_per_cluster")
    assert bench._traffic("prep", "poisson3d_128", 1000, 10) == per * 1000 / 10
