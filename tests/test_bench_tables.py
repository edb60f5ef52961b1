"""bench.py's host-side tables (CPU): the byte counts its roofline fractions divide by, the
workload tables, and the committed DRAM counters' bookkeeping."""
import json
import os

import bench


def test_algorithmic_bytes_per_node():
    # nine populations read and written, plus the fields the step reads once per node
    assert bench.algorithmic_bytes_per_node(4) == 84  # FP32: u_x, u_y, D
    assert bench.algorithmic_bytes_per_node(2) == 48  # 2-byte offsets, FP32 fields
    assert bench.algorithmic_bytes_per_node(8, 8) == 168  # FP64
    # one two-step launch: populations once, the five packed fields once
    assert bench.two_step_bytes_per_node(4) == 92
    assert bench.two_step_bytes_per_node(2) == 56


def test_companions_share_grid_and_physics():
    for main, comp in bench.COMPANIONS.items():
        mp, mkey, mbytes = bench.WORKLOADS[main]
        cp, ckey, cbytes = bench.WORKLOADS[comp]
        assert mkey == "f32" and mbytes == 4 and cbytes == 2 and ckey in ("f16", "bf16")
        assert mp == cp  # the same pulse: grid, Courant number, D field, source, steps


def test_default_workload_is_the_4096_fp32_pulse():
    pulse, key, nbytes = bench.WORKLOADS[bench.DEFAULT_WORKLOAD]
    assert (pulse.nx, pulse.ny, key, nbytes) == (4096, 4096, "f32", 4)
    assert pulse.steps == 10000


def test_committed_counters_are_keyed_by_kernel_and_command():
    path = os.path.join(bench.ROOT, "profiles", "step_kernel_counters.json")
    with open(path) as f:
        d = json.load(f)
    for workload, e in d.items():
        assert workload in bench.WORKLOADS
        assert e["kernel"] in bench.KERNEL_SOURCES
        assert e["dram_bytes_per_launch"] == e["dram_read"] + e["dram_write"]
        assert e["command"].startswith("ncu ") and "--clock-control none" in e["command"]
        assert f"--workload {workload}" in e["command"] or workload == bench.DEFAULT_WORKLOAD
        # a stale entry (kernel sources changed since the capture) is reported as no traffic
        expect = e["dram_bytes_per_launch"] if e["kernel_sha"] == bench.kernel_sha(e["kernel"]) else None
        assert bench.ncu_traffic(workload, e["kernel"]) == expect
