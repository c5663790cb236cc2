"""Host-side logic of bench.py (no GPU): the --launch parser, the step kernel's name
for a launch, the per-kernel DRAM traffic taken from the committed ncu summary (which
must describe the committed source of the step kernel), and the JSON config keys."""
import json
import os

import pytest

import bench


def test_parse_launch():
    assert bench.parse_launch("auto") == ("auto", "auto")
    assert bench.parse_launch("pair:40x24") == ((40, 24), "pair")
    assert bench.parse_launch("fused:26X16") == ((26, 16), "fused")
    with pytest.raises(Exception):
        bench.parse_launch("pair:40")


def test_kernel_name_and_source():
    name, src = bench.kernel_name("f32", "pair", [40, 24])
    assert name == "pair_persistent<float, 40, 24>" and src.endswith("amlbm_step_pair.cu")
    name, src = bench.kernel_name("bf16", "fused", [26, 16])
    assert name.startswith("lbm_persistent<") and src.endswith("amlbm_step.cu")


def test_profiled_traffic_matches_the_committed_step_kernel():
    p = os.path.join(bench.ROOT, "profiles", "step_kernel_traffic.json")
    d = json.load(open(p))
    _, src = bench.kernel_name("f32", "pair", [40, 24])
    for kernel, k in d["kernels"].items():
        assert k["dram_bytes_per_launch"] == k["dram_bytes_read_per_launch"] + k["dram_bytes_write_per_launch"]
        # the algorithmic reads are 40 B per site of the 694,696-site sweep: ncu's
        # reads may exceed them (halo, partial sectors), never fall below
        assert k["dram_bytes_read_per_launch"] >= 40 * 694696
        assert bench.profiled_traffic(src, kernel) == k["dram_bytes_per_launch"], kernel
    assert bench.profiled_traffic(src, "pair_persistent<float, 12, 34>") is None


def test_config_keys():
    c = bench.config(694696, tile=(40, 24), schedule="pair")
    assert c["sites_per_step"] == 694696 and c["tile"] == [40, 24] and c["schedule"] == "pair"
    assert "workload" in c and "l2" in c
