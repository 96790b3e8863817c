"""The bench's algorithmic work per lattice point (the roofline numerator)
against the hot-path table's count, for both pass-B rules, and the profile
records it reads (CPU only)."""
import json
import os

import bench

HERE = os.path.dirname(os.path.abspath(__file__))


def test_flop_count_per_point_two_passes_and_shared():
    phi, qinv = bench.PHI_FLOPS, bench.PHIINV_FLOPS
    for r in range(1, 7):
        rp = r * (r + 1) // 2
        # two passes: 2r Phi, 2r - 1 Phi^-1, r(r - 1) conditional FMAs, r + r(r+1)/2 moment FMAs (FMA = 2)
        assert bench.sweep_flops_per_point(r) == 2 * r * phi + (2 * r - 1) * qinv + 2 * r * (r - 1) + 2 * (r + rp)
        # one chain for both passes: r Phi, r Phi^-1, r(r - 1)/2 conditional FMAs, the same moment FMAs
        assert bench.sweep_flops_per_point(r, shared=True) == r * phi + r * qinv + r * (r - 1) + 2 * (r + rp)
        # pass A alone: r Phi, r - 1 Phi^-1, r(r - 1)/2 conditional FMAs
        assert bench.sweep_flops_per_point(r, density_only=True) == r * phi + (r - 1) * qinv + r * (r - 1)
    assert bench.sweep_flops_per_point(4) == 454
    assert bench.sweep_flops_per_point(4, shared=True) == 256


def test_profile_records_name_their_rule_and_carry_a_source_hash():
    for name, rule in (("estep_kernel_p4r4g3_n100000_N4096.json", "its own lattice sweep"),
                       ("estep_kernel_shared_p4r4g3_n100000_N4096.json", "on pass A's lattice points")):
        with open(os.path.join(HERE, "..", "profiles", name)) as f:
            rec = json.load(f)
        assert rec["pass_b"] == rule
        assert rec["dram_bytes_read"] > 0 and rec["gpu_time_ms"] > 0
        assert len(rec["source_sha256"]) == 64
