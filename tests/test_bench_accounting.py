"""The benchmark's bookkeeping, on the CPU: the unit count of the metric
(DOF-steps of one five-level estimate), the scaling of captured DRAM traffic
to a launch, the issue-rate ceiling, the members and extrapolation of the
oracle's bounded sample, and the clock record parsed from nvidia-smi
samples.  Each is checked against numbers worked out by hand."""
import json
import os

import pytest

import bench


def test_dof_steps_per_estimate_is_the_level_table():
    # one DOF-step = one node x one time block x one sample; both members of
    # a level pair count.  Levels 17^2 .. 257^2 with dt = 0.1 2^-l over
    # T = 10 (100 .. 1600 blocks) and 4096 / 1024 / 256 / 64 / 16 samples:
    #   l  fine                        coarse
    #   0  4096 x   289 x  100 = 118 374 400
    #   1  1024 x  1089 x  200 = 223 027 200   1024 x   289 x 100 =  29 593 600
    #   2   256 x  4225 x  400 = 432 640 000    256 x  1089 x 200 =  55 756 800
    #   3    64 x 16641 x  800 = 852 019 200     64 x  4225 x 400 = 108 160 000
    #   4    16 x 66049 x 1600 = 1 690 854 400   16 x 16641 x 800 = 213 004 800
    fine = 118_374_400 + 223_027_200 + 432_640_000 + 852_019_200 + 1_690_854_400
    coarse = 29_593_600 + 55_756_800 + 108_160_000 + 213_004_800
    assert bench.dof_steps_per_estimate() == fine + coarse == 3_723_430_400
    assert [bench.level_steps(l) for l in range(5)] == [100, 200, 400, 800, 1600]


def _fake_root(tmp_path, monkeypatch, entry_for):
    """A repository tree with one kernel source and a traffic record whose
    hash is that source's; returns the kernel key."""
    csrc = tmp_path / "paper_2105_02007_gb300" / "csrc"
    csrc.mkdir(parents=True)
    for f in bench.KERNEL_SOURCES["slab_solve_mg_kernel"]:
        (csrc / f).write_text(f"// {f}\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    key = "slab_solve_mg_kernel<16,12>"
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps({key: entry_for(bench.kernel_source_hash(key))}))
    return key


def test_traffic_scales_by_setup_and_per_block_parts(tmp_path, monkeypatch):
    # two captures of one sample at 4 and 8 blocks: 5376 B more over 4 more
    # blocks gives 1344 B per block and 3 681 280 - 4 x 1344 = 3 675 904 B
    # per sample of set-up; 16 samples x 1600 blocks:
    # 16 x (3 675 904 + 1600 x 1344) = 93 220 864 B
    caps = [dict(samples=1, steps=4, dram_bytes=3_681_280), dict(samples=1, steps=8, dram_bytes=3_686_656)]
    key = _fake_root(tmp_path, monkeypatch, lambda h: dict(source_hash=h, captures=caps))
    assert bench.load_traffic(key, 1, 4) == pytest.approx(3_681_280, abs=1e-6)
    assert bench.load_traffic(key, 1, 8) == pytest.approx(3_686_656, abs=1e-6)
    assert bench.load_traffic(key, 16, 1600) == pytest.approx(93_220_864, abs=1e-6)


def test_one_capture_scales_by_samples_and_blocks_and_a_stale_one_is_dropped(tmp_path, monkeypatch):
    caps = [dict(samples=16, steps=1, dram_bytes=700_000_000)]
    key = _fake_root(tmp_path, monkeypatch, lambda h: dict(source_hash=h, captures=caps))
    assert bench.load_traffic(key, 32, 3) == pytest.approx(700_000_000 * 6)
    # the kernel source changes after the capture: no traffic figure
    src = tmp_path / "paper_2105_02007_gb300" / "csrc" / bench.KERNEL_SOURCES["slab_solve_mg_kernel"][0]
    src.write_text(src.read_text() + "// changed\n")
    assert bench.load_traffic(key, 32, 3) is None


def test_issue_ceiling(tmp_path, monkeypatch):
    # 20 warp instructions per DOF and CG iteration, 100 iterations over
    # 1000 nodes in 1 ms: 2e6 instructions, 2e9 per second, against
    # 152 SMs x 4 schedulers x 2 GHz = 1.216e12 per second
    iss = dict(inst_per_dof_iter=20.0, sms=152, sm_mhz=2000.0, source="test")
    key = _fake_root(tmp_path, monkeypatch, lambda h: dict(source_hash=h, captures=[], issue=iss))
    r = bench.load_issue(key, dict(cg_iterations=100, nodes=1000, kernel_ms=1.0))
    assert r["inst"] == pytest.approx(2e6)
    assert r["achieved_inst_per_s"] == pytest.approx(2e9)
    assert r["peak_inst_per_s"] == pytest.approx(1.216e12)
    assert r["frac"] == pytest.approx(2e9 / 1.216e12)


def test_oracle_sample_members_and_extrapolation():
    # nine members (level 0 alone, then fine and coarse of pairs 1-4); pairs
    # 0-1 over the whole horizon, the others over max(40, 1 %) of their
    # blocks; with one rate r for every member the extrapolated whole
    # workload takes its DOF-steps / r
    pytest.importorskip("oracle")
    mem = bench.oracle_members(0)
    assert [(m["level"], m["coarse"], m["mesh"]) for m in mem] == [
        (0, 0, 0), (1, 0, 1), (1, 1, 0), (2, 0, 2), (2, 1, 1), (3, 0, 3), (3, 1, 2), (4, 0, 4), (4, 1, 3)]
    assert [m["blocks"] for m in mem] == [100, 200, 100, 40, 40, 40, 40, 40, 40]
    assert all(m["xi"].shape == (m["samples"], bench.K_MODES) for m in mem)
    rates = {(m["level"], m["coarse"]): 2.5e6 for m in mem}
    assert bench.whole_workload_seconds(rates) == pytest.approx(bench.dof_steps_per_estimate() / 2.5e6)


@pytest.mark.parametrize("M,K", [(9, 1), (9, 4), (9, 9), (9, 20)])
def test_reference_steps_cover_every_member(M, K):
    g = bench.step_groups(M, K)
    assert len(g) == K
    seen = sorted(i for idx in g for i in idx)
    assert set(seen) == set(range(M))
    if K <= M:
        assert seen == list(range(M))                       # each member once
        assert max(map(len, g)) - min(map(len, g)) <= 1     # balanced steps
    else:
        assert all(len(idx) == 1 for idx in g)


def test_estimate_against_the_oracle_whole_workload_record():
    # the header of the oracle's whole-workload fixture; a library estimate
    # 1e-10 off reads as 1e-10, and the record compared with itself as 0
    ref = bench.oracle_whole_workload()
    assert ref is not None and len(ref["var"]) == 5
    e = ref["estimate"][0]
    r = bench.compare_with_oracle_whole(e * (1 + 1e-10), ref["var"])
    assert r["estimate_rel"] == pytest.approx(1e-10, rel=1e-3)
    assert r["var_rel_max"] == 0.0
    assert "var_rel_max" not in bench.compare_with_oracle_whole(e, None)


class _Done:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def test_clock_record_median_and_throttle_reasons(tmp_path):
    # nvidia-smi rows: index, clocks.sm, clocks.max.sm, power, active mask,
    # hw_slowdown, hw_thermal_slowdown, sw_thermal_slowdown, sw_power_cap
    rows = ["0, 2070, 2070, 900.1, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
            "0, 1980, 2070, 1390.5, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
            "0, 2070, 2070, 1100.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
            "0, [N/A], 2070, 1000.0, 0x0, Not Active, Not Active, Not Active, Not Active"]
    path = tmp_path / "clocks.csv"
    path.write_text("\n".join(rows) + "\n")
    cs = bench.ClockSampler(0)
    cs.proc, cs.path = _Done(), str(path)
    r = cs.stop()
    assert r["sm_mhz"] == 2070.0 and r["sm_max_mhz"] == 2070.0
    assert r["reasons"] == ["sw_power_cap"]
    assert r["samples"] == 4
    assert not os.path.exists(path)
