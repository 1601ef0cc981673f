"""Host-side logic of the benchmark and the learned-guess pipeline that runs
without a GPU: the level-history summary (the paper's Sec. 5 shares), the
launch count against the schedule, and the face-frame marshalling."""
import json
import os
import sys

import numpy as np
import pytest

from conftest import ROOT

sys.path.insert(0, ROOT)


class FakeMesh:
    def __init__(self, counts, dtm):
        self._c, self._d = np.asarray(counts, dtype=np.int32), np.asarray(dtm)

    def level_history(self):
        return self._c, self._d


def test_level_history_summary_shares_and_cost_ratio():
    import bench
    # Table 1 of the paper, theta = 3: cells per level 5 / 5 / 10 / 80 (of
    # 100), cost 2^(3-k) |Omega_k| = 40 + 20 + 20 + 80 = 160 against 800
    counts = np.zeros((2, 8), dtype=np.int32)
    counts[0, :4] = [5, 5, 10, 80]
    counts[1, :4] = [10, 10, 20, 60]
    s = bench.level_history_summary(FakeMesh(counts, [1e-3, 9e-4]), 4)
    assert s["cycles_recorded"] == 2
    f = s["first"]
    assert f["cells_share"] == [0.05, 0.05, 0.1, 0.8]
    assert f["cost_share"] == [0.25, 0.125, 0.125, 0.5]
    assert f["global_over_adaptive_cost"] == 5.0
    assert s["last"]["global_over_adaptive_cost"] == round(800 / (80 + 40 + 40 + 60), 4)
    assert bench.level_history_summary(FakeMesh(np.zeros((0, 8)), []), 4) is None
    assert bench.level_history_summary(None, 4) is None


@pytest.mark.parametrize("L", [1, 2, 4, 6])
def test_launch_count_matches_the_schedule(L):
    import bench
    from paper_1704_01144_gb300 import schedule as S
    nph = len(S.phases(L - 1))
    assert nph == 3 * 2 ** (L - 1) - 1
    # k_init_min2, k_dt32, k_dt_min_exact, k_levels0_certified, L-1 x k_smooth,
    # k_keys_hist, k_sort_scan2, k_sort_scatter2 (launch_assign_levels)
    level_assignment = 4 + (L - 1) + 3
    assert bench.launches_per_cycle(L, fp32=True) == level_assignment + 3 * nph + 1
    assert bench.launches_per_cycle(L, fp32=False) == level_assignment + 4 * nph + 1


def test_face_frame_marshalling():
    torch = pytest.importorskip("torch")
    from paper_1704_01144_gb300 import learned_guess as LG
    pairs = torch.tensor([[1.0, 0.5, 2.0, 0.5, -0.25, 1.0]], dtype=torch.float64)
    WL, WR, n = LG.face_frame(pairs)
    assert WL[:, 0].tolist() == [1.0, 0.5, 0.0, 0.0, 2.0]
    assert WR[:, 0].tolist() == [0.5, -0.25, 0.0, 0.0, 1.0]
    assert n[:, 0].tolist() == [1.0, 0.0, 0.0]


def test_paper_order_host_schedule_matches_oracle(oracle_mod):
    """The library's host schedule for FV_ORDER_PAPER (mirrored in
    schedule.phases) is the oracle's order-1 phase list."""
    from paper_1704_01144_gb300 import schedule as S
    for theta in range(6):
        assert S.phases(theta, 1) == oracle_mod.phase_list(theta, order=1)
        assert S.phases(theta) == oracle_mod.phase_list(theta)


def test_roofline_entry_arithmetic():
    """achieved = algorithmic bytes per unit x units / time; frac against the
    peak; traffic = committed per-unit DRAM bytes x units per launch."""
    import bench
    prof = {"flux": (2.0, 46), "update": (0.0, 0)}
    fe, cu = 11_187_220, 2_728_706  # two cycles of the 1M-tet blast
    r = bench.roofline_entry(prof, fe, cu, True, "flux", 6690.8, "measured",
                             {"flux_fp32_dram_bytes_per_unit": "139.0"})
    assert r["algorithmic_bytes_per_unit"] == 121.0
    assert r["achieved"] == round(fe * 121.0 / 2e-3 / 1e9, 1)
    assert r["frac"] == round(r["achieved"] / 6690.8, 4)
    assert r["traffic"] == round(139.0 * fe / 46)
    assert r["units_per_launch"] == round(fe / 46, 1) and r["launches"] == 46
    assert bench.roofline_entry(prof, fe, cu, True, "update", 6690.8, "measured", None) is None
    r64 = bench.roofline_entry({"update": (1.0, 46)}, fe, cu, False, "update", 6690.8, "measured", None)
    assert r64["algorithmic_bytes_per_unit"] == 383 and r64["traffic"] is None


def test_algorithmic_bytes_match_the_documented_breakdown():
    """Per face evaluation: index 4, two cells 8, geometry 28/56, half of
    each cell's primitives and gradients 40/80; the predictor writes its
    flux record (20/40), the corrector reads it back, writes the FP64
    integral (40) and reads 2 level bytes; mean of the two stages 121 / 209.
    Per cell update, both stages: 319 / 383."""
    import bench
    assert bench.flux_bytes_per_eval(True) == 121.0
    assert bench.flux_bytes_per_eval(False) == 209.0
    assert bench.update_bytes_per_cell_update(True) == 319
    assert bench.update_bytes_per_cell_update(False) == 383


class FakeNvml:
    """Stands in for the NVIDIA management library: a device count, an SM
    clock that follows a script, and clock-event reason bits."""

    def __init__(self, count=1, clocks=(2070, 2070, 1980), reasons=(0, 0x4, 0x4), fail_at=None):
        self.count, self.clocks, self.reasons = count, list(clocks), list(reasons)
        self.i, self.fail_at, self.index, self.shut = 0, fail_at, None, False

    def nvmlInit_v2(self):
        return 0

    def nvmlShutdown(self):
        self.shut = True
        return 0

    def nvmlDeviceGetCount_v2(self, p):
        p._obj.value = self.count
        return 0

    def nvmlDeviceGetHandleByIndex_v2(self, idx, p):
        self.index = idx.value
        p._obj.value = 1234
        return 0

    def nvmlDeviceGetMaxClockInfo(self, h, kind, p):
        assert kind == 1  # the SM clock
        p._obj.value = 2070
        return 0

    def nvmlDeviceGetClockInfo(self, h, kind, p):
        assert kind == 1
        if self.i == self.fail_at:
            self.i += 1
            return 999
        p._obj.value = self.clocks[min(self.i, len(self.clocks) - 1)]
        return 0

    def nvmlDeviceGetCurrentClocksEventReasons(self, h, p):
        p._obj.value = self.reasons[min(self.i, len(self.reasons) - 1)]
        self.i += 1
        return 0


def test_nvml_clock_samples_decode_reasons():
    import bench
    lib = FakeNvml(reasons=(0, 0x4 | 0x1, 0x8 | 0x40 | 0x20))
    nv = bench.NvmlClocks(3, lib)
    assert lib.index == 0  # one visible device is index 0 whatever the CUDA index
    assert nv.sample() == (2070.0, 2070.0, set())
    assert nv.sample() == (2070.0, 2070.0, {"sw_power_cap"})  # the idle bit is not a reason
    assert nv.sample() == (1980.0, 2070.0,
                           {"hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"})
    lib8 = FakeNvml(count=8)
    bench.NvmlClocks(3, lib8)
    assert lib8.index == 3
    with pytest.raises(OSError):
        bench.NvmlClocks(8, FakeNvml(count=8))


def test_clock_sampler_summary_over_the_timed_region():
    import time
    import bench
    lib = FakeNvml(clocks=(2070, 1, 1500, 2070, 2070), reasons=(0, 0x8, 0, 0x4, 0), fail_at=1)
    with bench.ClockSampler(0, nvml_lib=lib, interval_s=0.001) as clk:
        assert clk.rows  # entering waits for the first sample
        while lib.i < 8:
            time.sleep(0.001)
    s = clk.summary()
    assert lib.shut and s["sm_max_mhz"] == 2070.0 and s["sm_mhz"] == 2070.0
    # the failed query (index 1) is skipped with its reasons
    assert s["reasons"] == ["sw_power_cap"] and s["samples"] >= 6
    assert s["sampler"].startswith("NVML")


def test_clock_rejection_rule():
    import bench
    ok = {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": []}
    assert not bench.clocks_rejected(ok)
    assert not bench.clocks_rejected({**ok, "sm_mhz": 1700.0, "reasons": ["sw_power_cap"]})
    for r in ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"):
        assert bench.clocks_rejected({**ok, "reasons": [r]})
    assert bench.clocks_rejected({**ok, "sm_mhz": 1200.0})  # stuck low, no reason
    assert not bench.clocks_rejected({"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]})


class _FakeClock:
    t = 0.0


class _FakeEvent:
    def __init__(self, enable_timing=False):
        self.t = None

    def record(self, stream=None):
        self.t = _FakeClock.t

    def synchronize(self):
        pass

    def elapsed_time(self, other):
        return other.t - self.t


class _FakeTarget:
    """A mesh whose cycle costs more the farther its blocks per SM are from
    an optimum; advance() moves the fake clock on."""

    def __init__(self, opt):
        self.opt, self.launch, self.advances, self.resets = opt, [8, 8, 16, 8], 0, 0

    def get_launch(self):
        return list(self.launch)

    def set_launch(self, per_sm):
        self.launch = list(per_sm)

    def advance(self, n, stream=None, want_time=True):
        self.advances += 1
        _FakeClock.t += 1.0 + sum((a - b) ** 2 for a, b in zip(self.launch, self.opt)) * 1e-3


def test_autotuner_descends_and_caches(tmp_path, monkeypatch):
    """Coordinate descent over the kernel kinds finds the optimum a separable
    cost puts among the candidates, times every candidate from the reset
    state, stores the choice under the GPU and workload key, and a second
    call applies the cached choice without timing anything."""
    import torch
    from paper_1704_01144_gb300 import autotune as AT
    monkeypatch.setattr(torch.cuda, "get_device_name", lambda *a: "FakeGPU")
    monkeypatch.setattr(torch.cuda, "current_device", lambda: 0)
    monkeypatch.setattr(torch.cuda, "Event", _FakeEvent)
    cache = str(tmp_path / "tune.json")
    opt = [16, 4, 32, 16]
    tgt = _FakeTarget(opt)

    def reset():
        tgt.resets += 1

    best, info = AT.autotune(tgt, "sig", stream=object(), reps=2, cache_path=cache, reset=reset)
    assert best == opt and tgt.launch == opt and not info["cached"]
    n_timed = len(info["tried"])
    assert n_timed == 1 + sum(len(AT.CANDIDATES[k]) - 1 for k in AT.KINDS)
    assert tgt.resets == n_timed and tgt.advances == n_timed * 3  # capture + 2 reps each
    assert info["ms"] == pytest.approx(1.0)
    stored = json.load(open(cache))
    assert stored["FakeGPU|sig"]["per_sm"] == opt
    other = _FakeTarget([4, 4, 8, 4])
    best2, info2 = AT.autotune(other, "sig", stream=object(), cache_path=cache)
    assert info2["cached"] and best2 == opt and other.launch == opt and other.advances == 0
    best3, info3 = AT.autotune(_FakeTarget(opt), "other-workload", stream=object(), reps=1,
                               cache_path=cache)
    assert not info3["cached"] and set(json.load(open(cache))) == {"FakeGPU|sig",
                                                                   "FakeGPU|other-workload"}


def test_kernel_hash_ignores_comments_only():
    """The hash that gates the committed DRAM counters changes with code,
    not with comments or trailing blanks; string literals keep their
    comment-like text."""
    import bench
    a = 'int f(int x) { // twice\n  return 2 * x; /* plain */ }\nconst char *s = "a // b";\n'
    b = 'int f(int x) { // two times x\n  return 2 * x; /* doubled */ }   \n\nconst char *s = "a // b";\n'
    c = 'int f(int x) {\n  return 3 * x; }\nconst char *s = "a // b";\n'
    assert bench.strip_comments(a) == bench.strip_comments(b)
    assert bench.strip_comments(a) != bench.strip_comments(c)
    assert '"a // b"' in bench.strip_comments(a)


def test_committed_traffic_counters_parse(monkeypatch):
    """The committed ncu summary yields the per-unit DRAM bytes of both
    kernel classes in both modes when the sources hash to its recorded
    value, and nothing otherwise."""
    import bench
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "not-the-recorded-hash")
    assert bench.measured_traffic() is None
    monkeypatch.undo()
    recorded = None
    with open(os.path.join(ROOT, "profiles", "dram_traffic_blast1m.md")) as fh:
        for ln in fh:
            if "kernel_source_sha256_16:" in ln:
                recorded = ln.split(":", 1)[1].strip()
    assert recorded and len(recorded) == 16
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: recorded)
    t = bench.measured_traffic()
    for key in ("flux_fp32", "update_fp32", "flux_fp64", "update_fp64"):
        v = float(t[f"{key}_dram_bytes_per_unit"])
        assert 50.0 < v < 1000.0
    # only the machine-readable block is read, not the commands above it
    assert all(k == "kernel_source_sha256_16" or k.endswith("_per_unit") for k in t), t


def test_branch_free_minmod_equals_the_limiter():
    """The FP32 flux's limiter, max(min(a, b), 0) + min(max(a, b), 0), is the
    minmod of the branches (the smaller magnitude when a and b share a sign,
    else 0) for every pair of finite floats, signed zeros and subnormals
    included; checked in float32."""
    rng = np.random.default_rng(3)
    special = np.array([0.0, -0.0, 1e-45, -1e-45, 1e-38, -1e-38, 1.0, -1.0, 3.4e38, -3.4e38,
                        np.float32(2.0) ** -126, 7.0, -7.0], dtype=np.float32)
    mags = np.exp(rng.uniform(-80, 80, 20000)).astype(np.float32)
    vals = np.concatenate([special, mags * rng.choice([-1.0, 1.0], mags.size).astype(np.float32)])
    a = np.repeat(vals, 7)
    b = np.concatenate([np.roll(vals, k) for k in range(7)])
    a = np.concatenate([a, np.repeat(special, special.size)])
    b = np.concatenate([b, np.tile(special, special.size)])
    zero = np.float32(0.0)
    got = np.fmax(np.fmin(a, b), zero) + np.fmin(np.fmax(a, b), zero)
    same = (a > 0) & (b > 0)
    neg = (a < 0) & (b < 0)
    want = np.where(same, np.minimum(a, b), np.where(neg, np.maximum(a, b), zero))
    assert got.dtype == np.float32
    assert np.array_equal(got, want)


def test_reference_arm_prints_its_contract_line():
    """`bench.py --impl reference` times the FP64 oracle on the host cores and
    prints one JSON line with the reference keys (a small workload here)."""
    import subprocess
    import sys
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--workload", "sod", "--steps", "2", "--warmup", "3"],
                         capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    r = json.loads(lines[0])
    assert r["impl"] == "reference" and r["unit"] == "cell-updates/s" and r["value"] > 0
    assert r["steps"] == 2 and r["warmup"] >= 3 and r["higher_is_better"] is True
    assert r["data"].startswith("synthetic (Sod")
    cb = r["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == r["value"] and cb["sample"]
    e = r["e2e"]
    assert e["value"] == r["value"] and e["h2d_bytes_per_step"] == 0 == e["d2h_bytes_per_step"]


def test_reference_arm_samples_the_default_workload(monkeypatch, capsys):
    """The default workload is the 79.87M-tet ground blast; the oracle's
    reference arm runs a bounded sample of it (the same recipe on a smaller
    mesh, here shrunk further), restarted from its initial state every few
    cycles outside the timed region, and says so in its line."""
    import argparse
    import bench
    shape, L = bench.build_workload_shape(bench.DEFAULT_WORKLOAD)
    assert bench.DEFAULT_WORKLOAD == "ground80m" and shape.n_tets == 79872318 and L == 6
    assert bench.describe("ground80m", shape, L)["workload"].startswith("ground-plane half-sphere blast")
    monkeypatch.setattr(bench, "ORACLE_SAMPLE", {"ground80m": (dict(n=12, ratio=8.0), 2)})
    mesh, prim, Ls = bench.build_workload("ground80m", sample=True)
    assert mesh.n_tets == 6 * 12 ** 3 and Ls == 6
    args = argparse.Namespace(workload="ground80m", steps=3, warmup=3)
    bench.main_reference(args)
    line = json.loads([ln for ln in capsys.readouterr().out.splitlines() if ln.startswith("{")][-1])
    assert line["impl"] == "reference" and line["value"] > 0 and line["steps"] == 3
    assert "79872318 tets" in line["config"]["workload"]
    assert "10368 tets" in line["config"]["oracle_sample"] and "every 2 cycles" in line["config"]["oracle_sample"]
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["cpu_baseline"]["kind"] == "oracle"
