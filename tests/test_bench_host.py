"""Host logic of bench.py's double-buffered end-to-end loop, on CPU.

The loop drives two handles from two host threads; a copy token alternates
between them so that one thread copies its step's inputs while the other runs
its sweep.  Here the handles are fakes that record when each call starts and
ends, and torch's CUDA calls are stubbed, so the protocol itself is checked:
every step runs once, the copies never overlap, each copy overlaps the other
handle's sweep, and a failing handle ends the loop with its error instead of a
hang.

Also on CPU: the oracle sample scaling and its spawned replicas, the
parsing of the nvidia-smi clock record (median SM clock, throttle reasons),
and the guard that reports recorded DRAM traffic only for the kernel text it
was measured on."""
import importlib.util
import os
import threading
import time

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def load_bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


class FakeHandle:
    log = []
    lock = threading.Lock()
    fail_at = None            # (handle id, call count) that raises

    def __init__(self, hid):
        self.hid = hid
        self.calls = 0

    def _rec(self, what, dur):
        t0 = time.perf_counter()
        time.sleep(dur)
        with FakeHandle.lock:
            FakeHandle.log.append((self.hid, what, t0, time.perf_counter()))

    def set_stream(self, s):
        pass

    def set_tensor(self, X):
        self.calls += 1
        if FakeHandle.fail_at == (self.hid, self.calls):
            raise RuntimeError("planted failure")
        self._rec("copy", 0.02)

    def set_factors(self, A):
        pass

    def iterate(self, n, **kw):
        self._rec("sweep", 0.02)
        return 1

    def get_factors(self):
        return None, None

    def fit(self):
        return 0.5


class FakeCpals:
    def __init__(self):
        self.made = 0

    def CPALS(self, dims, R, prec):
        h = FakeHandle(self.made)
        self.made += 1
        return h


@pytest.fixture
def bench(monkeypatch):
    torch = pytest.importorskip("torch")
    monkeypatch.setattr(torch.cuda, "Stream", lambda *a, **k: object())
    monkeypatch.setattr(torch.cuda, "synchronize", lambda *a, **k: None)
    monkeypatch.setattr(torch.cuda, "current_device", lambda: 0)
    monkeypatch.setattr(torch.cuda, "set_device", lambda d: None)
    FakeHandle.log = []
    FakeHandle.fail_at = None
    return load_bench()


def test_double_buffered_steps_alternate_and_overlap(bench):
    steps = 8
    bench.e2e_double_buffered(FakeCpals(), (4, 4, 4), 2, None, None, "qr", steps)
    timed = [e for e in FakeHandle.log]
    # warm-up: one copy and one sweep per handle before the timed loop
    copies = sorted([e for e in timed if e[1] == "copy"], key=lambda e: e[2])[2:]
    sweeps = [e for e in timed if e[1] == "sweep"][2:]
    assert len(copies) == steps and len(sweeps) == steps
    # each handle took half the steps, alternating
    assert [c[0] for c in copies] == [i % 2 for i in range(steps)]
    # copies never overlap each other
    for a, b in zip(copies, copies[1:]):
        assert b[2] >= a[3] - 1e-4
    # every copy after the first overlaps a sweep of the other handle
    overl = 0
    for c in copies[1:]:
        if any(s[0] != c[0] and s[2] < c[3] and c[2] < s[3] for s in sweeps):
            overl += 1
    assert overl >= steps - 2


def test_double_buffered_failure_propagates_without_hang(bench):
    FakeHandle.fail_at = (1, 3)     # handle 1's third copy (its second timed step) raises
    done = []

    def run():
        try:
            bench.e2e_double_buffered(FakeCpals(), (4, 4, 4), 2, None, None, "qr", 10)
        except RuntimeError as e:
            done.append(str(e))

    t = threading.Thread(target=run)
    t.start()
    t.join(timeout=30)
    assert not t.is_alive(), "the loop hung after a failure"
    assert done == ["planted failure"]


def test_oracle_sample_rates_scale_by_elements_and_memory_bounds_replicas(bench, monkeypatch):
    # the sample timed 2 s for half a sweep over a quarter of the workload's
    # elements: 0.25 sweeps/s of the sample -> 0.0625 sweeps/s of the workload
    calls = []

    def fake_sample(task):
        calls.append(task)
        return 2.0, 0.5, 250

    monkeypatch.setattr(bench, "_oracle_sample", fake_sample)
    monkeypatch.setattr(bench, "_replica_map", lambda fn, tasks: [fn(t) for t in tasks])
    import oracle
    monkeypatch.setattr(oracle, "build", lambda: None)
    monkeypatch.setattr(bench.os, "cpu_count", lambda: 16)
    # room for 3 replicas: a quarter of the free memory over 4 copies of 8-byte elements
    monkeypatch.setattr(bench, "_host_mem_available", lambda: 4 * 3 * 4 * 8 * 250)
    cpu = bench.oracle_sample_baseline("c3", 1000, "sample", modes=1)
    assert cpu["value"] == pytest.approx(0.5 / 2.0 * 250 / 1000)
    assert cpu["cores"] == 1 and cpu["kind"] == "oracle" and cpu["sample"] == "sample"
    assert cpu["all_cores"]["cores"] == 3 and cpu["all_cores"]["value"] == pytest.approx(3 * cpu["value"])
    assert len(calls) == 1 + 3
    # too little memory for two replicas: no all-cores figure
    monkeypatch.setattr(bench, "_host_mem_available", lambda: 4 * 1 * 4 * 8 * 250)
    assert "all_cores" not in bench.oracle_sample_baseline("c3", 1000, "sample", modes=1)


def test_replica_map_runs_single_threaded_children_and_restores_env(bench, monkeypatch):
    monkeypatch.setenv("OMP_NUM_THREADS", "7")
    monkeypatch.delenv("OPENBLAS_NUM_THREADS", raising=False)
    out = bench._replica_map(os.getenv, ["OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS"])
    assert out == ["1", "1"]
    assert os.environ["OMP_NUM_THREADS"] == "7" and "OPENBLAS_NUM_THREADS" not in os.environ


def test_clock_summary_takes_median_and_throttle_reasons(bench, tmp_path):
    # nvidia-smi rows: index, clocks.sm, clocks.max.sm, power.draw, active mask,
    # then the four named reasons; a malformed row and a "[N/A]" row are skipped
    path = tmp_path / "clocks.csv"
    path.write_text("0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active\n"
                    "0, 1980, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active\n"
                    "0, 2070, 2070, 1200.5, 0x0, Not Active, Not Active, Not Active, Not Active\n"
                    "garbage line\n"
                    "0, [N/A], 2070, 1.0, 0x0, Not Active, Not Active, Not Active, Not Active\n"
                    "0, 1500, 2100, 1399.9, 0x8, Active, Not Active, Not Active, Not Active\n")
    clk = bench.ClockSampler(0)
    clk.path = str(path)
    s = clk.summary()
    assert s == {"sm_mhz": 2025.0, "sm_max_mhz": 2100.0, "reasons": ["hw_slowdown", "sw_power_cap"], "samples": 4}
    assert not path.exists()            # the temporary record is removed


def test_clock_summary_without_samples_is_none(bench, tmp_path):
    path = tmp_path / "empty.csv"
    path.write_text("")
    clk = bench.ClockSampler(0)
    clk.path = str(path)
    assert clk.summary() is None
    assert bench.ClockSampler(0).summary() is None       # sampler never started


def test_kernel_source_spans_template_line_to_closing_brace(bench):
    src = bench.kernel_source("ttm_rows_kernel")
    lines = src.split("\n")
    assert lines[0].startswith("template") and "__global__" in lines[1]
    assert lines[-1] == "}" and src.count("__global__") == 1
    assert bench.kernel_source("no_such_kernel") == ""


def test_recorded_traffic_needs_the_recorded_kernel_text(bench, monkeypatch):
    # the committed summary holds the DRAM bytes and the hash of the kernel
    # text they were taken on; any other text gives no traffic figure
    t = bench.recorded_traffic()
    assert isinstance(t, int) and 512_000_000 <= t <= 530_000_000
    real = bench.kernel_source
    monkeypatch.setattr(bench, "kernel_source", lambda name: real(name) + "\n// changed")
    assert bench.recorded_traffic() is None
    assert bench.recorded_traffic("no_such_profile.md") is None


def test_single_thread_oracle_sample_is_bounded(bench):
    # the 1-thread oracle sample times whole sweeps: at least 2, at most the
    # cap, as many as the first sweep's time says fit the target
    from paper_2112_10855_gb300 import inputs
    p = inputs.workload_c2(size=24, rank=3)
    rate, dt, n = bench.cpu_oracle_rate(p, target_s=0.0)
    assert n == 2 and dt > 0 and abs(rate - n / dt) < 1e-9 * rate
    rate, dt, n = bench.cpu_oracle_rate(p, target_s=1e9, max_sweeps=7)
    assert n == 7 and abs(rate - n / dt) < 1e-9 * rate
    rate, dt, n = bench.cpu_oracle_rate(p, target_s=0.3, max_sweeps=10000)
    assert 2 <= n < 10000 and dt >= 0.1


def test_profile_commands_use_flags_the_bench_accepts(bench, monkeypatch):
    # every committed ncu summary names the command that made it; its bench.py
    # part must still parse, so the command can be run again as written
    import glob
    import re
    import shlex
    import sys
    found = 0
    for path in sorted(glob.glob(os.path.join(ROOT, "profiles", "*.md"))):
        text = open(path).read()
        assert re.search(r"^Commands? ", text, re.M), f"{path}: no command"
        joined = text.replace("\\\n", " ")
        for m in re.finditer(r"python bench\.py([^\n`]*)", joined):
            argv = ["bench.py"] + shlex.split(m.group(1))
            monkeypatch.setattr(sys, "argv", argv)
            bench.parse()       # argparse exits on an unknown flag or a bad value
            found += 1
    assert found >= 8
