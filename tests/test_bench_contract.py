"""The reference arm of bench.py (the FP64 oracle's Eq. (3) apply timed on
host cores) prints one JSON line with the keys the benchmark contract
fixes; checked on the CPU with a shortened sample."""
import json
import types


def test_reference_line_keys(monkeypatch, capsys):
    import bench
    full = bench.oracle_coarse_apply_sample

    def short(**kw):
        return full(n=8, cdims=(2, 2, 2, 4), budget_s=0.05, cores=2)

    monkeypatch.setattr(bench, "oracle_coarse_apply_sample", short)
    monkeypatch.delenv("RANK", raising=False)
    args = types.SimpleNamespace(steps=2, warmup=1, gpus=1)
    assert bench.reference_main(args) == 0
    lines = [ln for ln in capsys.readouterr().out.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC
    assert d["unit"] == "GB/s" and d["higher_is_better"] is True
    assert d["n_gpus"] == 1 and d["steps"] == 2 and d["warmup"] == 1
    assert d["value"] > 0 and d["ms_per_step"] > 0
    assert d["config"]["workload"] == bench.WORKLOAD
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] == 2 and cb["sample"]
    assert cb["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": "GB/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}


def test_reference_arm_other_ranks_do_no_work(monkeypatch, capsys):
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setattr(bench, "oracle_coarse_apply_sample",
                        lambda **kw: (_ for _ in ()).throw(AssertionError("ran on rank 1")))
    assert bench.reference_main(types.SimpleNamespace(steps=1, warmup=0, gpus=2)) == 0
    assert capsys.readouterr().out == ""


def test_oracle_sample_counts_fp64_algorithmic_bytes(monkeypatch):
    """One process's chunk: sites x (9 n^2 links + 2 n spinor) x 16 B per
    repetition, with a clock that advances one second per reading (one
    repetition); the baseline sums the processes' rates."""
    import itertools

    import bench
    clock = itertools.count()
    monkeypatch.setattr(bench.time, "perf_counter", lambda: float(next(clock)))
    reps, el, nbytes = bench._oracle_apply_worker((8, (2, 2, 2, 4), 0, 8, 0.5))
    assert (reps, el) == (1, 1.0)
    assert nbytes == 8 * (9 * 64 * 16 + 2 * 8 * 16)


def test_oracle_sample_uses_every_requested_core():
    import bench
    r = bench.oracle_coarse_apply_sample(n=8, cdims=(2, 2, 2, 4), budget_s=0.2, cores=3)
    assert r["unit"] == "GB/s" and r["cores"] == 3 and r["value"] > 0
    assert "all 32 sites" in r["sample"] and "3 processes" in r["sample"]


def test_clock_sampler_summary(tmp_path):
    """Median SM clock, maximum clock and the throttle reasons seen, from
    nvidia-smi's csv,noheader,nounits lines of the query the bench issues."""
    import bench

    class Done:
        def terminate(self):
            pass

        def wait(self, timeout=None):
            return 0

    path = tmp_path / "clocks.csv"
    path.write_text(
        "0, 2070, 2070, 950.1, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active\n"
        "0, 1965, 2070, 1390.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active\n"
        "0, 2010, 2070, 1200.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active\n"
        "garbage line\n")
    s = bench.ClockSampler(0, str(path))
    s.proc, s.fh = Done(), open(path, "a")
    out = s.stop()
    assert out == {"sm_mhz": 2010.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"],
                   "samples": 3}
