"""Host-side logic of the benchmark: parameter parsing, the workload table,
the DRAM-traffic records tied to kernel-source revisions, the clock sampler's
summary of throttle reasons, and the oracle's bounded batch sample."""
import json
import os
import shutil

import numpy as np
import pytest

import bench
from paper_1405_5483_gb300 import workloads as W


def test_parse_params_accepts_json_and_key_value_lists():
    assert bench.parse_params("q=5,sigma_r=65536,k=1") == {"q": 5, "sigma_r": 65536, "k": 1}
    assert bench.parse_params(' {"q": 4, "kernel": 2} ') == {"q": 4, "kernel": 2}
    assert bench.parse_params("") == {}
    with pytest.raises(ValueError):
        bench.parse_params("q=five")


def test_every_workload_names_a_generator_and_its_arguments():
    for name, entry in bench.WORKLOADS.items():
        gen, sigma, desc = entry[:3]
        assert callable(getattr(W, gen)), name
        assert 1 <= sigma <= 256 and desc
        if len(entry) > 3:
            import inspect
            params = inspect.signature(getattr(W, gen)).parameters
            assert set(entry[3]) <= set(params), name


def test_small_workload_builds():
    case, sigma, desc = bench.make_case("dna-1MiB")
    assert case.n == 1 << 20 and case.P.shape == (100, 16) and sigma == 4


def _fake_tree(tmp_path, files):
    csrc = tmp_path / "paper_1405_5483_gb300" / "csrc"
    csrc.mkdir(parents=True)
    for f in files:
        shutil.copy(os.path.join(bench.ROOT, "paper_1405_5483_gb300", "csrc", f), csrc / f)
    (tmp_path / "profiles").mkdir()
    return csrc


def test_recorded_traffic_follows_the_kernel_revision(tmp_path, monkeypatch):
    files = ("keyhash.h", "multiword.h", "scan_jit_args.h", "ptx_common.cuh",
             "window_check.cuh", "jit_types.h", "scan_stage.cuh", "scan_jit.cuh", "jit.cpp")
    csrc = _fake_tree(tmp_path, files)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    rev = bench.kernel_rev()
    rec = {"params": {"q": 5, "kernel": 2}, "traffic_bytes_per_launch": 123456}
    (tmp_path / "profiles" / "mpm_scan_jit_w.md").write_text(
        "# summary\n\n- `kernel_rev`: `%s`\n- `record`: `%s`\n" % (rev, json.dumps(rec)))
    assert bench.recorded_traffic("w", {"q": 5, "kernel": 2, "k": 1}) == 123456
    assert bench.recorded_traffic("w", {"q": 4, "kernel": 2}) is None
    assert bench.recorded_traffic("other", {"q": 5, "kernel": 2}) is None
    # a change to any of the kernel's sources retires the record
    with open(csrc / "jit.cpp", "a") as f:
        f.write("\n// changed\n")
    assert bench.kernel_rev() != rev
    assert bench.recorded_traffic("w", {"q": 5, "kernel": 2}) is None


def test_batch_traffic_record_uses_its_own_revision(tmp_path, monkeypatch):
    files = ("batch.cu", "batch_args.h", "stepper.cuh", "multiword.h", "device_common.cuh",
             "window_check.cuh", "keyhash.h")
    _fake_tree(tmp_path, files)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    rev = bench.batch_kernel_rev()
    (tmp_path / "profiles" / "batch_scan_kernel_b.md").write_text(
        "- `kernel_rev`: `%s`\n- `record`: `{\"params\": {}, "
        "\"traffic_bytes_per_launch\": 99}`\n" % rev)
    assert bench.recorded_traffic("b", {}, "batch_scan_kernel", rev) == 99
    assert bench.recorded_traffic("b", {}, "batch_scan_kernel", "0" * 12) is None


def test_committed_profiles_parse():
    # every committed summary that carries records names a revision and
    # well-formed JSON records
    pdir = os.path.join(bench.ROOT, "profiles")
    for f in os.listdir(pdir):
        revs, recs = 0, 0
        for line in open(os.path.join(pdir, f)):
            if line.startswith("- `kernel_rev`"):
                revs += 1
            elif line.startswith("- `record`"):
                val = line.split(":", 1)[1].strip().strip("`")
                rec = json.loads(val)
                assert int(rec["traffic_bytes_per_launch"]) > 0
                recs += 1
        assert recs == 0 or revs == 1, f


def test_clock_summary_names_throttle_reasons():
    cs = bench.ClockSampler.__new__(bench.ClockSampler)
    cs.max_mhz = 2070
    cs.samples = [(2070, 0), (1900, 0x4), (2070, 0x4 | 0x40), (2070, 0)]
    s = cs.summary()
    assert s["sm_mhz"] == 2070 and s["sm_max_mhz"] == 2070 and s["samples"] == 4
    assert s["reasons"] == ["hw_thermal_slowdown", "sw_power_cap"]
    cs.samples = []
    assert cs.summary() is None


def test_oracle_batch_sample_is_bounded_and_in_text_order(oracle_native):
    class B:
        pass
    rng = np.random.default_rng(3)
    b = B()
    b.texts = [rng.integers(65, 69, size=n).astype(np.uint8) for n in (1000, 5000, 300, 7000)]
    b.sets = [rng.integers(65, 69, size=(5, 6)).astype(np.uint8) for _ in range(2)]
    b.set_of_text = np.array([0, 1, 1, 0], np.uint32)
    o = bench.OracleBatchSample(b, 5500)
    assert o.picked == [0, 1] and o.total == 6000
    z = o.step()
    want = sum(oracle_native.aho_corasick(b.texts[t], b.sets[int(b.set_of_text[t])])[0].size
               for t in o.picked)
    assert z == want
    o.close()
