"""Host-side pieces of bench.py, no GPU: the DRAM traffic record is reported
only while the CUDA sources hash to the recorded value, and the clock sampler
reads nvidia-smi's CSV rows into the median SM clock and the throttle reasons."""
import json
import os
import shutil

import pytest

bench = pytest.importorskip("bench")


def test_traffic_record_follows_the_sources(tmp_path, monkeypatch):
    root = bench.ROOT
    shutil.copytree(os.path.join(root, "paper_1905_09071_gb300", "csrc"),
                    tmp_path / "paper_1905_09071_gb300" / "csrc")
    (tmp_path / "profiles").mkdir()
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    rec = {"csrc_sha256": bench.csrc_sha256(), "kernels": {"k_fwd_col": {"dram_bytes": 123456.0}}}
    json.dump(rec, open(tmp_path / "profiles" / "traffic.json", "w"))
    assert bench.recorded_traffic("k_fwd_col") == 123456.0
    assert bench.recorded_traffic("no_such_kernel") is None
    with open(tmp_path / "paper_1905_09071_gb300" / "csrc" / "dw.cuh", "a") as fh:
        fh.write("\n")  # any change to the CUDA sources voids the record
    assert bench.recorded_traffic("k_fwd_col") is None


class _Done:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def test_clock_sampler_summary(tmp_path):
    s = bench.ClockSampler(0)
    s.path = str(tmp_path / "clocks.csv")
    s.proc = _Done()
    rows = ["0, 2070, 2070, 900.5, 0x0, Not Active, Not Active, Not Active, Not Active",
            "0, 2055, 2070, 1201.0, 0x4, Not Active, Not Active, Not Active, Active",
            "0, 2070, 2070, 1250.0, 0x4, Not Active, Not Active, Not Active, Active"]
    open(s.path, "w").write("\n".join(rows) + "\n")
    got = s.stop()
    assert got == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
