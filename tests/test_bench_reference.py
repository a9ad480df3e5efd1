"""Host logic of bench.py's reference arm on CPU: it times the FP64 oracle and prints one
JSON line with the keys of the bench contract (run here on a tiny workload in place of the
2048 x 256 wakefield, which takes seconds per oracle cycle)."""
import json
import types

import bench
from paper_1611_05712_gb300 import workloads as W


def test_reference_arm_prints_one_contract_line(monkeypatch, capsys):
    monkeypatch.setattr(bench, "workload", lambda order, rank=0: W.tiny(order_p=16, Nz=16, Nr=8, Nm=2, n_beam=32))
    monkeypatch.delenv("RANK", raising=False)
    args = types.SimpleNamespace(order=32, warmup=1, steps=2, gpus=1)
    assert bench.run_reference(args) == 0
    out = capsys.readouterr().out.strip().splitlines()
    assert len(out) == 1
    line = json.loads(out[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in line, k
    assert line["impl"] == "reference" and line["metric"] == "pic_steps_per_s"
    assert line["steps"] == 2 and line["warmup"] == 1 and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"] == {"value": line["value"], "unit": "steps/s", "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
    assert line["config"]["workload"] == "tiny" or line["config"]["Nz"] == 16


def test_reference_arm_other_ranks_do_no_work(monkeypatch, capsys):
    monkeypatch.setenv("RANK", "1")
    args = types.SimpleNamespace(order=32, warmup=1, steps=2, gpus=2)
    assert bench.run_reference(args) == 0
    assert capsys.readouterr().out == ""
