"""The benchmark script's host logic: the algorithmic byte counts behind every
roofline figure, and the reference arm (the FP64 oracle on the host cores),
which runs without a GPU and must print the contract's JSON line."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
from paper_1912_00695_gb300 import inputs  # noqa: E402


def test_algorithmic_bytes_of_the_sweep_shot():
    spec = inputs.sweep_shot(8, n=256, nt=10)
    pts = 276 ** 3
    layer = 276 ** 3 - 256 ** 3
    assert spec.points == pts and bench.layer_points(spec) == layer
    # FP32: read u^n, u^{n-1}, w, write u^{n+1}; g only in the layer
    assert bench.algorithmic_bytes_per_step(spec) == pts * 16 + layer * 4 == 353382656
    # 16-bit levels: the method's three 2-byte levels and the 4-byte coefficient
    assert bench.algorithmic_bytes_per_step(spec, "bf16") == pts * 10 + layer * 4
    # two steps per launch: read u^n, u^{n-1}, w, write u^{n+1}, u^{n+2}
    assert bench.algorithmic_bytes_two_steps(spec) == pts * 20 + layer * 4 == 437480960


def test_reference_arm_prints_the_contract_line():
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "3"],
                         cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["unit"] == "Gpts/s" and line["value"] > 0
    assert line["higher_is_better"] is True and line["steps"] == 1 and line["warmup"] >= 3
    cpu = line["cpu_baseline"]
    assert cpu["kind"] == "oracle" and cpu["cores"] >= 1 and cpu["value"] == line["value"] and cpu["sample"]
    e2e = line["e2e"]
    assert e2e["value"] == line["value"] and e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0
    assert line["metric"].startswith("Gpts/s")


def test_clock_record_rules():
    """The timed region is measured again when it saw a hardware or thermal
    slowdown or clocks well below maximum with no reason; a power cap is kept."""
    ok = {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": []}
    assert bench.clocks_ok(ok)
    assert bench.clocks_ok(dict(ok, sm_mhz=1800.0, reasons=["sw_power_cap"]))
    for r in ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"):
        assert not bench.clocks_ok(dict(ok, reasons=[r]))
    assert not bench.clocks_ok(dict(ok, sm_mhz=1200.0))  # locked low, no reason given
    assert bench.clocks_ok({"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]})


def test_committed_traffic_is_keyed_to_the_kernel_code(tmp_path, monkeypatch):
    """The ncu DRAM figure in profiles/traffic.json is used only while the step
    kernels' code is the one it was measured on; comments and layout do not
    count as a change. The committed figure lies between the algorithmic bytes
    and 1.5 times them (re-reads, not a different workload)."""
    h = bench._kernel_hash()
    per_step = bench._ncu_traffic(h, "sweep_n256")
    assert per_step is not None, "profiles/traffic.json is keyed to other kernel code"
    alg = bench.algorithmic_bytes_per_step(inputs.sweep_shot(8, n=256, nt=10))
    assert alg <= per_step <= 1.5 * alg
    two = bench._ncu_traffic(h, "sweep_n256_two_step")
    assert two is not None and bench.algorithmic_bytes_two_steps(inputs.sweep_shot(2, n=256, nt=10)) <= two
    assert bench._ncu_traffic("0" * 16, "sweep_n256") is None
    # a comment-only edit keeps the hash, a code edit changes it
    src = os.path.join(ROOT, "paper_1912_00695_gb300", "csrc")
    fake = tmp_path / "paper_1912_00695_gb300" / "csrc"
    fake.mkdir(parents=True)
    names = ("fd_stencil.cuh", "fd_tma.cuh", "fd_tma2.cuh", "fd_flow.cuh", "fd_flow.h", "fd_internal.h")
    for name in names:
        (fake / name).write_text(open(os.path.join(src, name), encoding="utf-8").read(), encoding="utf-8")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench._kernel_hash() == h
    with open(fake / "fd_flow.h", "a", encoding="utf-8") as f:
        f.write("\n// a note\n/* and a block\n   comment */\n")
    assert bench._kernel_hash() == h
    with open(fake / "fd_flow.h", "a", encoding="utf-8") as f:
        f.write("\nnamespace fdgb { constexpr int kUnused = 1; }\n")
    assert bench._kernel_hash() != h
