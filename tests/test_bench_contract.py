"""bench.py's reference arm (the FP64 CPU oracle chain) and its JSON-line contract,
on the CPU: one line with the shared workload config, an end-to-end object with
no host transfers, and under torchrun only rank 0 prints."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _json_lines(out):
    return [json.loads(l) for l in out.splitlines() if l.strip().startswith("{")]


def _check_reference_line(line, n):
    import bench

    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC and line["unit"] == "TFLOP/s"
    assert line["value"] > 0 and line["ms_per_step"] > 0 and line["higher_is_better"] is True
    for k, v in bench.workload_config(n, n // 2).items():
        assert line["config"][k] == v
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == line["value"] and cb["cores"] >= 1 and cb["sample"]
    assert line["e2e"] == {"value": line["value"], "unit": line["unit"], "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}


def test_reference_arm_prints_one_contract_line():
    n = 256
    res = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--n", str(n), "--steps", "2",
                          "--warmup", "1"], cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert res.returncode == 0, res.stderr
    lines = _json_lines(res.stdout)
    assert len(lines) == 1
    _check_reference_line(lines[0], n)
    assert lines[0]["steps"] == 2 and lines[0]["warmup"] == 1


def test_reference_arm_under_torchrun_prints_on_rank_zero_only():
    n = 128
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes", "1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py", "--impl", "reference",
           "--gpus", "2", "--size", str(n), "--steps", "1", "--warmup", "1"]
    res = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert res.returncode == 0, res.stderr[-2000:]
    lines = _json_lines(res.stdout)
    assert len(lines) == 1
    _check_reference_line(lines[0], n)
    assert lines[0]["n_gpus"] == 2


@pytest.mark.parametrize("n,big", [(8192, True), (4096, False)])
def test_l2_note_states_whether_inputs_exceed_l2(n, big):
    import bench

    note = bench.l2_note(n)
    assert note.startswith("inputs larger than L2" if big else "inputs NOT larger than L2")
    assert f"{n * n * 8 / 1e6:.0f} MB FP64" in note


def test_executed_flops_count_the_upper_triangle_tiles():
    """The roofline's executed rate counts every tile with at least one element on or
    above the diagonal (256 x 256 for CTA pairs, 128 x 256 for single CTAs, the last
    tiles overhanging the padded size) and three split products per tile and layer."""
    import bench

    def enumerate_tiles(n, bm, bn=256):
        np_ = -(-n // 128) * 128
        return sum(1 for bj in range(-(-np_ // bn)) for bi in range(-(-np_ // bm)) if bi * bm < (bj + 1) * bn), np_

    for n in (128, 300, 1000, 4096, 8192):
        for cg, bm in ((2, 256), (1, 128)):
            t, np_ = enumerate_tiles(n, bm)
            assert bench.chain_executed_flops(n, 3, cg) == 3 * t * 3 * 2.0 * bm * 256 * np_
    # N = 8192 with CTA pairs: 528 tiles per layer, 5.44e13 flops over 32 layers
    assert bench.chain_executed_flops(8192, 32, 2) == 32 * 528 * 3 * 2.0 * 256 * 256 * 8192
