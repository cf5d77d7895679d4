"""The benchmark's algorithmic byte model and workload naming (host logic,
no GPU).  The field kernels of one 3D step move 49 words per cell: the
right-hand side 3d + 5 (u, p, psi, N(u^{n-1}) in; R, N(u^n) out), the
momentum sweeps 2d, 2d and 3d (the last adds u^n), the psi sweeps d + 5 (the
divergence prologue reads u, D.u^n and p and writes D.u^{n+1}, p and psi),
2 and 4 (the p epilogue)."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

FIELD_SLOTS = ("rhs", "mom_sweep_1", "mom_sweep_2", "mom_sweep_3", "psi_sweep_1", "psi_sweep_2", "psi_sweep_3")
MARKER_SLOTS = ("interp", "update", "force", "spread")


def test_field_words_per_cell():
    for w in (4, 8):
        cells = 128 ** 3
        words = sum(bench.kernel_bytes(k, cells, 0, 0, w) for k in FIELD_SLOTS) / (cells * w)
        assert words == 49


def test_step_bytes_is_the_sum_over_the_slots():
    cells, nm, ne = 128 ** 3, 40962, 122880
    assert set(bench.STEP_SLOTS) == set(FIELD_SLOTS) | set(MARKER_SLOTS)
    total = bench.step_bytes(cells, nm, ne, 4)
    assert total == sum(bench.kernel_bytes(k, cells, nm, ne, 4) for k in bench.STEP_SLOTS)
    # marker kernels scale with the markers and connections only
    assert bench.step_bytes(cells, 0, 0, 4) == 49 * cells * 4
    # the 128^3 FP32 workload: 453 969 440 bytes per step
    assert total == 453969440


def test_marker_models_count_marker_arrays_not_stencil_nodes():
    # interpolation and spreading stream their marker arrays (locations: an
    # index and 4 weights per axis, plus U or G) from HBM; the 4^d stencil
    # nodes are cache traffic, counted as updates instead
    nm = 40962
    for k in ("interp", "spread"):
        assert bench.kernel_bytes(k, 128 ** 3, nm, 0, 4) == nm * 3 * (3 * (4 + 16) + 4)
    assert bench.stencil_updates(nm) == nm * 3 * 64


def test_survey_per_pass_model():
    # 55 words per cell: 461 MB per 128^3 FP32 step, 29.5 GB per 512^3 step
    assert bench.survey_step_bytes(128 ** 3, 4) == 461373440
    assert abs(bench.survey_step_bytes(512 ** 3, 4) - 29.5e9) < 0.05e9


def test_fp64_operation_counts():
    assert bench.fp64_ops("rhs", 10) == 900 and bench.fp64_ops("sweep", 10) == 40


def test_workload_names_its_grid_and_mesh():
    assert bench.WORKLOAD == bench.workload(128, 64)
    assert "128^3" in bench.WORKLOAD and "40962 markers" in bench.WORKLOAD and "122880 springs" in bench.WORKLOAD
    w = bench.workload(256, 32, "FP64 fields")
    assert "256^3" in w and "nu=32" in w and "10242 markers" in w and "FP64 fields" in w


def test_reference_arm_prints_the_contract_line(capsys):
    # the oracle on a small grid: one JSON line with the reference-arm keys
    args = type("A", (), {"steps": 2, "warmup": 1, "n": 16, "nu": 4, "gpus": 1})()
    assert bench.run_reference(args, 0, 1) == 0
    import json
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["unit"] == "cell-updates/s" and line["value"] > 0
    assert line["steps"] == 2 and line["warmup"] == 1 and line["dtype"] == "f64"
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] == 1
    assert line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"] == {"value": line["value"], "unit": line["unit"], "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
    assert "16^3" in line["config"]["workload"]
