"""Host-side checks of bench.py (no GPU): argument defaults of the measured
workloads and the byte/flop models the roofline objects are built from."""
import json

import bench


def test_default_workload_and_contract_arguments():
    a = bench.parse_args([])
    assert a.gpus == 1 and a.warmup >= 3 and a.impl == "ours"
    # the largest single-GPU configuration: the 384^3 cavity on the learned +
    # mixed-precision path
    assert a.workload == "cavity384" and bench.WORKLOADS["cavity384"]["n"] == 384 and a.solver == "guess"
    assert a.concurrent_diffusion == "on" and a.ir_form == "tuned"
    assert set(bench.SOLVER_DESC) == {"cg", "ir", "fpcg", "guess"}


def test_oracle_sample_scaling_is_stated():
    # the reference arm scales a sampled oracle step by the FP64 CG count
    # measured at 384^3
    assert bench.CG_ITERS_PER_STEP[(384, False)] > bench.CG_ITERS_PER_STEP[(384, True)] > 1000
    assert bench.FP64_PEAK_TFLOPS > 1.0 and "clocks" in bench.FP64_PEAK_SOURCE


def test_byte_models_per_cell():
    # FP32 iteration of the graph form: direction reads r32, p_old and writes
    # p (12 B); the update reads p, r32 and writes r32 (12 B), and reads and
    # writes x32 every other iteration (+8 B): 16 B on average
    assert bench.IR_GRAPH_BYTES_PER_CELL_ITER == 12 + (12 + 20) // 2
    # persistent form: direction also stores q (16 B), update reads q (24 B)
    assert bench.IR_BYTES_PER_CELL_ITER == 16 + 24
    # textbook FP64 CG: (r, p_old -> p, q) 32 B + (x, p, r, q -> x, r) 48 B
    assert bench.CG_BYTES_PER_CELL_ITER == 32 + 48


def test_graph_traffic_matches_the_byte_model():
    # the ncu capture of the 256^3 graph-form solve moved the algorithmic
    # bytes of its FP32 iterations plus a few FP64 passes: within 2 %
    assert bench.IR_GRAPH_DRAM_BYTES_PER_CELL_ITER is not None
    ratio = bench.IR_GRAPH_DRAM_BYTES_PER_CELL_ITER / bench.IR_GRAPH_BYTES_PER_CELL_ITER
    assert 1.0 <= ratio < 1.02


def test_traffic_belongs_to_one_launch_shape():
    assert bench.CGT_CAVITY64_SHAPE == {"blocks": 128, "tile_depth": 8, "register_path": True, "tile_resident": True}
    assert bench.CGT_CAVITY64_DRAM_BYTES > 0 and 0 < bench.CGT_CAVITY64_LTS_PCT < 100


def test_measured_hbm_peak_fallback(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.measured_hbm_gbs(default=1234.0) == 1234.0
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"hbm_gbs": 6000.5}))
    assert bench.measured_hbm_gbs() == 6000.5


def test_aggregate_is_all_ranks_over_the_slowest():
    # 2 ranks x 1000 cells x 10 steps in 2 s (the slowest rank's time)
    assert bench.aggregate(1000, 10, 2, 2.0) == 1000 * 10 * 2 / 2.0


def test_committed_weights_match_the_network_layout():
    """The trained parameters the learned solvers load: the oracle network's
    parameter count, finite values, and a header naming the training run."""
    import os

    import numpy as np
    from oracle import unet

    path = bench.weights_path()
    assert os.path.exists(path) and os.path.exists(path + ".json")
    w = np.fromfile(path, dtype="<f4")
    assert w.size == unet.param_count() and np.isfinite(w).all()
    meta = json.load(open(path + ".json"))
    assert meta["count"] == w.size and meta["n"] == 128 and meta["loss"] == "cos"
