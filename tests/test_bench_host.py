"""Host logic of bench.py (CPU): both arms describe a workload with the same config object,
and the oracle's timing sample reports its block."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_grid_configs_name_the_workload():
    for name, (gen, shape, K, lim) in bench.WORKLOADS.items():
        c = bench.grid_config(name, 1, False)
        assert c["workload"] == name and c["shape"] == list(shape) and c["K"] == K
        assert c["parallelism"] == "single" and c["positivity_limiter"] is False
        assert "> L2" in c["l2"]
        assert bench.grid_config(name, 4, True)["parallelism"] == "replicas"


def test_batch_config_counts_the_cells_and_flushes_l2():
    for name, (nprob, seed, nmin, nmax, K, lim) in bench.BATCH_WORKLOADS.items():
        c = bench.batch_config(name, 1)
        assert c["problems"] == nprob and c["K"] == K
        assert nprob * nmin <= c["cells"] <= nprob * nmax
        assert "flushed" in c["l2"]


def test_launch_count_per_step():
    """Launches of one SSP-RK3 step: signal speed, dt and time update, then per stage the
    primitives, one sweep per axis and the cell update: 15 per step in 2D, 18 in 3D; with
    the positivity limiter per stage also a limiter pass per axis: 21 in 2D (the committed
    limited launch list counts 126 solver launches over 6 steps)."""
    assert bench.launches_per_step(2, False) == 3 + 3 * 4
    assert bench.launches_per_step(3, False) == 3 + 3 * 5
    assert 6 * bench.launches_per_step(2, True) == 36 + 36 + 18 + 18 + 6 + 6 + 6
