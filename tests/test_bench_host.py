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


def test_launch_count_matches_the_committed_launch_lists():
    """The ncu launch lists under profiles/ (2D 2048^2 TENO6-MP, 6 RK3 steps in the process:
    3 warm-up, 1 timed, 2 end-to-end) count 90 solver launches without the limiter (face
    2 x 18, primitives 18, update 18, signal speed, dt and time update 6 each) and 126 with
    it (plus 2 x 18 limiter passes): 15 and 21 per step."""
    assert 6 * bench.launches_per_step(2, False) == 36 + 18 + 18 + 6 + 6 + 6
    assert 6 * bench.launches_per_step(2, True) == 36 + 36 + 18 + 18 + 6 + 6 + 6
