"""The benchmark's byte models, checked on the CPU: the unfused pass model of
one mu_ex (26 real 3D transforms for three species, three passes each, read
and write of the padded grid) and this design's per-stage algorithmic bytes,
which must stay far below it (fused stages, zero rows skipped)."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

DIMS = (128, 128, 128, 256, 256, 256)


def test_pass_model_of_the_bench_workload():
    # 26 transforms x 3 passes x (read + write) x 256^3 values
    assert bench.pass_model_bytes(DIMS, 3, 8) == 26 * 3 * 2 * 256 ** 3 * 8      # 20.94 GB in FP64
    assert bench.pass_model_bytes(DIMS, 3, 4) == 26 * 3 * 2 * 256 ** 3 * 4      # 10.47 GB in FP32
    # two species: 2 + 10 + 9 + 2 = 23 transforms
    assert bench.pass_model_bytes(DIMS, 2, 4) == 23 * 3 * 2 * 256 ** 3 * 4


def test_path_bytes_are_the_stage_sum():
    for cs in (8, 16):
        assert bench.path_bytes(DIMS, cs, 3) == sum(bench.stage_bytes(n, DIMS, cs, 3) for n in bench.STAGES)
    # the z_back stage is the bench's dominant FP32 kernel: 568 MB per launch
    assert bench.stage_bytes("z_back", DIMS, 8, 3) == 568416828
    assert bench.path_bytes(DIMS, 8, 3) < 0.3 * bench.pass_model_bytes(DIMS, 3, 4)


def test_kernels_per_step_of_the_bench_workload():
    # nine stages, the derivative stage split into three kernels on a register length
    assert sum(bench.kernels_per_stage(n, 256) for n in bench.STAGES) == 11
    assert sum(bench.kernels_per_stage(n, 270) for n in bench.STAGES) == 9


def test_oracle_sweep_timing_helper():
    """The film workload's CPU baseline: the oracle's per-sweep time on a small
    film (timing only; the sweep itself is pinned elsewhere)."""
    from workloads import film_gummel
    per, threads = bench.oracle_sweep_seconds(film_gummel(8, 8, 8), 2)
    assert per > 0 and threads >= 1


def test_oracle_rate_helper_restores_threads():
    """The CPU legs of the benchmark: the oracle's mu_ex rate on a sub-box, at
    all cores and at one core, leaving the thread count as it found it."""
    from oracle import oracle
    from workloads import mu_microbench
    spec, rho = mu_microbench(16)
    before = oracle.num_threads()
    v, used, dt = bench.oracle_mu_rate(spec, rho, 6, threads=1)
    assert v > 0 and used == 1 and dt > 0
    assert oracle.num_threads() == before
    v2, used2, _ = bench.oracle_mu_rate(spec, rho, 6)
    assert v2 > 0 and used2 == before
