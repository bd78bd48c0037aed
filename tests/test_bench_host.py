"""The roofline accounting of bench.py (CPU only).

* algorithmic bytes per DOF and stage at N = 4: FP64 32 B of state + 80/9 B
  of metric terms + the face values of the three faces an element owns =
  43.0 B (the per-DOF figure of the survey of this path), FP32 geometry
  37.5 B; the first stage reads no register (8 B less);
* FP64 flops per element as the kernel is written (N = 4: 104,475, 93 per
  DOF), with the staged volume form from N = 6 on, where it costs fewer
  operations than the combined form (equal at N = 5: 36 + 18 n = 24 n).
"""
import bench


def test_bytes_per_dof():
    fp64 = bench.algorithmic_bytes_per_dof(4, 8)
    mixed = bench.algorithmic_bytes_per_dof(4, 4)
    assert abs(fp64 - (32 + 80 / 9 + 3 * 25 * 4 * 8 / (9 * 125))) < 1e-12
    assert abs(fp64 - 43.0) < 0.05
    assert abs(mixed - 37.51) < 0.01
    assert abs(bench.algorithmic_bytes_per_dof(4, 4, first_stage=True) - (mixed - 8)) < 1e-12
    step = bench.step_bytes_per_dof(4, 4)
    assert abs(step - (mixed - 8 + 4 * mixed)) < 1e-12


def test_flops_per_element():
    f4 = bench.algorithmic_flops_per_element(4)
    assert f4 == 125 * (3 * 5 * 42 + 69) + 6 * 25 * 114 == 104475
    assert 92 < f4 / (125 * 9) < 94
    # volume operations per node and direction of the two forms cross at n = 6 (N = 5)
    assert 36 + 18 * 6 == 24 * 6
    for N in (6, 7):
        n = N + 1
        staged = 3 * (27 + 36 * n + 27 + 18) + 69
        assert bench.algorithmic_flops_per_element(N) == n ** 3 * staged + 6 * n * n * 114
