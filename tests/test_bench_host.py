"""The benchmark's host-side arithmetic (CPU): the distinct table entries a
set of window queries reads, which the window roofline counts as
algorithmic bytes."""
import numpy as np

import bench


def brute_corners(rows, cols, windows):
    pts = set()
    for wh, ww, sy, sx in windows:
        for i in range((rows - wh) // sy + 1):
            for j in range((cols - ww) // sx + 1):
                for y in (i * sy - 1, i * sy + wh - 1):
                    for x in (j * sx - 1, j * sx + ww - 1):
                        if y >= 0 and x >= 0:
                            pts.add((y, x))
    return len(pts)


def test_union_of_corner_sets_equals_brute_force():
    rng = np.random.default_rng(9)
    cases = [[(16, 16, 4, 4), (24, 8, 4, 4), (10, 10, 3, 3)],
             [(5, 7, 1, 1)], [(30, 30, 30, 30), (60, 30, 30, 15)],
             [(64, 64, 16, 16), (128, 128, 16, 16), (16, 32, 16, 16)]]
    for _ in range(20):
        cases.append([(int(rng.integers(1, 40)), int(rng.integers(1, 40)),
                       int(rng.integers(1, 9)), int(rng.integers(1, 9)))
                      for _ in range(int(rng.integers(1, 4)))])
    for ws in cases:
        want = brute_corners(123, 157, ws) * 8 * 2
        assert bench.distinct_corner_bytes_all(123, 157, ws, 2) == want, ws


def test_default_workload_corners_are_the_lattice():
    """Windows 256 and 1,024 at stride 16 on 70,000 x 85,000 read exactly the
    corner lattice of stride 16, S and Q."""
    w = [(256, 256, 16, 16), (1024, 1024, 16, 16)]
    assert bench.distinct_corner_bytes_all(70000, 85000, w, 2) == (70000 // 16) * (85000 // 16) * 16
