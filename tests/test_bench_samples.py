"""The oracle's samples that bench.py times on the host cores (CPU): every part of a split is
a valid mesh of the requested size taken from the workload, the parts start at different
places, and one worker process's oracle pass counts the sample's candidate pairs."""
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import bench  # noqa: E402
import oracle as O  # noqa: E402
import ttie_inputs as ti  # noqa: E402


def _check(sub, m):
    assert sub.F > 0 and sub.tri.min() >= 0 and sub.tri.max() < sub.V
    assert np.isin(sub.x, m.x).all()   # positions come from the workload


def test_grid_patches_spread_over_the_cloth():
    m = ti.cloth(256, seed=2).as_f32()
    subs = [bench.oracle_sample(m, 20, 0, part=i, parts=4) for i in range(4)]
    for s in subs:
        _check(s, m)
        assert s.F == 2 * 19 * 19          # a 20 x 20-vertex patch
    assert len({tuple(s.x[0]) for s in subs}) == 4


def test_patches_around_different_triangles():
    m = ti.two_icospheres().as_f32()
    subs = [bench.oracle_sample(m, 8, 0, part=i, parts=3) for i in range(3)]
    for s in subs:
        _check(s, m)
        assert s.F == 2 * 8 * 8
    assert len({s.x.tobytes() for s in subs}) == 3


def test_instance_samples_start_at_different_instances():
    m, _, _ = ti.ellipsoid_batch(12, seed=4, f_min=60, f_max=600)
    m = m.as_f32()
    subs = [bench.oracle_sample(m, 10, 2, part=i, parts=3) for i in range(3)]
    for s in subs:
        _check(s, m)
    assert subs[0].group.min() < subs[1].group.min() < subs[2].group.min()


def test_worker_counts_the_sample_candidates():
    m = ti.two_icospheres().as_f32()
    sub = bench.oracle_sample(m, 6, 1)
    n, secs = bench._oracle_worker(sub, 1, 0.0)
    assert n == len(O.candidate_pairs(sub.x, sub.tri, sub.group, "inter")) and secs > 0
