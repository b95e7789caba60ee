"""The batched workload's scene recipes (host logic, no GPU): the default mix draws the same
scenes as before its sizes became parameters, the small mix stays inside its declared ranges, the
pools follow the voxel-size rule, and the recipes are deterministic in their seed."""
import numpy as np

import synth


def _sizes(scenes):
    return [(round(s.volume.voxel_size * 1000), s.volume.max_blocks, s.name) for s in scenes]


def test_default_mix_is_the_recipe_of_the_scaled_rooms():
    scenes = synth.batch_scenes(32, 3)
    assert len(scenes) == 32
    rng = np.random.default_rng(synth.SEED_BASE + 5)
    for s in scenes:
        scale = float(np.exp(rng.uniform(0.0, np.log(3.5))))  # the recipe's own draws, in its order
        l_mm = int(rng.integers(5, 11))
        assert round(s.volume.voxel_size * 1000) == l_mm
        assert s.name == "room_%.1fx%.1fx3_640x480_l%dmm" % (6.0 * scale, 4.0 * scale, l_mm)
        assert s.volume.trunc == 4 * s.volume.voxel_size
        assert (s.W, s.H) == (640, 480) and s.max_range == 4.5
        mb = 1 << 18 if l_mm <= 6 else (1 << 17 if l_mm <= 8 else 1 << 16)
        assert s.volume.max_blocks == mb and s.volume.hash_buckets == 4 * mb


def test_small_mix_and_pool_shift():
    scenes = synth.batch_scenes(32, 3, scale_range=(0.5, 1.0), voxel_mm=(8, 10))
    for l_mm, mb, name in _sizes(scenes):
        assert 8 <= l_mm <= 10
        sx = float(name.split("_")[1].split("x")[0])
        assert 3.0 - 0.05 <= sx <= 6.0 + 0.05
        assert mb == (1 << 17 if l_mm <= 8 else 1 << 16)
    shifted = synth.batch_scenes(4, 3, pool_shift=1)
    plain = synth.batch_scenes(4, 3)
    for a, b in zip(shifted, plain):
        assert a.name == b.name and a.volume.max_blocks == 2 * b.volume.max_blocks


def test_recipes_are_deterministic():
    a, b = synth.batch_scenes(3, 4, seed=synth.SEED_BASE + 99), synth.batch_scenes(3, 4, seed=synth.SEED_BASE + 99)
    for x, y in zip(a, b):
        assert x.name == y.name
        np.testing.assert_array_equal(x.depth(2), y.depth(2))
        np.testing.assert_array_equal(x.pose(3), y.pose(3))
