"""The seeded input generators: drawing the batched workload in several
processes gives exactly the points of the one-process draw."""
import numpy as np

import synth


def test_batched_instances_parallel_equals_serial():
    sizes = synth.batched_sizes(23, seed=3, lo=10, hi=5_000)
    sizes[5] = 0  # an empty instance
    a, oa = synth.batched_instances(sizes, seed=3)
    b, ob = synth.batched_instances(sizes, seed=3, workers=3)
    assert np.array_equal(oa, ob)
    assert a.dtype == b.dtype == np.float32 and a.shape == b.shape == (int(sizes.sum()), 3)
    assert np.array_equal(a.view(np.uint32), b.view(np.uint32))
