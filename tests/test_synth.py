"""The seeded scene generator: drawing scenes in several processes and
concatenating them gives the arrays one process draws, and subsets of a
batch reproduce the batch's scenes."""
import dataclasses

import numpy as np

from paper_2310_08710_b300 import synth


def _same(a, b):
    for f in dataclasses.fields(a):
        x, y = getattr(a, f.name), getattr(b, f.name)
        if isinstance(x, np.ndarray):
            assert x.dtype == y.dtype and x.shape == y.shape, f.name
            assert np.array_equal(x, y), f.name
        elif f.name != "extra":
            assert x == y, f.name


def test_parallel_draw_equals_serial():
    for cfg, S in ((2, 9), (4, 5)):
        serial = synth.make_batch(cfg, seed=3, S=S, R=None if cfg == 2 else 3000)
        par = synth.make_batch(cfg, seed=3, S=S, R=None if cfg == 2 else 3000, workers=2)
        _same(serial, par)


def test_concat_of_subsets_is_the_batch():
    b = synth.make_batch(2, seed=1, S=6)
    _same(synth.concat([b.subset([0, 1, 2]), b.subset([3]), b.subset([4, 5])]), b)
