"""The seeded input generator: determinism and the workload shapes."""
import numpy as np

import synth


def test_seeded_and_shaped():
    a = synth.workload("sars_32x250")
    b = synth.workload("sars_32x250")
    np.testing.assert_array_equal(a.queries.events, b.queries.events)
    q = a.queries
    assert q.nq == 32 and (q.lengths == 250).all()
    assert q.on_target.sum() == 16
    assert a.genome.shape[0] == 29_903 and a.model.shape[0] == 4096
    # raw currents in pA around the pore model's N(90, 12)
    assert 60 < float(q.events.mean()) < 120


def test_uneven_lengths():
    w = synth.workload("sars_uneven_8192", nq=300)
    lens = w.queries.lengths
    assert lens.min() >= 100 and lens.max() <= 500
    assert w.queries.offsets[-1] == lens.sum()


def test_subset_roundtrip():
    w = synth.workload("sars_32x250")
    s = w.queries.subset([3, 1])
    np.testing.assert_array_equal(s.query(0), w.queries.query(3))
    np.testing.assert_array_equal(s.query(1), w.queries.query(1))


def test_flowcell_schedule_is_time_ordered():
    chunks, q = synth.flowcell_schedule(8, 3.0, seed=105)
    t = [c.t for c in chunks]
    assert t == sorted(t)
    last = [c for c in chunks if c.last]
    assert len(last) == q.nq
    for c in last:
        assert c.events.shape[0] == 40
    assert (q.lengths == 250).all()
