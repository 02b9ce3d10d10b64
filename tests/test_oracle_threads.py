"""The oracle's per-gene loops (steps 1, 2 and 5 of Algorithm 1) on several
host threads give bit-identical states and the same counters as on one thread:
each gene's update reads only its own state and its own Philox counters."""
import numpy as np
import pytest

import oracle
from paper_1606_06659_gb300 import synthetic


@pytest.mark.parametrize("all_slice", [0, 1])
def test_threads_do_not_change_the_chain(all_slice):
    d = synthetic.make_config(1, G=700)
    runs = []
    for threads in (1, 4):
        old = oracle.set_threads(threads)
        try:
            ch = oracle.Chain(d["y"], d["X"], d["h"], d["priors"], seed=8, burnin=4,
                              tune_start=2, all_slice=all_slice).init_default()
            for _ in range(6):
                ch.sweep()
            runs.append((ch.get_state(), ch.counters_dict(), ch.moments_dict()))
        finally:
            oracle.set_threads(old)
    (s1, c1, m1), (s4, c4, m4) = runs
    for k in s1:
        assert np.array_equal(s1[k], s4[k]), k
    assert c1 == c4
    for k in m1:
        assert np.array_equal(np.asarray(m1[k]), np.asarray(m4[k])), k
