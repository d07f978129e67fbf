"""The process-pool runner of the oracle (used by the full-size GPU parity
tests) gives exactly the single-process result: slices keep their global
event ids, counts are summed, per-event outputs concatenated."""
import numpy as np

import synth
from synth import analyses
from tests import oracle_pool


def test_pool_equals_single_process(orc):
    cols = synth.gen_semilep(3000, 41)
    an = analyses.config2()
    one = orc.run(an, cols, seed=5, V=4, first_event_id=123)
    many = oracle_pool.run(an, cols, seed=5, V=4, first_event_id=123, procs=3, pieces=7)
    for k in ("cutflow", "hist", "mask", "n_surv", "reco", "reco_abs"):
        assert np.array_equal(one[k], many[k]), k
