"""The stage-2 tile autotuner (hf_autotune): picks one of its candidate tile
sizes from timed runs, and results after tuning still equal the oracle's."""
import pytest

import synth
from synth import analyses
from tests.parity import assert_parity

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("model,V", [("semi", 16), ("semi", 1), ("dilep", 8)])
def test_autotune_choice_and_parity(orc, model, V):
    import torch
    assert torch.cuda.is_available()
    from paper_2211_14346_gb300 import build, Engine, DeviceColumns
    build.build()
    if model == "semi":
        an, cols, seed = analyses.config2(), synth.gen_semilep(3000, 71), 5
        cands = (128, 256, 512, 1024)
    else:
        an, cols, seed = analyses.config3(), synth.gen_dilep(300, 72), 6
        cands = (32, 64, 128, 256)
    with Engine(0) as eng:
        aid = eng.define(an)
        dc = DeviceColumns(cols)
        k = eng.autotune(aid, dc, V=V, seed=seed)
        assert k in cands
        g = eng.run_device(aid, dc, V=V, seed=seed).numpy()
        assert eng.device_error() == 0
    o = orc.run(an, cols, seed=seed, V=V)
    assert_parity(g, o, model="dilep" if model == "dilep" else "semilep", what="after autotune %s V=%d" % (model, V))
