"""The divergence study's shared-start run (every env of a cartridge started
from the same state, paper Section 4, Fig. 3) is bit-exact against the
oracle started the same way, and the lockstep counters it reports are sane.
Each side builds the shared states from its own start-state cache."""
import numpy as np
import pytest
import torch

from paper_1907_08467_gb300 import synth
from paper_1907_08467_gb300.env import FORM_BATCHED
from tests.test_gpu_parity import pair, run_parity

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("config,n,steps", [(2, 96, 40), (3, 64, 40)])
def test_shared_start_run_matches_oracle(config, n, steps):
    w = synth.workload(config, n_envs=n)
    g, o = pair(w.roms, w.env_rom, sticky=w.sticky, seed=w.seed, form=FORM_BATCHED)
    score = [r.score_addr for r in w.roms]
    sg = synth.shared_start_states(g.state().cpu().numpy(), g.cache().cpu().numpy(), w.env_rom, score)
    so = synth.shared_start_states(o.state(), o.cache(), w.env_rom, score)
    assert np.array_equal(sg, so)
    # every env of a cartridge holds the same machine state
    for r in set(w.env_rom):
        rows = so[np.asarray(w.env_rom) == r]
        assert (rows[:, 0x80:] == rows[0, 0x80:]).all() and (rows[:, :0x60] == rows[0, :0x60]).all()
    g.set_state(torch.from_numpy(sg).cuda())
    o.set_state(so)
    run_parity(g, o, synth.actions(60 + config, steps, n))
    ins, _, rounds = g.counters()
    assert rounds > 0 and 0 < ins / rounds <= 1.0
