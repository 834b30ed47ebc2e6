"""The autotuner on the GPU: every candidate launch shape of the batched engine gives
the same results; the chosen one is among the candidates."""

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


def test_autotuned_batch_shapes_keep_results():
    import torch

    import __graft_entry__

    __graft_entry__.build()
    assert torch.cuda.is_available()
    from paper_1603_06757_gb300 import api, tune

    specs = synth.batch_specs(120, 16, 36, 2, 3, seed=5, seed_base=900000)
    codes = [(synth.random_systematic(s.n, s.k, s.seed), s.n) for s in specs]
    r = tune.autotune_batch(codes, sample=48, blocks_per_sm=(0, 1), rounds_per_graph=(0, 4))
    assert r["blocks_per_sm"] in (0, 1) and r["rounds_per_graph"] in (0, 4) and len(r["table"]) == 4
    out = []
    for bps, rpg in ((0, 0), (r["blocks_per_sm"], r["rounds_per_graph"]), (1, 4)):
        with api.Batch(blocks_per_sm=bps) as b:
            for G, n in codes:
                b.add(G, n)
            b.run(rpg)
            out.append([b.result(i) for i in range(len(codes))])
    for res in out[1:]:
        for a, b in zip(out[0], res):
            assert a["key"] == b["key"] and a["d"] == b["d"]
            assert np.array_equal(a["counts"], b["counts"])
