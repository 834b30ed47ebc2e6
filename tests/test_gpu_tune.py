"""The autotuner on the GPU: every candidate shape of the batched engine (CTAs per SM,
routing threshold of the tensor-core path) gives the same results; the chosen one is
among the candidates."""

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

    specs = synth.batch_specs(120, 16, 40, 2, 3, seed=5, seed_base=900000)
    codes = [(synth.random_systematic(s.n, s.k, s.seed), s.n) for s in specs]
    r = tune.autotune_batch(codes, sample=48, blocks_per_sm=(0, 1), route_work_log10=(6, 9))
    assert r["blocks_per_sm"] in (0, 1) and r["route_work_log10"] in (6, 9) and len(r["table"]) == 4
    out = []
    for bps, rw in ((0, 9), (r["blocks_per_sm"], r["route_work_log10"]), (1, 6)):
        with api.Batch(blocks_per_sm=bps, route_work_log10=rw) as b:
            for G, n in codes:
                b.add(G, n)
            b.run()
            out.append(([b.result(i) for i in range(len(codes))], b.info()["large_codes"]))
    assert out[2][1] > out[0][1]  # a lower threshold routes more codes
    out = [o[0] for o in out]
    for res in out[1:]:
        for a, b in zip(out[0], res):
            assert a["key"] == b["key"] and a["d"] == b["d"]
            assert np.array_equal(a["counts"], b["counts"])
