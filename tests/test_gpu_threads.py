"""Handles driven from several host threads at once, each on its own stream, with codes
of different shapes, so that the kernels' launch settings (dynamic shared memory
sized by k, the row width, the histogram and the tables of each level) differ from
thread to thread: every run equals the same code's run alone, and the codes with
k <= 36 equal the oracle."""

import threading

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

CODES = [(192, 64, 8), (150, 40, 4), (96, 24, 5), (120, 36, 3), (260, 30, 9), (80, 64, 3)]


@pytest.fixture(scope="module")
def api():
    import torch

    import __graft_entry__

    __graft_entry__.build()
    assert torch.cuda.is_available()
    from paper_1603_06757_gb300 import api

    return api


def _same(got, want):
    for key in ("d", "key", "message", "g_final", "j_final", "m", "L_final"):
        assert got[key] == want[key], key
    assert np.array_equal(got["witness"], want["witness"])
    assert np.array_equal(got["counts"], want["counts"])


def test_threads_with_different_codes(api):
    import torch

    alone = {c: api.min_distance(synth.random_systematic(*c), c[0]) for c in CODES}
    results, errors = {}, []

    def work(c, reps):
        try:
            stream = torch.cuda.Stream()
            with torch.cuda.stream(stream):
                for r in range(reps):
                    results[(c, r)] = api.min_distance(synth.random_systematic(*c), c[0], stream=stream)
        except Exception as e:  # noqa: BLE001 - reported below
            errors.append((c, e))

    threads = [threading.Thread(target=work, args=(c, 3)) for c in CODES]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    assert not errors, errors
    for c in CODES:
        for r in range(3):
            _same(results[(c, r)], alone[c])
    for c in CODES:
        if c[1] <= 36:
            want = oracle.min_distance(synth.random_systematic(*c), c[0])
            _same(alone[c], want)
