"""The single-code workloads: sizes, seeds and the information-set ranks each one
asks for.  The caller supplies the rank function (the library's or the oracle's)."""

from __future__ import annotations

from . import accept_seed, random_systematic

# name -> (n, k, wanted ranks or None, first seed)
SINGLE = {
    "60x30": (60, 30, None, 1),
    "192x64": (192, 64, [64, 64, 64], 1),
    "150x64": (150, 64, [64, 64, 22], 1),
    "300x50": (300, 50, [50] * 6, 1),
    "96x64": (96, 64, None, 1),
    "112x64": (112, 64, None, 1),
}


def single_code(name: str, rank_fn):
    """(n, k, seed, G) for a named single-code workload; seeds are tried upwards from
    the listed one until the ranks match (when ranks are asked for)."""
    n, k, ranks, seed0 = SINGLE[name]
    if ranks is None:
        return n, k, seed0, random_systematic(n, k, seed0)
    seed, G = accept_seed(n, k, ranks, rank_fn, seed0)
    return n, k, seed, G
