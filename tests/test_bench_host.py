"""Host-side pieces of bench.py that set the roofline figures (no GPU).

The roofline's `achieved` is the algorithmic FLOP count of a configuration over
the kernel's time, so the count must be the one the method defines: conv1 on
the taps that can reach fixed sites (the masked input is zero elsewhere), conv2
dense over all sites, conv3 at the updated half of the sites.  These tests count
them independently by enumerating the checkerboard.
"""
import itertools

import numpy as np
import pytest

import bench
import gf_inputs as gi


def live_conv1_taps_per_site(nd, L):
    """Average over all sites (and both fixed parities) of the conv1 taps that
    land on a fixed site of the periodic lattice: only those can be non-zero."""
    coords = np.array(list(itertools.product(range(L), repeat=nd)))
    offs = np.array(list(itertools.product((-1, 0, 1), repeat=nd)))
    total = 0
    for frozen in (0, 1):
        for c in coords:
            nb = (c + offs) % L
            total += int((nb.sum(axis=1) % 2 == frozen).sum())
    return total / (2 * len(coords))


@pytest.mark.parametrize("nd,L,expect", [(2, 4, 4.5), (2, 8, 4.5), (3, 4, 13.5), (3, 6, 13.5)])
def test_live_conv1_taps(nd, L, expect):
    assert live_conv1_taps_per_site(nd, L) == expect


def direct_flops(shape):
    nd, L, C1, C2 = shape.nd, shape.L, shape.c1, shape.c2
    V, T = L ** nd, 3 ** nd
    offs = list(itertools.product((-1, 0, 1), repeat=nd))
    odd = sum(1 for o in offs if sum(o) % 2)
    live = (odd + (T - odd)) / 2                       # half the sites see each count
    conv1 = 2 * V * C1 * live
    conv2 = 2 * V * C1 * C2 * T
    conv3 = 2 * (V // 2) * 2 * C2 * T                  # (s, t) at the updated sites
    return (conv1 + conv2 + conv3) * shape.n_layers


@pytest.mark.parametrize("name", ["c1", "c3"])
def test_flops_per_config_matches_direct_count(name):
    shape = gi.WORKLOADS[name]["shape"]
    assert bench.flops_per_config(shape) == pytest.approx(direct_flops(shape), rel=1e-12)


def test_c3_headline_flop_count():
    # 3D L=16, 16 couplings, hidden 32: 3.794 GFLOP per configuration
    shape = gi.WORKLOADS["c3"]["shape"]
    assert bench.flops_per_config(shape) == pytest.approx(3.793747968e9, rel=1e-12)
