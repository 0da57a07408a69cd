"""The host-side threshold fit of the percolation binding (no GPU): it must
return the midpoint of an exact logistic curve, stay within its own error bar
on binomially sampled fractions, and refuse data it cannot fit."""
import numpy as np
import pytest

from paper_cs_0312006_gb300.percolation import spanning_threshold


def test_exact_logistic_midpoint():
    pc, slope = 0.5927, 180.0
    Ps = pc + np.linspace(-0.02, 0.02, 7) + 0.003
    f = 1.0 / (1.0 + np.exp(-slope * (Ps - pc)))
    p_half, sd = spanning_threshold(Ps, f, 4096)
    assert abs(p_half - pc) < 1e-12
    assert 0.0 < sd < 1e-3


def test_sampled_fractions_cover_the_truth():
    pc, slope, n = 0.6, 120.0, 2000
    Ps = pc + np.linspace(-0.015, 0.015, 5)
    p = 1.0 / (1.0 + np.exp(-slope * (Ps - pc)))
    rng = np.random.default_rng(3)
    z = []
    for _ in range(200):
        f = rng.binomial(n, p) / n
        p_half, sd = spanning_threshold(Ps, f, n)
        z.append((p_half - pc) / sd)
    z = np.array(z)
    assert abs(z.mean()) < 0.3 and 0.8 < z.std() < 1.25


def test_points_at_zero_or_one_are_dropped_and_too_few_refused():
    Ps = [0.50, 0.58, 0.60, 0.70]
    p_half, _ = spanning_threshold(Ps, [0.0, 0.25, 0.75, 1.0], 1000)
    assert abs(p_half - 0.59) < 1e-12  # symmetric logits about 0.59
    with pytest.raises(ValueError):
        spanning_threshold(Ps, [0.0, 0.5, 1.0, 1.0], 1000)
