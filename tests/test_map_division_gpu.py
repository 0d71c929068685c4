"""The FP32 map's division against IEEE division.

The FP32 epilogues (Eq. dyn: F = u / (theta_j - theta_{i_c}), u = Z d - P) divide
by multiplying u with the hardware reciprocal estimate of the gap refined by one
Newton-Raphson step.  Over the gaps and numerators the map meets (both signs,
gaps 1e-6 .. 1e5, numerators 1e-10 .. 1e2) the quotient must stay within 2 units
in the last place of the correctly rounded IEEE quotient, and powers of two must
divide exactly.
"""

import numpy as np
import pytest
import torch

from paper_2012_14702_gb300 import workloads as w

pytestmark = pytest.mark.gpu


def ordered(x):
    """float32 -> integers whose differences count units in the last place."""
    i = np.asarray(x, dtype=np.float32).view(np.int32).astype(np.int64)
    return np.where(i < 0, -(i & 0x7FFFFFFF), i)


def test_refined_reciprocal_within_two_ulp_of_ieee(ipt):
    g = w.rng(123)
    m = 1 << 20
    gap = (10.0 ** g.uniform(-6, 5, m) * g.choice([-1.0, 1.0], m)).astype(np.float32)
    u = (10.0 ** g.uniform(-10, 2, m) * g.choice([-1.0, 1.0], m)).astype(np.float32)
    # the gaps of the dense workloads: (i - j) / 8 in FP32
    ij = g.integers(1, 8192, size=(2, 4096))
    gap[:4096] = ((ij[0] - ij[1]) / 8.0).astype(np.float32)
    gap[:4096][gap[:4096] == 0] = 0.125
    q = ipt.check_map_division(torch.as_tensor(gap, device="cuda"),
                               torch.as_tensor(u, device="cuda")).cpu().numpy()
    ref = u / gap  # float32 / float32: IEEE, correctly rounded
    assert ref.dtype == np.float32
    d = np.abs(ordered(q) - ordered(ref))
    assert d.max() <= 2, (d.max(), np.argmax(d))
    assert d.mean() < 0.5


def test_refined_reciprocal_exact_for_powers_of_two(ipt):
    e = np.arange(-20, 21)
    gap = np.concatenate([2.0 ** e, -(2.0 ** e)]).astype(np.float32)
    u = np.full_like(gap, 3.0)
    q = ipt.check_map_division(torch.as_tensor(gap, device="cuda"),
                               torch.as_tensor(u, device="cuda")).cpu().numpy()
    np.testing.assert_array_equal(q, u / gap)
