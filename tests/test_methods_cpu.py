"""Host-side parts of the method variants: TV operators and the u-shift of the
centre search (no GPU)."""
import math

import numpy as np
import torch

from paper_2401_11101_gb300 import regularize as R
from paper_2401_11101_gb300 import search as S


def test_div_is_minus_adjoint_of_grad():
    torch.manual_seed(0)
    for shape in [(5, 6, 7), (1, 4, 3), (2, 1, 5)]:
        u = torch.randn(shape, dtype=torch.float64)
        p = torch.randn((3,) + shape, dtype=torch.float64)
        lhs = float((R.grad(u) * p).sum())
        rhs = -float((u * R.div(p)).sum())
        assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_grad_of_a_ramp_and_shrink():
    u = torch.arange(24, dtype=torch.float64).reshape(2, 3, 4)    # x1 step 1, x2 step 4, x3 step 12
    g = R.grad(u)
    assert torch.all(g[2, :, :, :-1] == 1) and torch.all(g[2, :, :, -1] == 0)
    assert torch.all(g[1, :, :-1] == 4) and torch.all(g[0, :-1] == 12)
    v = torch.tensor([[3.0], [4.0], [0.0]])                        # |v| = 5
    out = R.shrink(v, 2.0)
    assert torch.allclose(out, v * 3.0 / 5.0)
    assert torch.all(R.shrink(v, 6.0) == 0)


def test_shift_u_integer_and_half():
    d = torch.arange(2 * 3 * 8, dtype=torch.float32).reshape(2, 3, 8)
    s2 = S.shift_u(d, 2.0)
    ref = torch.zeros_like(d)
    ref[..., 2:] = d[..., :-2]
    assert torch.equal(s2, ref)
    h = S.shift_u(d, 0.5)
    assert torch.allclose(h[..., 1:], 0.5 * (d[..., 1:] + d[..., :-1]))


def test_sparsity_regions():
    v = torch.zeros(2, 16, 16)
    v[:, 7:9, 7:9] = 1.0                       # a spot in the middle
    assert abs(S.sparsity(v, "center") - 8 / math.sqrt(8)) < 1e-12
    assert S.sparsity(v, "border") == 0
    w = v.clone()
    w[:, 4:12, 4:12] += 0.1                    # spread some mass around: less sparse
    assert S.sparsity(w, "center") > S.sparsity(v, "center")
