"""The oracle-side helpers that build and grade the GPU parity inputs (CPU)."""
import numpy as np

import parity_points as pp
import synth
from oracle import mock, model


def _case(n, box, nr, seed):
    cfg = synth.Config(f"{n}^3", n, box, n_regions=nr, seed_truth=seed, seed_counts=seed + 1)
    bias = synth.default_bias(cfg)
    nu = synth.white_noise(n, seed)
    return cfg, bias, nu, mock.mock_counts(nu, cfg, bias, seed + 1)


def test_bias_terms_sum_to_the_gradient():
    """The per-cell bias-gradient terms sum to the oracle's autograd gradient (alpha and beta, both
    webs), and the absolute sums bound it entry by entry."""
    for n, box, nr, seed in [(16, 160.0, 4, 1101), (16, 200.0, 16, 1201)]:
        cfg, bias, nu, counts = _case(n, box, nr, seed)
        nu = pp.f32(nu)
        _, _, ga, gb = model.logpost_and_grad(nu, counts, cfg, bias)
        abs_a, abs_b, sum_a, sum_b = pp.bias_abs_terms(nu, counts, cfg, bias)
        np.testing.assert_allclose(sum_a, ga, rtol=1e-10, atol=1e-10 * np.abs(ga).max())
        np.testing.assert_allclose(sum_b, gb, rtol=1e-10, atol=1e-10 * np.abs(gb).max())
        assert np.all(abs_a >= np.abs(ga) * (1 - 1e-12)) and np.all(abs_b >= np.abs(gb) * (1 - 1e-12))


def test_off_collapse_keeps_the_gap():
    """Every cell ends at least the gap from D delta0 = 3/2, and nu stays FP32-representable."""
    cfg, bias, nu, counts = _case(32, 300.0, 4, 1001)
    nu = nu * 2.0   # enough cells near the threshold to move some
    x, moved = pp.off_collapse(nu, cfg, 1e-3)
    assert np.array_equal(x, pp.f32(x))
    import torch
    y = cfg.growth_d * model.delta0_from_nu(torch.tensor(x), cfg)
    assert float((y - 1.5).abs().min()) >= 1e-3
    print(f"{moved} cells moved")


def test_clear_near_empty_clears_only_light_cells():
    """Only tracers of cells with CIC mass below 1e-2 go (a field at twice the amplitude has a few
    such cells with tracers at 16^3)."""
    cfg, bias, nu, counts = _case(16, 160.0, 4, 1101)
    nu = pp.f32(2.0 * nu)
    counts = mock.mock_counts(nu, cfg, bias, 1102)
    c = pp.clear_near_empty(nu, counts, cfg, bias)
    rho = 1.0 + model.forward_fields(nu, counts, cfg, bias)["delta"]
    changed = c != counts
    assert changed.sum() > 0
    assert np.all(rho[changed] < 1e-2) and np.all(c[rho < 1e-2] == 0)
    assert np.array_equal(c[rho >= 1e-2], counts[rho >= 1e-2])
