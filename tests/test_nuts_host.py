"""The host-side NUTS driver (paper_2506_03969_gb300.nuts) without a GPU: its control flow --
slice level, doubling directions, subtree proposals, U-turn test, divergence stop -- against the
oracle's NUTS transition on a standard normal target, with the same seeded draws.  A stand-in
context implements the two library calls the driver makes (leapfrog steps with the gradient
carried, FP64 dot products) on CPU tensors."""
import math

import numpy as np
import pytest
import torch

from oracle import hmc


class GaussianContext:
    """bridge_leapfrog_steps / bridge_dot of a one-chain context for log post = -|x|^2 / 2."""
    batch = 1

    def bridge_leapfrog_steps(self, nu, p, grad, counts, biases, n_steps, eps):
        for _ in range(n_steps):
            p += 0.5 * eps * grad
            nu += eps * p
            grad.copy_(-nu)
            p += 0.5 * eps * grad
        return np.array([-0.5 * float((nu.double() ** 2).sum())])

    def bridge_dot(self, a, b):
        return np.array([float((a.double() * b.double()).sum())])


@pytest.mark.parametrize("eps,max_depth", [(0.3, 8), (0.05, 5), (2.5, 6)])
def test_host_nuts_matches_oracle_decisions(eps, max_depth):
    from paper_2506_03969_gb300 import nuts
    grad_fn = lambda x: (-0.5 * float((x ** 2).sum()), -x)
    ctx = GaussianContext()
    sampler = nuts.NUTS(ctx, None, None, eps=eps, max_depth=max_depth)
    rng_o, rng_h, rng_p = np.random.default_rng(11), np.random.default_rng(11), np.random.default_rng(12)
    x_o = np.full(5, 1.5)
    x_h = torch.tensor(x_o)
    g_h, lp_h = -x_h.clone(), -0.5 * float((x_h ** 2).sum())
    for _ in range(20):
        p = rng_p.standard_normal(5)
        x_o, depth_o, steps_o = hmc.nuts_step(x_o, p, None, None, None, eps, rng_o, max_depth=max_depth,
                                              grad_fn=grad_fn)
        res = sampler.step(x_h, torch.tensor(p), g_h, lp_h, rng_h)
        x_h, g_h, lp_h = res.nu, res.grad, res.logpost
        assert res.depth == depth_o and res.n_leapfrog == steps_o
        assert np.allclose(x_h.numpy(), x_o, rtol=0, atol=1e-12)
        assert math.isclose(lp_h, -0.5 * float((x_o ** 2).sum()), rel_tol=1e-12, abs_tol=1e-12)


def test_host_step_size_adaptation_matches_oracle():
    """Warm-up with dual averaging: the host driver's acceptance statistic and adapted step
    sequence against the oracle's NUTS and dual averaging, transition by transition."""
    from paper_2506_03969_gb300 import nuts
    grad_fn = lambda x: (-0.5 * float((x ** 2).sum()), -x)
    ctx = GaussianContext()
    rng_o, rng_h, rng_p = np.random.default_rng(31), np.random.default_rng(31), np.random.default_rng(32)
    x_o = np.full(8, 0.5)
    x_h = torch.tensor(x_o)
    g_h, lp_h = -x_h.clone(), -0.5 * float((x_h ** 2).sum())
    da_o, da_h = hmc.DualAveraging(0.02), nuts.StepSizeAdaptation(0.02)
    eps_o = eps_h = 0.02
    for _ in range(40):
        p = rng_p.standard_normal(8)
        x_o, depth_o, steps_o, a_o = hmc.nuts_step(x_o, p, None, None, None, eps_o, rng_o, max_depth=6,
                                                   grad_fn=grad_fn, with_accept=True)
        res = nuts.NUTS(ctx, None, None, eps=eps_h, max_depth=6).step(x_h, torch.tensor(p), g_h, lp_h, rng_h)
        x_h, g_h, lp_h = res.nu, res.grad, res.logpost
        assert res.depth == depth_o and res.n_leapfrog == steps_o
        assert abs(res.accept_stat - a_o) < 1e-12
        eps_o, eps_h = da_o.update(a_o), da_h.update(res.accept_stat)
        assert math.isclose(eps_h, eps_o, rel_tol=1e-12)
    assert math.isclose(da_h.adapted_eps, da_o.final_eps, rel_tol=1e-12)
    assert 0.3 < da_h.adapted_eps < 2.0


def test_host_nuts_rejects_batched_contexts():
    from paper_2506_03969_gb300 import nuts
    ctx = GaussianContext()
    ctx.batch = 2
    with pytest.raises(ValueError):
        nuts.NUTS(ctx, None, None, eps=0.1)
