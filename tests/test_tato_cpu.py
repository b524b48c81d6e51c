"""The topology-optimisation design chain (Sec. 5.2 'Constraints') on the CPU:
filter, projection and continuation against their definitions written out by
brute force and against closed forms of their derivatives."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2509_15744_gb300 import tato


def brute_filter(g: np.ndarray, rf: float) -> np.ndarray:
    out = np.zeros_like(g)
    idx = list(np.ndindex(*g.shape))
    for i in idx:
        num = den = 0.0
        for k in idx:
            d = math.dist(i, k)
            if d < rf:
                w = rf - d
                num += w * g[k]
                den += w
        out[i] = num / den
    return out


def test_filter_kernel_weights():
    k2 = tato.filter_kernel(1.5, 2, torch.float64).numpy()
    assert k2.shape == (3, 3)
    assert k2[1, 1] == pytest.approx(1.5)
    assert k2[0, 1] == pytest.approx(0.5) and k2[1, 2] == pytest.approx(0.5)
    assert k2[0, 0] == pytest.approx(1.5 - math.sqrt(2.0))
    k3 = tato.filter_kernel(1.5, 3, torch.float64).numpy()
    assert k3[0, 0, 0] == 0.0                           # |x| = sqrt(3) > 1.5
    assert k3[0, 1, 1] == pytest.approx(0.5)
    assert k3[0, 0, 1] == pytest.approx(1.5 - math.sqrt(2.0))
    k12 = tato.filter_kernel(12.0, 2, torch.float64)
    assert k12.shape == (23, 23) and float(k12.min()) >= 0.0


@pytest.mark.parametrize("shape,rf", [((7, 9), 1.5), ((5, 6, 4), 1.5), ((8, 8), 2.7)])
def test_density_filter_matches_definition(shape, rf):
    rng = np.random.default_rng(3)
    g = rng.uniform(0.0, 1.0, shape)
    got = tato.density_filter(torch.from_numpy(g), rf).numpy()
    np.testing.assert_allclose(got, brute_filter(g, rf), rtol=1e-12, atol=1e-14)
    # a constant design is left unchanged, boundaries included
    c = tato.density_filter(torch.full(shape, 0.37, dtype=torch.float64), rf).numpy()
    np.testing.assert_allclose(c, 0.37, rtol=1e-14)


def test_filter_chain_rule_is_the_transposed_filter():
    # d gamma~ / d gamma_k = sum_i w(x_i - x_k) / sum_{k' in N_i} w(x_i - x_k') (Sec. 5.2)
    rng = np.random.default_rng(4)
    shape, rf = (6, 7), 1.5
    g = torch.from_numpy(rng.uniform(0, 1, shape)).requires_grad_(True)
    wout = torch.from_numpy(rng.standard_normal(shape))
    (tato.density_filter(g, rf) * wout).sum().backward()
    idx = list(np.ndindex(*shape))
    ref = np.zeros(shape)
    for i in idx:
        den = sum(rf - math.dist(i, k) for k in idx if math.dist(i, k) < rf)
        for k in idx:
            d = math.dist(i, k)
            if d < rf:
                ref[k] += wout.numpy()[i] * (rf - d) / den
    np.testing.assert_allclose(g.grad.numpy(), ref, rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("beta", [1.0, 1.1 ** 7, 30.0])
def test_projection_values_and_derivative(beta):
    eta = 0.5
    x = torch.linspace(-0.2, 1.2, 57, dtype=torch.float64, requires_grad=True)
    h = tato.heaviside_projection(x, beta, eta)
    assert float(tato.heaviside_projection(torch.tensor(0.0, dtype=torch.float64), beta, eta)) == pytest.approx(0.0, abs=1e-15)
    assert float(tato.heaviside_projection(torch.tensor(1.0, dtype=torch.float64), beta, eta)) == pytest.approx(1.0)
    assert float(tato.heaviside_projection(torch.tensor(eta, dtype=torch.float64), beta, eta)) == pytest.approx(0.5)
    h.sum().backward()
    den = math.tanh(beta * eta) + math.tanh(beta * (1 - eta))
    ref = beta / (den * np.cosh(beta * (x.detach().numpy() - eta)) ** 2)
    # (tiny far-tail derivatives at large beta lose relative digits in 1 - tanh^2)
    np.testing.assert_allclose(x.grad.numpy(), ref, rtol=1e-10, atol=1e-12 * ref.max())
    # monotone, and sharper for larger beta
    assert bool((h[1:] >= h[:-1]).all())


def test_beta_continuation_and_design_range():
    assert tato.beta_schedule(0) == 1.0 and tato.beta_schedule(4) == 1.0
    assert tato.beta_schedule(5) == pytest.approx(1.1) and tato.beta_schedule(12) == pytest.approx(1.21)
    rng = np.random.default_rng(5)
    g = torch.from_numpy(rng.uniform(-0.3, 1.3, (9, 11)))
    d = tato.design(g, 1.5, 1.0)
    assert float(d.min()) >= 0.0 and float(d.max()) <= 1.0
