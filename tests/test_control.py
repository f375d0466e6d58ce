"""The App. D controller module on the CPU: N phase-shifted sinusoids of the
simulation time, one fully connected layer without bias, tanh."""
import math

import torch

from paper_2104_02646_gb300.control import SinusoidController


def test_structure_and_invariants():
    g = torch.Generator().manual_seed(0)
    c = SinusoidController(5, n_sin=8, omega=2 * math.pi * 10, amplitude=0.2, generator=g)
    assert c.W.shape == (5, 8) and len(list(c.parameters())) == 1  # no bias
    t = torch.linspace(0.0, 0.3, 61)
    with torch.no_grad():
        a = c(t)
        assert a.shape == (61, 5) and float(a.abs().max()) < 0.2
        # periodic with period 2 pi / omega
        assert torch.allclose(c(t + 2 * math.pi / c.omega), a, atol=1e-5)
        # N equally spaced phases sum to zero: equal weights give no actuation
        c.W.fill_(0.7)
        assert float(c(t).abs().max()) < 1e-5
        # one weight on sinusoid k alone: amplitude tanh(w sin(omega t + 2 pi k / N))
        c.W.zero_()
        c.W[2, 3] = 1.5
        t0 = torch.tensor([0.0123])
        ref = 0.2 * math.tanh(1.5 * math.sin(c.omega * 0.0123 + 2 * math.pi * 3 / 8))
        assert abs(float(c(t0)[0, 2]) - ref) < 1e-6 and float(c(t0)[0, 0]) == 0.0


def test_gradient_reaches_the_weights():
    c = SinusoidController(3, generator=torch.Generator().manual_seed(1))
    t = torch.linspace(0.0, 0.1, 11)
    c(t).sum().backward()
    assert c.W.grad is not None and float(c.W.grad.abs().sum()) > 0
