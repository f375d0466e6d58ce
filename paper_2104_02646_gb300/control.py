"""The paper's controller for its visuomotor control experiments (Sec. 3,
architecture in App. D), as a torch module that drives the simulator's
time-varying actuation.

The simulation time t goes through N phase-shifted sinusoids
s_k(t) = sin(omega t + 2 pi k / N), then one fully connected layer without
bias, then tanh, giving one activation per actuated element:
a_e(t) = amplitude * tanh(sum_k W_ek s_k(t)).  The activations feed
``autograd.actuated_rollout`` as the per-step actuation sequence, so a loss on
the final state back-propagates through the library's adjoint into W.
"""
from __future__ import annotations

import math

import torch


class SinusoidController(torch.nn.Module):
    def __init__(self, n_out: int, n_sin: int = 8, omega: float = 2.0 * math.pi * 10.0, amplitude: float = 0.2,
                 generator: torch.Generator | None = None):
        super().__init__()
        self.n_sin = int(n_sin)
        self.omega = float(omega)
        self.amplitude = float(amplitude)
        w = torch.randn(n_out, self.n_sin, generator=generator) / math.sqrt(self.n_sin)
        self.W = torch.nn.Parameter(w)
        self.register_buffer("phase", 2.0 * math.pi * torch.arange(self.n_sin, dtype=torch.float32) / self.n_sin)

    def forward(self, t: torch.Tensor) -> torch.Tensor:
        """t [S] simulation times -> activations [S][n_out]."""
        s = torch.sin(self.omega * t[:, None].to(self.W.dtype) + self.phase[None, :])
        return self.amplitude * torch.tanh(s @ self.W.t())
