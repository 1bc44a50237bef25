"""CPU oracle of the Adam optimiser used by the library's two training loops
(the surrogate MLP's weights and the relaxed model's calibration of theta).

TEST INFRASTRUCTURE ONLY: the tests may use this module; the product path never
does.  Plain numpy in FP64.

It follows Kingma and Ba, "Adam: a method for stochastic optimization" (ICLR
2015), Algorithm 1, with the step counter t starting at 1:
    m_t = beta1 m_{t-1} + (1 - beta1) g_t
    v_t = beta2 v_{t-1} + (1 - beta2) g_t^2
    mhat_t = m_t / (1 - beta1^t),   vhat_t = v_t / (1 - beta2^t)
    theta_t = theta_{t-1} - alpha mhat_t / (sqrt(vhat_t) + eps)
with the paper's defaults beta1 = 0.9, beta2 = 0.999, eps = 1e-8.  The
calibration of the relaxed model keeps every parameter non-negative: its step
is followed by the projection theta <- max(theta, 0) (projected gradient
descent onto the non-negative orthant).  The DeepABM paper names gradient-based
calibration (Abstract, Sec. 1, Sec. 6) without fixing an optimiser; Adam with
these defaults is the reading both the oracle and the library take.
Pins: ``tests/test_oracle_adam.py``.
"""
from __future__ import annotations

import numpy as np

BETA1, BETA2, EPS = 0.9, 0.999, 1e-8


class Adam:
    """Adam state over one flat parameter vector (FP64)."""

    def __init__(self, n: int, lr: float, beta1: float = BETA1, beta2: float = BETA2, eps: float = EPS,
                 nonneg: bool = False):
        self.m = np.zeros(n, np.float64)
        self.v = np.zeros(n, np.float64)
        self.t = 0
        self.lr, self.beta1, self.beta2, self.eps, self.nonneg = float(lr), beta1, beta2, eps, nonneg

    def step(self, theta, g) -> np.ndarray:
        """One update of Algorithm 1: returns theta_t from theta_{t-1} and g_t."""
        g = np.asarray(g, np.float64)
        self.t += 1
        self.m = self.beta1 * self.m + (1.0 - self.beta1) * g
        self.v = self.beta2 * self.v + (1.0 - self.beta2) * g * g
        mhat = self.m / (1.0 - self.beta1 ** self.t)
        vhat = self.v / (1.0 - self.beta2 ** self.t)
        out = np.asarray(theta, np.float64) - self.lr * mhat / (np.sqrt(vhat) + self.eps)
        return np.maximum(out, 0.0) if self.nonneg else out
