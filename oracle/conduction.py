"""Steady heat-conduction solutions used to check the kinetic walls.

TEST INFRASTRUCTURE ONLY: loaded by the tests, never by the library.

cavity_series is the steady temperature of the cavity heated at the top as
the paper prints it (Sec. "2D cavity heated at the top"): a sine series
in x times sinh(n pi y / L) / sinh(n pi H / L), with T = T0 on the side and
bottom walls and T = T1 on the top wall."""
import math

import numpy as np


def cavity_series(X, Y, L, H, nmax=399):
    """(T - T0) / (T1 - T0) at (X, Y), 0 <= X <= L, 0 <= Y <= H:
    (2 / pi) sum_{n <= nmax} ((-1)^(n+1) + 1) / n sin(n pi X / L) sinh(n pi Y / L) / sinh(n pi H / L).
    The sinh ratio is evaluated as exp(a - b) (1 - exp(-2a)) / (1 - exp(-2b)), which does not
    overflow for large n."""
    s = np.zeros(np.broadcast(X, Y).shape)
    for n in range(1, nmax + 1):
        c = ((-1) ** (n + 1) + 1) / n
        if c == 0:
            continue
        a = n * math.pi * np.asarray(Y, dtype=np.float64) / L
        b = n * math.pi * H / L
        s += (2 / math.pi) * c * np.sin(n * math.pi * np.asarray(X) / L) * np.exp(a - b) * (1 - np.exp(-2 * a)) / (
            1 - np.exp(-2 * b))
    return s
