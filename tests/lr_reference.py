"""FP64 plaintext reference of the worker's update (Li & Huang, Eq. 5-8).

w' = w + lr * sum_i p(y_i w.x_i) y_i x_i, with p the Table 2 polynomial of
the loss gradient.  Table 2's polynomials are positive at 0 and decreasing,
i.e. they approximate the negated derivative of the loss (for the binomial
deviance, sigma(-m)); the update therefore adds lr * sum p(.) y x, which is
a descent step on the loss of Eq. 4, with the L2 regulariser's gradient when
l2 > 0."""
import os

import numpy as np

_GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                       "table2_gradient_polynomials.txt")


def table2():
    out = {}
    with open(_GOLDEN) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            name, *vals = line.split()
            out[name] = [float(v) for v in vals]
    return out


def poly(coeffs, x):
    c0, c1, c2, c3 = coeffs
    return c0 + c1 * x + c2 * x * x + c3 * x * x * x


def lr_step_fp64(X, y, w, coeffs, lr, l2=0.0):
    """One step; l2 > 0 adds the gradient l2 * w of the regulariser
    R(w) = (l2/2) |w|^2 of Eq. 4 (Eq. 6, 8): w' = w + lr (sum p y x - l2 w)."""
    m = y * (X @ w)
    return w + lr * ((poly(coeffs, m) * y) @ X - l2 * w)
