"""Scalar functions of the split form and their derivatives (oracle; test infrastructure only).

Function classes of Sec. 3.2.2: rational (numerator/denominator coefficients),
principal square root, exponential, argument/result scaling g(z) = beta f(alpha z)
and combinations (sum, product, quotient, composition). Derivatives follow from
the chain, product and quotient rules (Sec. 3.2.2 notes every function provides
both f and f').

Pinned by tests/test_oracle_fn_band.py against finite differences and closed-form values.
"""
from __future__ import annotations

import numpy as np


def _poly(c, x):
    r = np.zeros_like(x, dtype=np.complex128)
    for a in c:
        r = r * x + a
    return r


def _dpoly(c, x):
    d = len(c) - 1
    r = np.zeros_like(x, dtype=np.complex128)
    for k, a in enumerate(c[:-1]):
        r = r * x + a * (d - k)
    return r


def evaluate(spec: dict, z):
    """Return (g(z), g'(z)) for an array z of complex points."""
    z = np.asarray(z, dtype=np.complex128)
    alpha = complex(spec.get("alpha", 1.0))
    beta = complex(spec.get("beta", 1.0))
    x = alpha * z
    kind = spec["kind"]
    if kind == "rational":
        p, dp = _poly(spec["num"], x), _dpoly(spec["num"], x)
        den = spec.get("den")
        if den is None:
            h, dh = p, dp
        else:
            q, dq = _poly(den, x), _dpoly(den, x)
            h, dh = p / q, (dp * q - p * dq) / (q * q)
    elif kind == "exp":
        h = np.exp(x)
        dh = h
    elif kind == "sqrt":
        h = np.sqrt(x - complex(spec.get("shift", 0.0)))  # numpy: principal branch
        dh = 0.5 / h
    elif kind == "combine":
        a, da = evaluate(spec["a"], x)
        op = spec["op"]
        if op == "compose":
            b, db = evaluate(spec["b"], x)
            h0, dh0 = evaluate(spec["a"], b)
            h, dh = h0, dh0 * db
        else:
            b, db = evaluate(spec["b"], x)
            if op == "add":
                h, dh = a + b, da + db
            elif op == "mul":
                h, dh = a * b, da * b + a * db
            elif op == "div":
                h, dh = a / b, (da * b - a * db) / (b * b)
            else:
                raise ValueError(op)
    else:
        raise ValueError(f"unknown function kind {kind}")
    return beta * h, beta * alpha * dh


def values(spec: dict, z):
    return evaluate(spec, z)[0]


def derivatives(spec: dict, z):
    return evaluate(spec, z)[1]
