"""Error measures shared by the GPU parity tests, and an optional report.

Every comparison is made twice: norm-wise (|a - b|_2 / |b|_2) and element by
element (max |a - b| / max |b| for signed outputs such as the predictive
mean or a gradient; max |a - b| / |b| for positive outputs such as the
predictive variance).  When the environment variable LMA_PARITY_REPORT names
a file, each measured error is appended to it as one JSON line (test,
quantity, measure, value, bound), so that the bounds can be compared with
what the hardware delivers.
"""
from __future__ import annotations

import json
import os

import numpy as np


def rel(a, b) -> float:
    a, b = np.asarray(a, dtype=np.float64), np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(1e-300, np.linalg.norm(b)))


def max_scaled(a, b) -> float:
    """max |a - b| / max |b| (signed outputs)."""
    a, b = np.asarray(a, dtype=np.float64), np.asarray(b, dtype=np.float64)
    return float(np.max(np.abs(a - b)) / max(1e-300, np.max(np.abs(b)))) if b.size else 0.0


def max_rel(a, b) -> float:
    """max |a - b| / |b| (positive outputs)."""
    a, b = np.asarray(a, dtype=np.float64), np.asarray(b, dtype=np.float64)
    return float(np.max(np.abs(a - b) / np.maximum(np.abs(b), 1e-300))) if b.size else 0.0


def report(test: str, quantity: str, measure: str, value: float, bound: float) -> None:
    path = os.environ.get("LMA_PARITY_REPORT")
    if not path:
        return
    with open(path, "a") as fh:
        fh.write(json.dumps({"test": test, "quantity": quantity, "measure": measure, "value": value,
                             "bound": bound}) + "\n")


def check(test: str, quantity: str, a, b, tol_norm: float, tol_elem: float, positive: bool = False) -> None:
    """Assert (and report) the norm-wise and the element-wise error of a against b."""
    en = rel(a, b)
    ee = max_rel(a, b) if positive else max_scaled(a, b)
    report(test, quantity, "norm", en, tol_norm)
    report(test, quantity, "elem", ee, tol_elem)
    assert en <= tol_norm, f"{test}: {quantity} norm-wise error {en:.3e} > {tol_norm:.1e}"
    assert ee <= tol_elem, f"{test}: {quantity} element-wise error {ee:.3e} > {tol_elem:.1e}"


def check_scalar(test: str, quantity: str, a: float, b: float, tol: float) -> None:
    e = abs(a - b) / max(1e-300, abs(b))
    report(test, quantity, "scalar", e, tol)
    assert e <= tol, f"{test}: {quantity} relative error {e:.3e} > {tol:.1e}"


class Collector:
    """Runs every check and reports every measured error before failing with
    the list of exceeded bounds (so that one run records them all)."""

    def __init__(self):
        self.errors = []

    def check(self, *a, **k):
        try:
            check(*a, **k)
        except AssertionError as e:
            self.errors.append(str(e))

    def check_scalar(self, *a, **k):
        try:
            check_scalar(*a, **k)
        except AssertionError as e:
            self.errors.append(str(e))

    def done(self):
        assert not self.errors, "; ".join(self.errors)
