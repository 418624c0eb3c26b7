"""Angles for the parity tests, computed in a well-conditioned form.

arccos of a dot product loses half the digits near zero: an FP32 unit vector whose length is
off by one rounding (about 6e-8) already reads as 3.5e-4 rad from itself, a third of the
1e-3 rad normal tolerance. atan2(|a x b|, a . b) measures the angle itself, independent of
the vectors' lengths, to FP64 rounding at every angle.
"""
import numpy as np


def between(a, b):
    """Angle (rad) between the vectors of the last axis of `a` and `b` (any lengths)."""
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return np.arctan2(np.linalg.norm(np.cross(a, b), axis=-1), np.sum(a * b, axis=-1))


def rotation(Ra, Rb):
    """Angle (rad) of the rotation Ra^T Rb, from the chord ||Ra - Rb||_F = 2 sqrt(2) sin(angle / 2)."""
    d = np.linalg.norm(np.asarray(Ra, np.float64) - np.asarray(Rb, np.float64))
    return 2.0 * np.arcsin(min(1.0, d / (2.0 * np.sqrt(2.0))))
