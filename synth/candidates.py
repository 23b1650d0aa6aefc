"""Grasp-candidate initialisations.

The paper samples hand initialisations with an approach-sampling procedure it does
not specify (Sec. IV-A); the workloads here place the palm on a sphere around the
object centre with a uniformly random orientation and joint angles uniform within
their limits.  The base rotation is stored as a rotation vector w, so the
configuration is q = (t[3], w[3], theta[J]).
"""

from __future__ import annotations

import math
import numpy as np


def uniform_quaternions(rng: np.random.Generator, n: int) -> np.ndarray:
    """Uniform random unit quaternions (w, x, y, z) by Shoemake's subgroup method."""
    u1, u2, u3 = rng.random(n), rng.random(n), rng.random(n)
    a, b = np.sqrt(1.0 - u1), np.sqrt(u1)
    x = a * np.sin(2 * math.pi * u2)
    y = a * np.cos(2 * math.pi * u2)
    z = b * np.sin(2 * math.pi * u3)
    w = b * np.cos(2 * math.pi * u3)
    return np.stack([w, x, y, z], axis=-1)


def quat_to_rotvec(quat: np.ndarray) -> np.ndarray:
    """Rotation vector (axis * angle, angle in [0, pi]) of unit quaternions (w, x, y, z)."""
    q = np.where(quat[:, :1] < 0, -quat, quat)
    v = q[:, 1:]
    s = np.linalg.norm(v, axis=1)
    ang = 2.0 * np.arctan2(s, q[:, 0])
    scale = np.where(s > 1e-12, ang / np.where(s > 1e-12, s, 1.0), 2.0)
    return v * scale[:, None]


def sample_candidates(rng: np.random.Generator, hand: dict, n: int, radius: float,
                      centre=(0.0, 0.0, 0.0)) -> np.ndarray:
    """n candidates: palm origin on a sphere of ``radius`` around ``centre``, uniform
    orientation, joint angles ~ U(q_low, q_up).  Returns float32 [n, 6 + J]."""
    d = rng.normal(size=(n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    t = np.asarray(centre)[None, :] + radius * d
    w = quat_to_rotvec(uniform_quaternions(rng, n))
    lo, hi = hand["q_low"].astype(np.float64), hand["q_up"].astype(np.float64)
    th = lo[None, :] + (hi - lo)[None, :] * rng.random((n, hand["J"]))
    return np.concatenate([t, w, th], axis=1).astype(np.float32)


def unit_directions(n: int, dim: int = 6, seed: int = 2306081320) -> np.ndarray:
    """n seeded directions uniform on the unit sphere of R^dim (normalised Gaussians), float32."""
    rng = np.random.default_rng(seed)
    g = rng.normal(size=(n, dim))
    return (g / np.linalg.norm(g, axis=1, keepdims=True)).astype(np.float32)
