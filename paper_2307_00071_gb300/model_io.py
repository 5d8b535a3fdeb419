"""Compact storage of a fitted mixture (Sec. IV: the model's size in memory).

A D-dimensional full-covariance component is stored as binary32 values: its
weight, its mean (D values) and the upper triangle of its covariance
(D (D + 1) / 2 values, row by row), i.e. 1 + D + D (D + 1) / 2 floats; for the
paper's D = 4 that is 15 floats (60 bytes) per component.  ``pack_model`` and
``unpack_model`` convert between that byte string and (weights, means, covs)
arrays; nothing here runs on the GPU.
"""
from __future__ import annotations

import numpy as np


def floats_per_component(d: int) -> int:
    return 1 + d + d * (d + 1) // 2


def model_bytes(k: int, d: int = 4) -> int:
    """Bytes of a K-component model in the compact binary32 layout."""
    return 4 * k * floats_per_component(d)


def pack_model(weights, means, covs) -> bytes:
    """(K,), (K, D), (K, D, D) -> the compact little-endian binary32 byte string."""
    w = np.asarray(weights, np.float64).reshape(-1)
    m = np.asarray(means, np.float64)
    c = np.asarray(covs, np.float64)
    k, d = m.shape
    if w.shape != (k,) or c.shape != (k, d, d):
        raise ValueError("weights (K,), means (K, D), covs (K, D, D) expected")
    iu = np.triu_indices(d)
    rows = np.concatenate([w[:, None], m, c[:, iu[0], iu[1]]], axis=1)
    return rows.astype("<f4").tobytes()


def unpack_model(data: bytes, d: int = 4):
    """The inverse of pack_model: (weights (K,), means (K, D), covs (K, D, D)) as float32."""
    f = floats_per_component(d)
    rows = np.frombuffer(data, dtype="<f4")
    if rows.size % f:
        raise ValueError("byte string is not a whole number of components")
    rows = rows.reshape(-1, f)
    k = rows.shape[0]
    iu = np.triu_indices(d)
    covs = np.zeros((k, d, d), np.float32)
    covs[:, iu[0], iu[1]] = rows[:, 1 + d:]
    covs[:, iu[1], iu[0]] = rows[:, 1 + d:]
    return rows[:, 0].copy(), rows[:, 1:1 + d].copy(), covs
