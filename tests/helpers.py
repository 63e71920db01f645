"""Test helpers: conversion of the oracle's complex expansions to the real
form used by the library, and cached oracle runs."""
import numpy as np


def complex_to_real(X, L):
    """[..., (L+1)^2] complex (index l*l+l+m) -> [..., (L+1)^2] real form
    (for each l: Re m=0, then Re, Im for m = 1..l)."""
    out = np.zeros(X.shape[:-1] + ((L + 1) ** 2,))
    for l in range(L + 1):
        out[..., l * l] = X[..., l * l + l].real
        for m in range(1, l + 1):
            out[..., l * l + 2 * m - 1] = X[..., l * l + l + m].real
            out[..., l * l + 2 * m] = X[..., l * l + l + m].imag
    return out


def rel_err(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def tau_in_gap(norm2, q, gap=1e-6):
    """A threshold between two consecutive distinct pair norms near the
    q-quantile whose ratio exceeds 1 + gap, so that no pair sits near it."""
    sq = norm2.shape[0] == norm2.shape[1]
    n = np.unique(np.sqrt(norm2[np.triu_indices(norm2.shape[0])] if sq else norm2))
    k0 = int(q * (len(n) - 1))
    for d in range(len(n)):
        for k in (k0 + d, k0 - d):
            if 0 <= k < len(n) - 1 and n[k + 1] > n[k] * (1 + gap):
                return float(np.sqrt(n[k] * n[k + 1]))
    raise ValueError("no gap")
