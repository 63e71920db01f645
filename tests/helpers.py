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
