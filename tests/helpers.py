"""Shared helpers of the tests: parity masks, error norms, library build."""
import os
import subprocess
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def ensure_library():
    from paper_2201_09004_b300 import build
    return build.build()


def parity_mask(dims):
    lx, ly, lz, lt = dims
    t, z, y, x = np.meshgrid(np.arange(lt), np.arange(lz), np.arange(ly), np.arange(lx), indexing="ij")
    return ((x + y + z + t) % 2).astype(np.int64)


def rel_err(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def lex_index(dims, x, y, z, t):
    lx, ly, lz, lt = dims
    return x + lx * (y + ly * (z + lz * t))


# tolerances of the Dslash against the FP64 oracle, per storage precision
TOL = {0: 1e-13, 1: 1e-6, 2: 5e-3, 3: 1e-13}  # 3 = double-float (pairs of FP32)
