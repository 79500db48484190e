"""Shared set-up for the GPU tests: seeded graphs on the device, the oracle's
view of the same matrix, and a solver built through the C ABI."""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import torch

import synth


def graph(spec: synth.GraphSpec):
    rp, c, v = synth.make_graph(spec)
    return rp, c, v


def to_scipy(rp, c, v, n):
    return sp.csr_matrix((v.cpu().numpy().astype(np.float64), c.cpu().numpy(), rp.cpu().numpy()), shape=(n, n))


def to_cuda(*ts):
    return [t.cuda().contiguous() for t in ts]


def maxabs(a, b) -> float:
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.max(np.abs(a - b))) if a.size else 0.0
