"""The FP64 oracle spread over the host's cores (test infrastructure).

The oracle is single-threaded C called through ctypes, which releases the GIL for the call,
so threads that each call it on a disjoint slice of the points run in parallel. Each thread
binds its own Oracle (its own pole counter). The integrals are sums over points, so the full
result is the sum of the slices' results; each slice is already a compensated sum, and adding
a few dozen of them in FP64 adds a rounding of ~1e-16 of the magnitude sums, far below every
tolerance the tests apply. Per-point results (n, D) are simply concatenated.
"""
from __future__ import annotations

import concurrent.futures as cf
import os

import numpy as np

import oracle


def workers() -> int:
    return max(1, os.cpu_count() or 1)


def _slices(n: int, parts: int):
    edges = np.linspace(0, n, parts + 1).astype(np.int64)
    return [(int(a), int(b)) for a, b in zip(edges[:-1], edges[1:]) if b > a]


def _run(fn, n_points: int, parts: int | None = None):
    parts = parts or 4 * workers()
    sl = _slices(n_points, parts)
    with cf.ThreadPoolExecutor(workers()) as ex:
        return list(ex.map(fn, sl))


def hamiltonian(sys, pts, w, v=None, terms=oracle.TERM_POTENTIAL | oracle.TERM_KINETIC):
    """(H, A) over all basis functions: the oracle's hamiltonian on slices of the points, summed."""
    def one(r):
        a, b = r
        return oracle.Oracle(sys).hamiltonian(pts[a:b], w[a:b], None if v is None else v[a:b], terms)

    outs = _run(one, len(w))
    H = np.zeros_like(outs[0][0])
    A = np.zeros_like(outs[0][1])
    for h, a in outs:
        H += h
        A += a
    return H, A


def hamiltonian_block(sys, F, pts, w, v=None, terms=oracle.TERM_POTENTIAL | oracle.TERM_KINETIC):
    """(H, A) restricted to the basis functions F, over all points: slices summed."""
    def one(r):
        a, b = r
        return oracle.Oracle(sys).hamiltonian_block(F, pts[a:b], w[a:b], None if v is None else v[a:b], terms)

    outs = _run(one, len(w))
    H = np.zeros_like(outs[0][0])
    A = np.zeros_like(outs[0][1])
    for h, a in outs:
        H += h
        A += a
    return H, A


def density(sys, pts, P):
    """(n, D) at every given point: slices concatenated."""
    def one(r):
        a, b = r
        n, D, _ = oracle.Oracle(sys).density(pts[a:b], P)
        return n, D

    outs = _run(one, len(pts))
    return np.concatenate([o[0] for o in outs]), np.concatenate([o[1] for o in outs])
