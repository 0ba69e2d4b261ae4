"""Packed <-> dense conversion for antisymmetric amplitude tensors (oracle side).

Dense layout: t[h1, ..., h_nh, p1, ..., p_np] (holes first, then particles),
antisymmetric under any permutation within the hole group and within the
particle group. Packed layout: the unique elements h1<...<h_nh, p1<...<p_np,
holes-major, each group in lexicographic order of strictly increasing tuples.

Parity: pinned by the round-trip and sign tests in tests/test_oracle_pins.py.
"""
from __future__ import annotations

import itertools
import math
import numpy as np


def _perm_sign(perm):
    perm = list(perm)
    sign = 1
    for i in range(len(perm)):
        while perm[i] != i:
            j = perm[i]
            perm[i], perm[j] = perm[j], perm[i]
            sign = -sign
    return sign


def packed_size(nh, np_, o, v):
    """Number of unique elements: C(o, nh) C(v, np)."""
    return math.comb(o, nh) * math.comb(v, np_)


def unpack(packed, nh, np_, o, v):
    """Dense antisymmetric tensor from packed unique elements."""
    hs = list(itertools.combinations(range(o), nh))
    ps = list(itertools.combinations(range(v), np_))
    vals = np.asarray(packed, dtype=np.float64).reshape(len(hs), len(ps))
    out = np.zeros((o,) * nh + (v,) * np_)
    if len(hs) == 0 or len(ps) == 0:
        return out
    harr = np.array(hs, dtype=int).reshape(len(hs), nh)
    parr = np.array(ps, dtype=int).reshape(len(ps), np_)
    for hp in itertools.permutations(range(nh)):
        sh = _perm_sign(hp)
        for pp in itertools.permutations(range(np_)):
            s = sh * _perm_sign(pp)
            hidx = [harr[:, hp[k]][:, None] for k in range(nh)]
            pidx = [parr[:, pp[k]][None, :] for k in range(np_)]
            out[tuple(hidx + pidx)] = s * vals
    return out


def pack(dense, nh, np_, o, v):
    """Unique elements (h increasing, p increasing) of a dense tensor."""
    hs = list(itertools.combinations(range(o), nh))
    ps = list(itertools.combinations(range(v), np_))
    if len(hs) == 0 or len(ps) == 0:
        return np.zeros(0)
    harr = np.array(hs, dtype=int).reshape(len(hs), nh)
    parr = np.array(ps, dtype=int).reshape(len(ps), np_)
    hidx = [harr[:, k][:, None] for k in range(nh)]
    pidx = [parr[:, k][None, :] for k in range(np_)]
    return np.asarray(dense)[tuple(hidx + pidx)].reshape(-1).copy()
