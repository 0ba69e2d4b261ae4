"""Oracle: CCSDT amplitude equations and their iterative solution (Eq. 5-7).

Residuals R_n = <Phi^n| e^{-T} H e^{T} |Phi_0> for n = 1, 2, 3 and the energy
of Eq. 7 come from the Wick term lists of oracle/wick.py evaluated on dense
antisymmetric tensors. The equations keep f_ov and off-diagonal Fock blocks,
so they hold for any reference (needed for the 3-electron FCI pin).

Solver (the paper does not say which CC solution it means; the reading here
is the one reached from T1 = 0, T2 = MP2, T3 = 0): Jacobi steps T += R / D with
orbital-energy denominators from diag(f), accelerated by DIIS on the packed
amplitudes, until max|R| < tol_res and |dE| < tol_e.

Parity: residuals pinned to the Fock-space definition on random amplitudes;
converged energies pinned to FCI for 3-electron systems and by extensivity.
"""
from __future__ import annotations

import numpy as np

from . import packing, wick


def denominators(f, o, rank):
    """D_{i..}^{a..} = sum f_ii - sum f_aa as a dense [holes..., particles...] array."""
    fo = np.diag(f)[:o]
    fv = np.diag(f)[o:]
    d = np.zeros((o,) * rank + (len(fv),) * rank)
    for k in range(rank):
        shape = [1] * (2 * rank)
        shape[k] = o
        d = d + fo.reshape(shape)
        shape = [1] * (2 * rank)
        shape[rank + k] = len(fv)
        d = d - fv.reshape(shape)
    return d


def residuals(f, g, o, v, t1, t2, t3):
    """Dense residuals <Phi^n| (H e^T)_c |0>, n = 1..3 (Eq. 6), from the Wick terms."""
    amps = {"t1": t1, "t2": t2, "t3": t3}
    return [wick.evaluate(wick.cc_terms(n), n, n, f, g, amps, o, v) for n in (1, 2, 3)]


def energy(f, g, o, v, t1, t2, t3=None):
    """Correlation energy, Eq. 7 (T3 does not enter)."""
    amps = {"t1": t1, "t2": t2, "t3": t3 if t3 is not None else np.zeros((o,) * 3 + (v,) * 3)}
    return float(wick.evaluate(wick.cc_terms(0), 0, 0, f, g, amps, o, v))


def residuals_packed(f, g, o, v, p1, p2, p3):
    """Eq. 6 residuals of packed amplitudes, returned packed."""
    t1 = packing.unpack(p1, 1, 1, o, v)
    t2 = packing.unpack(p2, 2, 2, o, v)
    t3 = packing.unpack(p3, 3, 3, o, v)
    r = residuals(f, g, o, v, t1, t2, t3)
    return [packing.pack(r[k], k + 1, k + 1, o, v) for k in range(3)]


class Diis:
    def __init__(self, size=8):
        self.size = size
        self.vecs, self.errs = [], []

    def push(self, vec, err):
        self.vecs.append(vec.copy())
        self.errs.append(err.copy())
        if len(self.vecs) > self.size:
            self.vecs.pop(0)
            self.errs.pop(0)

    def extrapolate(self):
        m = len(self.vecs)
        if m < 2:
            return self.vecs[-1]
        b = np.zeros((m + 1, m + 1))
        for i in range(m):
            for j in range(m):
                b[i, j] = self.errs[i] @ self.errs[j]
        b[m, :m] = b[:m, m] = -1.0
        rhs = np.zeros(m + 1)
        rhs[m] = -1.0
        c = np.linalg.lstsq(b, rhs, rcond=None)[0][:m]
        return sum(ci * vi for ci, vi in zip(c, self.vecs))


def ccsdt(f, g, o, v, tol_res=1e-10, tol_e=1e-12, maxiter=200, diis=8, t_init=None):
    """Solve the CCSDT equations. Returns dict(e_corr, t1, t2, t3, iters, res)."""
    d1, d2, d3 = (denominators(f, o, r) for r in (1, 2, 3))
    if t_init is None:
        t1 = np.zeros((o, v))
        t2 = g[o:, o:, :o, :o].transpose(2, 3, 0, 1) / d2
        t3 = np.zeros((o,) * 3 + (v,) * 3)
    else:
        t1, t2, t3 = (np.array(x, copy=True) for x in t_init)
    sizes = [packing.packed_size(r, r, o, v) for r in (1, 2, 3)]
    acc = Diis(diis)
    e_old = None
    res_max = np.inf
    for it in range(1, maxiter + 1):
        r1, r2, r3 = residuals(f, g, o, v, t1, t2, t3)
        e = energy(f, g, o, v, t1, t2)
        res_max = max(np.max(np.abs(x)) if x.size else 0.0 for x in (r1, r2, r3))
        if e_old is not None and res_max < tol_res and abs(e - e_old) < tol_e:
            return dict(e_corr=e, t1=t1, t2=t2, t3=t3, iters=it, res=res_max, converged=True)
        e_old = e
        t1 = t1 + r1 / d1
        t2 = t2 + r2 / d2
        t3 = t3 + r3 / d3
        vec = np.concatenate([packing.pack(t1, 1, 1, o, v), packing.pack(t2, 2, 2, o, v),
                              packing.pack(t3, 3, 3, o, v)])
        err = np.concatenate([packing.pack(r1 / d1, 1, 1, o, v), packing.pack(r2 / d2, 2, 2, o, v),
                              packing.pack(r3 / d3, 3, 3, o, v)])
        acc.push(vec, err)
        vec = acc.extrapolate()
        p = np.split(vec, np.cumsum(sizes)[:-1])
        t1 = packing.unpack(p[0], 1, 1, o, v)
        t2 = packing.unpack(p[1], 2, 2, o, v)
        t3 = packing.unpack(p[2], 3, 3, o, v)
    return dict(e_corr=e, t1=t1, t2=t2, t3=t3, iters=maxiter, res=res_max, converged=False)
