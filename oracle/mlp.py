"""Oracle of the learned Davidson guess network (test infrastructure only).

The paper has no learned component; the network is the library's extension
for the Davidson start. This module restates, in plain NumPy (FP64), what the
library's kernels compute, so that the GPU forward pass, gradients, Adam steps
and features can be compared element by element:

  * forward: y = W3^T relu(W2^T relu(W1^T x + b1) + b2) + b3 per row (weights
    stored [in x out], row-major, input index first);
  * loss = sum_i sum_o w_io (y_io - t_io)^2 / n and its gradient by the chain
    rule, written out layer by layer;
  * one Adam step (beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected);
  * the eight per-amplitude features of an EOM operator space.

Pinned in tests/test_oracle_pins.py by central finite differences of the loss
(gradient), by the closed forms of a network with zero weights, by the first
Adam step's closed form, and by Slater-rule determinant energies (features).
"""
from __future__ import annotations

import itertools

import numpy as np

NIN, NOUT = 8, 2


def unpack(params, width, nin=NIN, nout=NOUT):
    """Split the flat parameter vector into (W1, b1, W2, b2, W3, b3)."""
    p = np.asarray(params, dtype=np.float64)
    shapes = [(nin, width), (width,), (width, width), (width,), (width, nout), (nout,)]
    out, off = [], 0
    for sh in shapes:
        size = int(np.prod(sh))
        out.append(p[off:off + size].reshape(sh))
        off += size
    if off != p.size:
        raise ValueError("parameter vector length %d does not match width %d" % (p.size, width))
    return out


def pack(layers):
    """Concatenated parameter vector of the weight and bias arrays."""
    return np.concatenate([np.ravel(x) for x in layers])


def forward(params, x, width):
    """Returns y and the intermediates (z1, a1, z2, a2)."""
    w1, b1, w2, b2, w3, b3 = unpack(params, width)
    x = np.asarray(x, dtype=np.float64)
    z1 = x @ w1 + b1
    a1 = np.maximum(z1, 0.0)
    z2 = a1 @ w2 + b2
    a2 = np.maximum(z2, 0.0)
    y = a2 @ w3 + b3
    return y, (z1, a1, z2, a2)


def loss_grad(params, x, t, w, width):
    """Weighted mean-squared error and its gradient (flat, parameter layout)."""
    x = np.asarray(x, dtype=np.float64)
    n = x.shape[0]
    w1, b1, w2, b2, w3, b3 = unpack(params, width)
    y, (z1, a1, z2, a2) = forward(params, x, width)
    d = y - t
    loss = float(np.sum(w * d * d) / n)
    dy = 2.0 * w * d / n
    gw3 = a2.T @ dy
    gb3 = dy.sum(axis=0)
    dz2 = (dy @ w3.T) * (z2 > 0)
    gw2 = a1.T @ dz2
    gb2 = dz2.sum(axis=0)
    dz1 = (dz2 @ w2.T) * (z1 > 0)
    gw1 = x.T @ dz1
    gb1 = dz1.sum(axis=0)
    return loss, pack([gw1, gb1, gw2, gb2, gw3, gb3])


def adam_step(params, grad, m, v, step, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One bias-corrected Adam update; returns (params, m, v)."""
    m = b1 * m + (1.0 - b1) * grad
    v = b2 * v + (1.0 - b2) * grad * grad
    mhat = m / (1.0 - b1 ** step)
    vhat = v / (1.0 - b2 ** step)
    return params - lr * mhat / (np.sqrt(vhat) + eps), m, v


def eom_features(spaces, variant_id, fdiag, g, o, v, virt_occ=None):
    """Features of every packed element, components in order, tuples in
    lexicographic order (holes, then particles): orbital-energy difference D;
    spin-averaged two-body (Epstein-Nesbet) shift of the element's
    determinant: over hole pairs and particle pairs +w, over hole-particle
    pairs -w, w = <pq||pq> averaged over the spin of q (J_PP within one
    spatial orbital, J_PQ - K_PQ/2 otherwise); highest hole and lowest
    particle energy; mean particle energy; sum of log10 natural occupations
    of the particles' virtuals (0 without them); component index; variant.
    g: antisymmetrised <pq||rs> (alpha even), occupied first."""
    rows = []
    for comp, (nh, np_) in enumerate(spaces):
        for hs in itertools.combinations(range(o), nh):
            for ps in itertools.combinations(range(v), np_):
                eh = [fdiag[i] for i in hs]
                ep = [fdiag[o + a] for a in ps]
                orbs = list(hs) + [o + a for a in ps]
                en = 0.0
                for x in range(len(orbs)):
                    for y in range(x + 1, len(orbs)):
                        p, q = orbs[x], orbs[y]
                        w = g[p, q, p, q]
                        if p // 2 != q // 2:
                            w = 0.5 * (w + g[p, q ^ 1, p, q ^ 1])
                        same = (x < nh) == (y < nh)
                        en += (1 if same else -1) * w
                occ = 0.0
                if virt_occ is not None:
                    occ = sum(np.log10(max(virt_occ[a // 2], 1e-12)) for a in ps)
                rows.append([sum(ep) - sum(eh), en,
                             max(eh) if nh else 0.0,
                             min(ep) if np_ else 0.0,
                             sum(ep) / np_ if np_ else 0.0,
                             occ, comp, variant_id])
    return np.array(rows, dtype=np.float64)
