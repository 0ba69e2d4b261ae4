"""Training data and training of the learned Davidson guess.

The network (fnocc_mlp_*) maps the eight features of an element mu of a
variant's packed operator space to two targets, both produced by the method
itself on small systems:

  0. importance: log10(1e-10 + max_r R_r[mu]^2) over the converged lowest
     roots R_r (unit norm) of a plain Davidson solve;
  1. preconditioner correction: H-bar_mumu - D_mu, the exact diagonal (one
     sigma product per element, fnocc_eom_diagonal) minus the orbital-energy
     difference D_mu (feature 0).

Every number here comes from the library's CUDA path (solves, features,
diagonals, training kernels); this module only assembles arrays. Elements
outside the variant's spin sector (exact diagonal 0) get weight 0.
"""
from __future__ import annotations

import numpy as np

from . import Context, FnoccError, Mlp, VARIANTS


def system_samples(ctx, variant, nroots):
    """(features, targets, weights) of one system whose ground state is
    solved in ctx; runs a plain Davidson solve and the exact diagonal."""
    res = ctx.eom_solve(variant, nroots, guess="koopmans")
    if not res["converged"]:
        return None
    feats = ctx.eom_features(variant)
    diag = ctx.eom_diagonal(variant)
    dim = feats.shape[0]
    r2 = np.zeros(dim)
    for root in range(nroots):
        vec = np.concatenate([ctx.get_block(("r", k), root) for k in (1, 2, 3)])
        nrm = np.linalg.norm(vec)
        if nrm > 0:
            r2 = np.maximum(r2, (vec / nrm) ** 2)
    target = np.stack([np.log10(1e-10 + r2), diag - feats[:, 0]], axis=1)
    weight = np.zeros((dim, 2))
    weight[diag != 0.0] = 1.0
    return feats, target.astype(np.float32), weight.astype(np.float32)


def training_set(systems, variants, nroots, device=0):
    """Samples of every (system, variant). systems: dicts with h, eri, nocc
    and threshold or nkeep. Returns (X, T, W, info); systems whose RHF or
    CCSDT fails are skipped."""
    xs, ts, ws, info = [], [], [], []
    for sy in systems:
        ctx = Context(device)
        try:
            ctx.fno_truncate(sy["h"], sy["eri"], sy["nocc"], sy.get("threshold", 0.0), nkeep=sy.get("nkeep", 0))
            if not ctx.ccsdt_solve()["converged"]:
                continue
            for var in variants:
                s = system_samples(ctx, VARIANTS.get(var, var), nroots)
                if s is not None:
                    xs.append(s[0])
                    ts.append(s[1])
                    ws.append(s[2])
                    info.append((sy.get("name", ""), var, s[0].shape[0]))
        except FnoccError:
            continue
        finally:
            ctx.close()
    return np.concatenate(xs), np.concatenate(ts), np.concatenate(ws), info


def train_guess_model(X, T, W, width=256, epochs=30, batch=4096, lr=1e-3, seed=0, device=0):
    """A new network trained on (X, T, W); returns (network, loss history)."""
    net = Mlp(device, width, seed)
    keep = W.sum(axis=1) > 0
    hist = net.train(X[keep], T[keep], W[keep], epochs=epochs, batch=batch, lr=lr, seed=seed)
    return net, hist


def seeded_training_systems(count=24, first_seed=100, electrons=(6, 8)):
    """The training workload: small seeded synthetic closed-shell systems
    cycling through the given electron counts (6 and 8 by default: 10-12
    orbitals; 10 electrons: 12-14 orbitals), 4-6 kept natural virtuals (the
    exact-diagonal target costs one product per element, which bounds the
    size)."""
    import synth
    out = []
    for s in range(count):
        ne = electrons[s % len(electrons)]
        n = 10 + (s % 3) + max(0, ne - 8)
        h, eri = synth.hamiltonian(ne, n, seed=first_seed + s)
        out.append(dict(h=h, eri=eri, nocc=ne // 2, nkeep=4 + (s % 3), name="train%d" % s))
    return out
