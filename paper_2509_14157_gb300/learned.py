"""Training data and training of the learned Davidson guess.

The network (fnocc_mlp_*) maps the eight features of an element mu of a
variant's packed operator space to two targets, both produced by the method
itself on small systems:

  0. importance: log10(1e-10 + max_r R_r[mu]^2) over the converged lowest
     roots R_r (unit norm) of a plain Davidson solve;
  1. preconditioner correction: H-bar_mumu - D_mu, the exact diagonal (one
     sigma product per element, fnocc_eom_diagonal) minus the orbital-energy
     difference D_mu (feature 0); on larger training sets only at a sample
     of each space's elements (fnocc_eom_diagonal_at), the others carrying
     weight 0 for this target.

Every number here comes from the library's CUDA path (solves, features,
diagonals, training kernels); this module only assembles arrays. Elements
outside the variant's spin sector (exact diagonal 0) get weight 0.
"""
from __future__ import annotations

import numpy as np

from . import Context, FnoccError, Mlp, VARIANTS


def sample_elements(r2, count, rng):
    """Packed indices of the elements whose exact diagonal is taken when
    the preconditioner target is sampled: count distinct elements of the
    spin sector (the converged roots vanish outside it), half of them the
    most important ones (largest r2), the rest uniform over the sector."""
    inside = np.flatnonzero(r2 > 0)
    if inside.size <= count:
        return inside
    top = inside[np.argsort(-r2[inside], kind="stable")[:count // 2]]
    rest = np.setdiff1d(inside, top)
    return np.sort(np.concatenate([top, rng.choice(rest, count - top.size, replace=False)]))


def system_samples(ctx, variant, nroots, diag_samples=None, rng=None):
    """(features, targets, weights) of one system whose ground state is
    solved in ctx; runs a plain Davidson solve and takes the exact diagonal
    of every sector element, or with diag_samples of that many sampled ones
    (sample_elements; the correction target of the others gets weight 0)."""
    res = ctx.eom_solve(variant, nroots, guess="koopmans")
    if not res["converged"]:
        return None
    feats = ctx.eom_features(variant)
    dim = feats.shape[0]
    r2 = np.zeros(dim)
    for root in range(nroots):
        vec = np.concatenate([ctx.get_block(("r", k), root) for k in (1, 2, 3)])
        nrm = np.linalg.norm(vec)
        if nrm > 0:
            r2 = np.maximum(r2, (vec / nrm) ** 2)
    weight = np.zeros((dim, 2))
    if diag_samples is None:
        diag = ctx.eom_diagonal(variant)
        weight[diag != 0.0] = 1.0
    else:
        pick = sample_elements(r2, diag_samples, rng if rng is not None else np.random.default_rng(0))
        diag = feats[:, 0].astype(np.float64).copy()  # correction 0 where not sampled (weight 0)
        diag[pick] = ctx.eom_diagonal(variant, pick)
        weight[r2 > 0, 0] = 1.0
        weight[pick, 1] = 1.0
    target = np.stack([np.log10(1e-10 + r2), diag - feats[:, 0]], axis=1)
    return feats, target.astype(np.float32), weight.astype(np.float32)


def training_set(systems, variants, nroots, device=0, diag_samples=None, max_samples=None, seed=0, workers=1):
    """Samples of every (system, variant). systems: dicts with h, eri, nocc
    and threshold or nkeep. Returns (X, T, W, info); systems whose RHF or
    CCSDT fails are skipped. Systems are taken in order of shape and split
    into `workers` contiguous runs, each on its own host thread and context
    (systems of the same shape keep its contraction plans; a context is
    rebuilt after a failure); the result does not depend on the split.
    diag_samples: sampled preconditioner targets (system_samples, element
    choice seeded per system); max_samples: at most that many samples,
    drawn uniformly (seeded) from those with a nonzero weight."""
    import threading

    order = sorted(range(len(systems)), key=lambda i: (systems[i]["h"].shape[0], systems[i]["nocc"],
                                                       systems[i].get("nkeep", 0), i))
    found = [None] * len(systems)
    errors = []

    def run(chunk):
        ctx = None
        try:
            for i in chunk:
                sy = systems[i]
                if ctx is None:
                    ctx = Context(device)
                try:
                    ctx.fno_truncate(sy["h"], sy["eri"], sy["nocc"], sy.get("threshold", 0.0),
                                     nkeep=sy.get("nkeep", 0))
                    if not ctx.ccsdt_solve()["converged"]:
                        continue
                    rng = np.random.default_rng([seed, i])
                    part = []
                    for var in variants:
                        s = system_samples(ctx, VARIANTS.get(var, var), nroots, diag_samples, rng)
                        if s is not None:
                            keep = s[2].sum(axis=1) > 0
                            part.append((s[0][keep], s[1][keep], s[2][keep], (sy.get("name", ""), var,
                                                                             int(keep.sum()))))
                    found[i] = part
                except FnoccError:
                    ctx.close()
                    ctx = None
        except Exception as e:  # reported after the join
            errors.append(e)
        finally:
            if ctx is not None:
                ctx.close()

    workers = max(1, min(int(workers), len(order)))
    step = (len(order) + workers - 1) // workers
    threads = [threading.Thread(target=run, args=(order[k:k + step],)) for k in range(0, len(order), step)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    if errors:
        raise errors[0]
    parts = [p for i in order if found[i] for p in found[i]]
    X = np.concatenate([p[0] for p in parts])
    T = np.concatenate([p[1] for p in parts])
    W = np.concatenate([p[2] for p in parts])
    info = [p[3] for p in parts]
    if max_samples is not None and X.shape[0] > max_samples:
        pick = np.sort(np.random.default_rng(seed).choice(X.shape[0], max_samples, replace=False))
        X, T, W = X[pick], T[pick], W[pick]
    return X, T, W, info


def train_guess_model(X, T, W, width=256, epochs=30, batch=4096, lr=1e-3, seed=0, device=0):
    """A new network trained on (X, T, W); returns (network, loss history)."""
    net = Mlp(device, width, seed)
    keep = W.sum(axis=1) > 0
    if not keep.all():
        X, T, W = X[keep], T[keep], W[keep]
    hist = net.train(X, T, W, epochs=epochs, batch=batch, lr=lr, seed=seed)
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
