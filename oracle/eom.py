"""Oracle: IP / EA / DIP / DEA EOM-CCSDT (Eq. 1-4) and the Davidson solver.

Operator spaces (Eq. 3-4 as printed would drop 1p / 2p for attachment and
4h2p for DIP; the reading here: every variant has three components, removal
uses n = m..m+2 holes, attachment n = 0..2):
    IP  1h, 2h1p, 3h2p        EA  1p, 1h2p, 2h3p
    DIP 2h, 3h1p, 4h2p        DEA 2p, 1h3p, 2h4p
and the excitation-energy variant the method builds on (Sec. 1):
    EE  1h1p, 2h2p, 3h3p (M_s unchanged)
sigma = <mu| (H-bar R)_c |Phi_0> from the Wick term lists (oracle/wick.py);
the eigenvalue omega is the energy relative to the CC ground state, so the
state's total energy is E_CC + omega.

Spin sector (the paper names none): 2*M_s change of +1 for IP (a beta
electron is removed) and EA (an alpha electron is added), 0 for DIP, DEA and
EE. The roots are the lowest Re(omega) in that sector.

Davidson (the paper names no eigensolver; this follows the standard
non-symmetric Davidson method): orthonormal subspace V, projected matrix
G = V^T sigma(V), Ritz pairs of G ordered by real part, residual
r = sigma(x) - theta x, diagonal preconditioner (theta - D)^-1 with D built
from diag(f), Gram-Schmidt (twice), and a thick restart from the 2*nroots
lowest Ritz vectors when the subspace exceeds max_sub. Guesses are 2*nroots unit vectors on the lowest
diagonal elements (of the first component for the Koopmans guess, of the
whole space for the diagonal guess); with only nroots guesses a low root of
weak overlap can be missed.

Parity: sigma pinned to the Fock-space definition for all four variants on
random T and R; eigenvalues pinned to FCI where the operator space spans the
whole (N +- m) sector; Davidson pinned to dense diagonalisation of the
explicitly built sigma matrix.
"""
from __future__ import annotations

import itertools

import numpy as np

from . import packing, wick

SECTOR_MS2 = {"ip": 1, "ea": 1, "dip": 0, "dea": 0, "ee": 0}


def comps(variant):
    """(holes, particles) of R1, R2, R3 of the variant (Eq. 3-4 as read here)."""
    return wick.EOM_SPACES[variant]


def sizes(variant, o, v):
    """Packed sizes of the three components."""
    return [packing.packed_size(nh, np_, o, v) for nh, np_ in comps(variant)]


def ms_mask(variant, o, v):
    """Packed-vector mask of the target spin sector (alpha = even spin orbital)."""
    out = []
    for nh, np_ in comps(variant):
        hs = list(itertools.combinations(range(o), nh))
        ps = list(itertools.combinations(range(v), np_))
        sh = np.array([sum(1 if i % 2 == 0 else -1 for i in t) for t in hs])
        sp_ = np.array([sum(1 if a % 2 == 0 else -1 for a in t) for t in ps])
        out.append((sp_[None, :] - sh[:, None] == SECTOR_MS2[variant]).reshape(-1))
    return np.concatenate(out)


def split(variant, o, v, vec):
    """Packed EOM vector -> dense antisymmetric components."""
    s = sizes(variant, o, v)
    parts = np.split(vec, np.cumsum(s)[:-1])
    return [packing.unpack(p, nh, np_, o, v) for p, (nh, np_) in zip(parts, comps(variant))]


def sigma_dense(variant, f, g, o, v, t1, t2, t3, rs):
    """sigma_out = sum_in <mu_out| (H-bar R_in)_c |0> (Eq. 1-4) on dense components."""
    amps = {"t1": t1, "t2": t2, "t3": t3, "r1": rs[0], "r2": rs[1], "r3": rs[2]}
    out = []
    for oc, (nh, np_) in enumerate(comps(variant)):
        acc = np.zeros((o,) * nh + (v,) * np_)
        for ic in range(3):
            acc += wick.evaluate(wick.eom_terms(variant, oc, ic), nh, np_, f, g, amps, o, v)
        out.append(acc)
    return out


def sigma_packed(variant, f, g, o, v, t1, t2, t3, vec):
    """sigma of a packed EOM vector, returned packed (Eq. 1-4)."""
    rs = split(variant, o, v, vec)
    out = sigma_dense(variant, f, g, o, v, t1, t2, t3, rs)
    return np.concatenate([packing.pack(x, nh, np_, o, v) for x, (nh, np_) in zip(out, comps(variant))])


def diagonal(variant, f, o, v):
    """Orbital-energy estimate of diag(H-bar): sum f_aa - sum f_ii per element."""
    fo = np.diag(f)[:o]
    fv = np.diag(f)[o:]
    out = []
    for nh, np_ in comps(variant):
        hs = list(itertools.combinations(range(o), nh))
        ps = list(itertools.combinations(range(v), np_))
        eh = np.array([sum(fo[i] for i in t) for t in hs])
        ep = np.array([sum(fv[a] for a in t) for t in ps])
        out.append((ep[None, :] - eh[:, None]).reshape(-1))
    return np.concatenate(out)


def _orthonormalise(vec, basis, tol=1e-10):
    for _ in range(2):
        for b in basis:
            vec = vec - (b @ vec) * b
    nrm = np.linalg.norm(vec)
    if nrm < tol:
        return None
    return vec / nrm


def davidson(apply, diag, mask, nroots, tol_res=1e-8, tol_e=1e-10, max_sub=None,
             maxiter=200, nguess=None, guess_mask=None, principal=None, min_weight=1e-6):
    """Lowest-Re roots of a non-symmetric operator restricted to `mask`.
    Guess unit vectors sit on the lowest `diag` entries inside guess_mask.
    When the subspace would exceed max_sub it is restarted from the 2*nroots
    lowest Ritz vectors, whose products follow as the same combinations.

    principal: length of the leading (principal, 1h/1p/2h/2p) block. Roots
    are counted only among Ritz vectors whose weight there is at least
    min_weight: states of other spin multiplicities (e.g. the quintet 3h1p
    states of DIP) have none, and a Davidson started on principal
    determinants reaches them only through rounding. Where the sector holds
    fewer principal states than nroots, the lowest others fill up."""
    n = len(diag)
    allowed = np.where(mask)[0]
    if nguess is None:
        nguess = 2 * nroots
    nguess = min(nguess, len(allowed))
    nroots = min(nroots, len(allowed))
    if max_sub is None:
        max_sub = max(6 * nroots, nguess + 3 * nroots)
    max_sub = max(max_sub, max(nguess, 2 * nroots) + nroots)
    pref = allowed if guess_mask is None else np.where(mask & guess_mask)[0]
    rest = np.setdiff1d(allowed, pref)
    order = pref[np.argsort(diag[pref], kind="stable")][:nguess]
    rest = rest[np.argsort(diag[rest], kind="stable")]
    basis, sig = [], []

    def add(vec, svec=None):
        vec = vec * mask
        if svec is not None:
            svec = svec * mask
        for _ in range(2):
            for b, sb in zip(basis, sig):
                c = b @ vec
                vec = vec - c * b
                if svec is not None:
                    svec = svec - c * sb
        nrm = np.linalg.norm(vec)
        if nrm < 1e-10:
            return
        basis.append(vec / nrm)
        sig.append(svec / nrm if svec is not None else apply(vec / nrm) * mask)

    def unit(k):
        e = np.zeros(n)
        e[k] = 1.0
        return e

    for k in order:
        add(unit(k))
    # fewer guess elements than nguess: Krylov vectors (products of the
    # basis), then the lowest-diagonal remaining elements
    src = 0
    while len(basis) < nguess and src < len(basis):
        add(sig[src])
        src += 1
    for k in rest:
        if len(basis) >= nguess:
            break
        add(unit(k))
    theta_old = None
    for it in range(1, maxiter + 1):
        vmat = np.array(basis)
        smat = np.array(sig)
        gmat = vmat @ smat.T
        w_all, y_all = np.linalg.eig(gmat)
        srt = np.argsort(w_all.real, kind="stable")
        if principal is not None:
            good, rest_idx = [], []
            for j in srt:
                yv = np.real(y_all[:, j])
                xv = vmat.T @ (yv / np.linalg.norm(yv))
                (good if xv[:principal] @ xv[:principal] >= min_weight else rest_idx).append(j)
            # fewer principal states than roots: the lowest others fill up
            chosen = good[:nroots] + rest_idx[:max(0, nroots - len(good))]
            chosen.sort(key=lambda j: w_all[j].real)
            srt = np.array(chosen + [j for j in good[nroots:]])
        w = w_all[srt][:nroots]
        yr = np.real(y_all[:, srt])
        theta = w.real
        xs, res, norms = [], [], []
        for r in range(nroots):
            yv = yr[:, r] / np.linalg.norm(yr[:, r])
            x = vmat.T @ yv
            rv = smat.T @ yv - theta[r] * x
            xs.append(x)
            res.append(rv)
            norms.append(np.linalg.norm(rv))
        # |d omega| against the nearest previous Ritz value (near-degenerate
        # roots may swap rank between iterations)
        done = [norms[r] < tol_res and theta_old is not None and np.min(np.abs(theta[r] - theta_old)) < tol_e
                for r in range(nroots)]
        if all(done):
            return dict(omega=theta, vectors=np.array(xs), iters=it, res=np.array(norms),
                        converged=True, imag=np.abs(w.imag))
        theta_old = theta.copy()
        new = []
        for r in range(nroots):
            if done[r]:
                continue
            den = theta[r] - diag
            den = np.where(np.abs(den) < 1e-8, 1e-8, den)
            new.append((res[r] / den) * mask)
        if len(basis) + len(new) > max_sub:
            nkeep = min(len(srt), 2 * nroots)
            keep = []
            for q in range(nkeep):
                yv = yr[:, q] / np.linalg.norm(yr[:, q])
                keep.append((vmat.T @ yv, smat.T @ yv))
            basis, sig = [], []
            for x, sx in keep:
                add(x, sx)
        for d in new:
            add(d)
    return dict(omega=theta, vectors=np.array(xs), iters=maxiter, res=np.array(norms),
                converged=False, imag=np.abs(w.imag))


def eom_ccsdt(variant, f, g, o, v, t1, t2, t3, nroots, tol_res=1e-8, tol_e=1e-10,
              max_sub=None, maxiter=200, nguess=None, guess="koopmans"):
    """Lowest nroots EOM-CCSDT excitation energies omega in the target sector.

    guess 'koopmans': unit vectors on the lowest diagonal elements of the
    first component (1h, 1p, 2h or 2p); 'diagonal': on the lowest diagonal
    elements of the whole operator space. Fewer elements than guesses: Krylov
    vectors, then the lowest-diagonal remaining elements (see davidson)."""
    mask = ms_mask(variant, o, v)
    diag = diagonal(variant, f, o, v)
    first = sizes(variant, o, v)[0]
    gmask = np.zeros_like(mask)
    if guess == "koopmans":
        gmask[:first] = True
    elif guess == "diagonal":
        gmask[:] = True
    else:
        raise ValueError(guess)

    def apply(x):
        return sigma_packed(variant, f, g, o, v, t1, t2, t3, x)

    return davidson(apply, diag, mask, nroots, tol_res, tol_e, max_sub, maxiter, nguess, gmask,
                    principal=first)


def sigma_matrix(variant, f, g, o, v, t1, t2, t3):
    """Explicit H-bar matrix in the target sector (for small pins)."""
    mask = ms_mask(variant, o, v)
    idx = np.where(mask)[0]
    n = len(mask)
    cols = []
    for k in idx:
        e = np.zeros(n)
        e[k] = 1.0
        cols.append(sigma_packed(variant, f, g, o, v, t1, t2, t3, e)[idx])
    return np.array(cols).T


def left_sigma_packed(variant, f, g, o, v, t1, t2, t3, lvec):
    """Left product lambda_nu = sum_mu L_mu <mu| (H-bar tau_nu)_c |0> (the row
    vector L times the product matrix), written out from its definition: one
    right product per element nu of the target sector, each dotted with L.
    O(dim) products: small systems only. Elements outside the sector are 0."""
    mask = ms_mask(variant, o, v)
    out = np.zeros(len(mask))
    e = np.zeros(len(mask))
    for k in np.where(mask)[0]:
        e[k] = 1.0
        out[k] = lvec[mask] @ sigma_packed(variant, f, g, o, v, t1, t2, t3, e)[mask]
        e[k] = 0.0
    return out
