"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module draws random numbers and arranges them into arrays. It holds none
of the method's arithmetic: no integral transformation, no antisymmetrisation,
no amplitude equation. Both the CPU oracle and the CUDA library consume what is
generated here, each with its own code.

Hamiltonian recipe (closed-shell, orthonormal basis, zero nuclear repulsion):
  * occupied orbital energies: sorted U(-1.5, -0.5), nocc of them;
  * virtual orbital energies: sorted U(0.2, 3.0), n - nocc of them;
  * one-electron operator h = diag(energies) + symmetric off-diagonal part whose
    upper triangle is N(0, 0.05^2);
  * a symmetric Gaussian factor G[Q, p, q] (upper triangle incl. diagonal
    N(0, 1), mirrored) of rank R = 30, damped as B = sigma_B * G * exp(-(p+q)/8);
  * two-electron integrals in chemists' notation (pq|rs) = sum_Q B_Qpq B_Qrs,
    which carry the full 8-fold permutational symmetry.
The draws are made in exactly that order from numpy.random.default_rng(seed).
"""
from __future__ import annotations

import itertools
import numpy as np

SIGMA_B = 0.2
RANK = 30


def hamiltonian(nelec: int, n: int, seed: int = 0, sigma_b: float = SIGMA_B,
                rank: int = RANK):
    """Return (h, eri) for a seeded closed-shell system of `nelec` electrons in
    `n` spatial orbitals; h is n x n, eri is n^4 in chemists' order (pq|rs)."""
    if nelec % 2:
        raise ValueError("closed-shell generator needs an even electron count")
    nocc = nelec // 2
    if not 0 < nocc < n:
        raise ValueError("need 0 < nocc < n")
    rng = np.random.default_rng(seed)
    e_occ = np.sort(rng.uniform(-1.5, -0.5, nocc))
    e_vir = np.sort(rng.uniform(0.2, 3.0, n - nocc))
    off = np.triu(rng.normal(0.0, 0.05, (n, n)), 1)
    h = np.diag(np.concatenate([e_occ, e_vir])) + off + off.T
    g = rng.normal(0.0, 1.0, (rank, n, n))
    g = np.triu(g) + np.transpose(np.triu(g, 1), (0, 2, 1))
    pq = np.arange(n)[:, None] + np.arange(n)[None, :]
    b = sigma_b * g * np.exp(-pq / 8.0)[None]
    eri = np.einsum("Qpq,Qrs->pqrs", b, b, optimize=True)
    return h, eri


def random_orthogonal(n: int, seed: int):
    """A seeded Haar-like orthogonal n x n matrix (QR of a Gaussian matrix)."""
    rng = np.random.default_rng(seed)
    q, r = np.linalg.qr(rng.normal(size=(n, n)))
    return q * np.sign(np.diag(r))[None, :]


def random_symmetric_mo_hamiltonian(n: int, seed: int, scale_h: float = 0.3,
                                    scale_eri: float = 0.05):
    """A seeded random spatial Hamiltonian in an orthonormal MO basis, used to
    feed contraction tests with general (non-canonical) operators.

    h has a diagonal spread like orbital energies plus symmetric noise; eri is
    (pq|rs) = sum_Q B_Qpq B_Qrs with a random symmetric factor (8-fold
    symmetric, positive semidefinite as a pq,rs matrix)."""
    rng = np.random.default_rng(seed)
    diag = np.sort(rng.uniform(-1.5, 2.5, n))
    off = np.triu(rng.normal(0.0, scale_h, (n, n)), 1)
    h = np.diag(diag) + off + off.T
    g = rng.normal(0.0, 1.0, (8, n, n))
    g = np.triu(g) + np.transpose(np.triu(g, 1), (0, 2, 1))
    eri = scale_eri * np.einsum("Qpq,Qrs->pqrs", g, g)
    return h, eri


def strictly_increasing(n: int, k: int):
    """All strictly increasing k-tuples over range(n) in lexicographic order
    (the packed ordering used at the library boundary)."""
    return list(itertools.combinations(range(n), k))


def packed_ms_mask(nh: int, np_: int, o: int, v: int, ms2: int):
    """Boolean mask over the packed (holes i1<..<i_nh) x (particles a1<..<a_np)
    list, True where 2*M_s of the operator a1^+..a_np^+ i_nh..i1 equals ms2.

    Spin orbitals alternate alpha (even) / beta (odd); occupied first. A
    particle of spin s adds s, a hole of spin s removes s (alpha=+1, beta=-1)."""
    def spin2(p):
        return 1 if p % 2 == 0 else -1
    hs = strictly_increasing(o, nh)
    ps = strictly_increasing(v, np_)
    hsum = np.array([sum(spin2(i) for i in t) for t in hs], dtype=int)
    psum = np.array([sum(spin2(a) for a in t) for t in ps], dtype=int)
    return (psum[None, :] - hsum[:, None] == ms2).reshape(-1)


def random_packed(count: int, seed: int, scale: float = 0.05):
    """`count` seeded N(0, scale^2) numbers, to be used as packed amplitudes."""
    return np.random.default_rng(seed).normal(0.0, scale, count)
