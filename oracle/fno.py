"""Oracle: RHF reference, spin-orbital integrals, MP2 natural orbitals and the
frozen-natural-orbital truncation (Sec. 1.2 "FNO approximation", Eq. 8-10).

Conventions
  * spatial chemists' integrals (pq|rs), orthonormal basis (S = I);
  * spin orbital P = 2*p + s (alpha s=0, beta s=1), occupied first;
  * <PQ||RS> = <PQ|RS> - <PQ|SR>, with <PQ|RS> = (pr|qs) delta_sP,sR delta_sQ,sS;
  * natural occupations are the alpha-block eigenvalues of Eq. 10 as printed
    (per spin orbital);
  * orbital phase: the largest-magnitude coefficient of every orbital is made
    positive (ties broken by the lowest index).

Parity: RHF is pinned by stationarity (Brillouin) and by the Fock-space energy
of its determinant; MP2 and D_vv by second-order perturbation theory written
out in determinant space (tests/test_oracle_pins.py); truncation by its
threshold-0 and nkeep special cases.
"""
from __future__ import annotations

import numpy as np


def fix_phase(c):
    """Make the largest-|c| element of every column positive."""
    c = np.array(c, dtype=np.float64, copy=True)
    if c.size == 0:
        return c
    idx = np.argmax(np.abs(c), axis=0)
    s = np.sign(c[idx, np.arange(c.shape[1])])
    s[s == 0] = 1.0
    return c * s[None, :]


def rhf(h, eri, nocc, max_iter=200, e_tol=1e-12, comm_tol=1e-10, diis_size=8):
    """Closed-shell Roothaan-Hall SCF with DIIS (the Hartree-Fock reference of
    Sec. 1.2). Returns dict(e, c, eps, f, d, iters)."""
    n = h.shape[0]
    eps, c = np.linalg.eigh(h)
    d = c[:, :nocc] @ c[:, :nocc].T
    fs, errs = [], []
    e_old = 0.0
    for it in range(1, max_iter + 1):
        j = np.einsum("pqrs,rs->pq", eri, d)
        k = np.einsum("prqs,rs->pq", eri, d)
        f = h + 2.0 * j - k
        e = float(np.sum(d * (h + f)))
        err = f @ d - d @ f
        fs.append(f)
        errs.append(err)
        if len(fs) > diis_size:
            fs.pop(0)
            errs.pop(0)
        if abs(e - e_old) < e_tol and np.max(np.abs(err)) < comm_tol:
            break
        e_old = e
        m = len(fs)
        if m >= 2:
            b = np.zeros((m + 1, m + 1))
            for a in range(m):
                for bb in range(m):
                    b[a, bb] = np.sum(errs[a] * errs[bb])
            b[m, :m] = b[:m, m] = -1.0
            rhs = np.zeros(m + 1)
            rhs[m] = -1.0
            coef = np.linalg.solve(b, rhs)[:m]
            f_use = sum(cf * ff for cf, ff in zip(coef, fs))
        else:
            f_use = f
        eps, c = np.linalg.eigh(f_use)
        d = c[:, :nocc] @ c[:, :nocc].T
    else:
        raise RuntimeError("RHF did not converge")
    eps, c = np.linalg.eigh(f)
    c = fix_phase(c)
    d = c[:, :nocc] @ c[:, :nocc].T
    return dict(e=e, c=c, eps=eps, f=f, d=d, iters=it)


def spin_orbital_integrals(eri_mo):
    """<PQ||RS> over spin orbitals from spatial MO integrals (pq|rs)."""
    n = eri_mo.shape[0]
    ns = 2 * n
    phys = eri_mo.transpose(0, 2, 1, 3)  # <pq|rs> = (pr|qs)
    g = np.zeros((ns, ns, ns, ns))
    for s1 in range(2):
        for s2 in range(2):
            g[s1::2, s2::2, s1::2, s2::2] = phys
    return g - g.transpose(0, 1, 3, 2)


def spin_orbital_one_body(h_mo):
    """Spatial one-body matrix -> spin orbitals (alpha even, beta odd; Sec. 1.2)."""
    n = h_mo.shape[0]
    out = np.zeros((2 * n, 2 * n))
    out[0::2, 0::2] = h_mo
    out[1::2, 1::2] = h_mo
    return out


def transform_eri(eri, c1, c2, c3, c4):
    """(pq|rs) transformed index by index with the coefficient matrices c1..c4 (Sec. 1.2)."""
    return np.einsum("pqrs,pa,qb,rc,sd->abcd", eri, c1, c2, c3, c4, optimize=True)


def fock_from_bare(hso, gso, o):
    """f_pq = h_pq + sum_i <pi||qi> (normal ordering w.r.t. the first o spin
    orbitals) and the reference energy."""
    f = hso + np.einsum("piqi->pq", gso[:, :o, :, :o])
    e_ref = float(np.trace(hso[:o, :o]) + 0.5 * np.einsum("ijij->", gso[:o, :o, :o, :o]))
    return f, e_ref


def mp2_amplitudes(f, g, o):
    """Eq. 8-9: t_ij^ab = <ab||ij> / (f_ii + f_jj - f_aa - f_bb)."""
    fo = np.diag(f)[:o]
    fv = np.diag(f)[o:]
    denom = (fo[:, None, None, None] + fo[None, :, None, None]
             - fv[None, None, :, None] - fv[None, None, None, :])
    abij = g[o:, o:, :o, :o]
    return abij.transpose(2, 3, 0, 1) / denom


def mp2_energy(g, t2, o):
    """E_MP2 = 1/4 sum <ij||ab> t_ij^ab."""
    return 0.25 * float(np.sum(g[:o, :o, o:, o:] * t2))


def mp2_vv_density(f, g, o):
    """Eq. 10 as printed: D_ab = 1/2 sum_cij <cb||ij><ij||ca> / (e_ij^cb e_ij^ca)."""
    fo = np.diag(f)[:o]
    fv = np.diag(f)[o:]
    eps_ijcd = (fo[:, None, None, None] + fo[None, :, None, None]
                - fv[None, None, :, None] - fv[None, None, None, :])  # [i,j,c,d]
    cbij = g[o:, o:, :o, :o]              # <cb||ij> as [c,b,i,j]
    ijca = g[:o, :o, o:, o:]              # <ij||ca> as [i,j,c,a]
    x = cbij.transpose(2, 3, 0, 1) / eps_ijcd   # [i,j,c,b]
    y = ijca / eps_ijcd                         # [i,j,c,a]
    return 0.5 * np.einsum("ijcb,ijca->ab", x, y)


def choose_kept(occ_sorted, threshold, criterion="abs", nkeep=0, degen_rel=1e-10):
    """Number of natural virtuals kept (Sec. 1.2 truncation; the paper defines
    neither of its two schemes, so both readings are offered below).

    occ_sorted: occupations in descending order.
    criterion 'abs': keep n_a >= threshold; 'occt': smallest prefix whose
    cumulative occupation fraction reaches `threshold`. nkeep > 0 overrides.
    Clusters of occupations equal within degen_rel * n_max are kept or
    dropped whole (the whole cluster is kept if its first member is)."""
    m = len(occ_sorted)
    if nkeep > 0:
        k = min(nkeep, m)
    elif criterion == "abs":
        k = int(np.sum(occ_sorted >= threshold))
    elif criterion == "occt":
        tot = float(np.sum(occ_sorted))
        if tot <= 0.0:
            k = m
        else:
            cum = np.cumsum(occ_sorted) / tot
            k = int(np.searchsorted(cum, threshold - 1e-15) + 1)
            k = min(k, m)
    else:
        raise ValueError(criterion)
    if 0 < k < m and nkeep <= 0:
        tol = degen_rel * max(abs(occ_sorted[0]), 1e-300)
        while k < m and abs(occ_sorted[k] - occ_sorted[k - 1]) <= tol:
            k += 1
    return k


def fno_truncate(h, eri, nocc, threshold, criterion="abs", nkeep=0):
    """RHF -> MP2 -> D_vv -> NOs -> truncation -> semicanonical active space.

    Returns a dict with the reference energy, E_MP2, the sorted occupations,
    the kept count and fraction, and the active spin-orbital Hamiltonian:
    f (normal-ordered Fock), g = <pq||rs>, o and v (spin-orbital counts)."""
    n = h.shape[0]
    scf = rhf(h, eri, nocc)
    c = scf["c"]
    e_rhf = scf["e"]
    # full canonical spin-orbital quantities for MP2 (Eq. 8-10)
    eri_mo = transform_eri(eri, c, c, c, c)
    g_full = spin_orbital_integrals(eri_mo)
    hso = spin_orbital_one_body(c.T @ h @ c)
    o = 2 * nocc
    f_full, _ = fock_from_bare(hso, g_full, o)
    t2 = mp2_amplitudes(f_full, g_full, o)
    e_mp2 = mp2_energy(g_full, t2, o)
    d_so = mp2_vv_density(f_full, g_full, o)
    d_sp = d_so[0::2, 0::2]
    occ, u = np.linalg.eigh(d_sp)
    order = np.argsort(-occ, kind="stable")
    occ = occ[order]
    u = u[:, order]
    k = choose_kept(occ, threshold, criterion, nkeep)
    kept_fraction = float(np.sum(occ[:k]) / np.sum(occ)) if np.sum(occ) > 0 else 1.0
    # semicanonicalise the kept NOs: diagonalise F_vv inside them
    eps_v = scf["eps"][nocc:]
    uk = u[:, :k]
    fvv = uk.T @ np.diag(eps_v) @ uk
    ev, w = np.linalg.eigh(fvv)
    c_vir = fix_phase(c[:, nocc:] @ uk @ w)
    c_act = np.concatenate([c[:, :nocc], c_vir], axis=1)
    act = active_hamiltonian(h, eri, c_act, nocc)
    # natural occupation carried by each semicanonical virtual (diagonal of
    # the kept NO density in the semicanonical basis): a feature of the
    # learned Davidson guess, not a quantity of the paper's method
    virt_occ = (w ** 2).T @ occ[:k] if k > 0 else np.zeros(0)
    act.update(e_rhf=e_rhf, e_mp2=e_mp2, occ=occ, nkept=k,
               kept_fraction=kept_fraction, c_act=c_act, scf_iters=scf["iters"], virt_occ=virt_occ)
    return act


def active_hamiltonian(h, eri, c_act, nocc):
    """Spin-orbital f and <pq||rs> over the active orbitals (columns of c_act,
    the first nocc doubly occupied)."""
    eri_mo = transform_eri(eri, c_act, c_act, c_act, c_act)
    g = spin_orbital_integrals(eri_mo)
    hso = spin_orbital_one_body(c_act.T @ h @ c_act)
    o = 2 * nocc
    f, e_ref = fock_from_bare(hso, g, o)
    return dict(f=f, g=g, hso=hso, e_ref=e_ref, o=o, v=g.shape[0] - o)


def mo_hamiltonian(h_mo, eri_mo, nocc):
    """Spin-orbital f, <pq||rs> directly from spatial MO-basis h and (pq|rs)."""
    g = spin_orbital_integrals(eri_mo)
    hso = spin_orbital_one_body(h_mo)
    o = 2 * nocc
    f, e_ref = fock_from_bare(hso, g, o)
    return dict(f=f, g=g, hso=hso, e_ref=e_ref, o=o, v=g.shape[0] - o)
