"""Oracle — test infrastructure only.  Hamiltonian interpolation (HI) for
two-form sites, as plain FP64 numpy on top of the Ewald oracle.

Definitions followed (arxiv 2410.01754):

* Multilinear HI Hamiltonian, Eq. "rek_ham_lambda" generalised to M sites:
  H = sum over protonation states X of prod_s w_s(X_s) H_X, with
  w_s(A) = 1 - lambda_s, w_s(B) = lambda_s, and H_X the periodic Coulomb energy
  of the charges of state X (Eq. "nbody_periodic").
* Scaled charges, Eq. under "lambda_tilde": q~_i = qA_i + lambda_s (qB_i - qA_i)
  (for two forms lambda~ = (1 - lambda, lambda)); environment atoms keep q.
* HI minus QI, Eqs. "DeltaFQIHI" and "Udiff": with
  k_s = f sum_{i,j in s} D_i D_j A(x_i - x_j), D = qB - qA, the HI energy is
  E = E(q~) + sum_s 1/2 lambda_s (1 - lambda_s) k_s and
  dE/dlambda_s = sum_{i in s} D_i phi~_i + (1/2 - lambda_s) k_s.
  The periodic kernel A replaces 1/r (images included; A_ii = xi), which is the
  reading this package takes for the paper's periodic correction terms.
* Forces: F_i = -q~_i grad phi~_i - lambda_s (1 - lambda_s) f
  sum_{j in s, j != i} D_i D_j grad A(x_i - x_j).

``hi_bruteforce`` evaluates the first definition literally (2^S Ewald energies)
and is the check on the closed form.
"""
from __future__ import annotations

import itertools

import numpy as np

from . import F_COULOMB, ewald, ewald_energy, pair_A


def scaled_charges(qA, qB, site_of, lam):
    qA = np.asarray(qA, dtype=np.float64)
    qB = np.asarray(qB, dtype=np.float64)
    site_of = np.asarray(site_of)
    lam = np.asarray(lam, dtype=np.float64)
    if lam.size == 0:
        return qA.copy()
    lam_atom = np.where(site_of >= 0, lam[np.maximum(site_of, 0)], 0.0)
    return qA + lam_atom * (qB - qA)


def site_lists(site_of, n_sites):
    site_of = np.asarray(site_of)
    return [np.where(site_of == s)[0] for s in range(n_sites)]


def site_kernel(xs, L, rc=None):
    """A_ij and grad_i A(x_i - x_j) for the atoms of one site (f = 1)."""
    n = xs.shape[0]
    A = np.zeros((n, n))
    G = np.zeros((n, n, 3))
    for i in range(n):
        for j in range(n):
            v, g = pair_A(xs[i] - xs[j], L, rc)
            A[i, j] = v
            G[i, j] = g
    return A, G


def site_terms(xs, D, L):
    """k_s = f-free D^T A D and the pair-force sums -D_i sum_{j != i} D_j grad A(r_ij)
    for one site, as the energy (times 2) and forces of the charge set D alone:
    E(D) = 1/2 D^T A D with A_ii = xi (the same periodic kernel)."""
    phi, grad, e = ewald(xs, D, L, rc=0.5 * L)
    return 2.0 * e, -D[:, None] * grad


def hi_eval(sys, rc=None, targets=None, f=F_COULOMB, energy_only_full=False):
    """HI energy, dE/dlambda and forces for a two-form system.

    ``sys`` holds x, qA, qB, site_of, lam, L.  With ``targets`` None the full
    energy and all forces are returned; otherwise forces only at ``targets``
    (site atoms are always evaluated for dE/dlambda) and the energy only if
    ``energy_only_full`` (computed without per-atom potentials)."""
    x, qA, qB = sys["x"], sys["qA"], sys["qB"]
    site_of, lam, L = np.asarray(sys["site_of"]), np.asarray(sys["lam"]), sys["L"]
    S = lam.shape[0]
    qt = scaled_charges(qA, qB, site_of, lam)
    sites = site_lists(site_of, S)
    site_atoms = np.concatenate(sites) if S else np.zeros(0, dtype=np.int64)
    if targets is None:
        phi, grad, e = ewald(x, qt, L, rc)
        tgt = np.arange(qt.shape[0])
    else:
        tgt = np.unique(np.concatenate([np.asarray(targets, dtype=np.int64), site_atoms]))
        phi, grad, e = ewald(x, qt, L, rc, targets=tgt)
        if energy_only_full:
            e = ewald_energy(x, qt, L, rc)
    phi = phi * f
    grad = grad * f
    F = -qt[tgt, None] * grad
    pos = {int(i): k for k, i in enumerate(tgt)}
    dq = np.asarray(qB) - np.asarray(qA)
    k_s = np.zeros(S)
    g_s = np.zeros(S)
    for s, at in enumerate(sites):
        D = dq[at]
        kk, fcorr = site_terms(x[at], D, L)
        k_s[s] = f * kk
        g_s[s] = float(np.sum(D * phi[[pos[int(i)] for i in at]]))
        w = lam[s] * (1.0 - lam[s])
        for a, i in enumerate(at):
            F[pos[int(i)]] += w * f * fcorr[a]
    dEdl = g_s + (0.5 - lam) * k_s
    out = dict(F=F, targets=tgt, dEdl=dEdl, k=k_s, g=g_s, qt=qt)
    out["phi"] = phi
    if e is not None:
        Et = e * f
        out["E_qi"] = Et
        out["E"] = Et + float(np.sum(0.5 * lam * (1.0 - lam) * k_s))
    else:
        out["E"] = None
    return out


def hi_charge_gradients(sys, rc=None, f=F_COULOMB, ref=None):
    """Derivatives of the HI energy with respect to the two charge sets.

    With q~_i = (1 - lambda_s) qA_i + lambda_s qB_i and D = qB - qA, the energy
    E = E(q~) + sum_s 1/2 lambda_s (1 - lambda_s) k_s, k_s = f D_s^T A D_s, has
        dE/dqA_i = (1 - lambda_s) phi~_i - lambda_s (1 - lambda_s) psi_i
        dE/dqB_i = lambda_s phi~_i + lambda_s (1 - lambda_s) psi_i
    for an atom of site s, where phi~_i = dE(q~)/dq~_i is the charge-scaled
    potential and psi_i = f sum_{j in s} A_ij D_j = 1/2 dk_s/dD_i the potential
    of the site's charge change (self term included).  Environment atoms have
    q~ = qA: dE/dqA_i = phi~_i, dE/dqB_i = 0.  ``ref`` may pass a hi_eval result
    (full targets) to reuse its potentials."""
    x, qA, qB = sys["x"], np.asarray(sys["qA"]), np.asarray(sys["qB"])
    site_of, lam, L = np.asarray(sys["site_of"]), np.asarray(sys["lam"]), sys["L"]
    if ref is None:
        ref = hi_eval(sys, rc=rc, f=f)
    phi = ref["phi"]
    dqA = phi.copy()
    dqB = np.zeros_like(phi)
    psi = np.zeros_like(phi)
    dq = qB - qA
    for s, at in enumerate(site_lists(site_of, lam.shape[0])):
        if len(at) == 0:
            continue
        psi[at] = f * ewald(x[at], dq[at], L, rc=0.5 * L)[0]
        l = lam[s]
        dqA[at] = (1.0 - l) * phi[at] - l * (1.0 - l) * psi[at]
        dqB[at] = l * phi[at] + l * (1.0 - l) * psi[at]
    return dict(dqA=dqA, dqB=dqB, psi=psi)


def energy(x, q, L, rc=None, f=F_COULOMB):
    """Periodic Coulomb energy of one charge vector."""
    return ewald(x, q, L, rc)[2] * f


def hi_bruteforce(sys, rc=None, f=F_COULOMB):
    """HI energy and dE/dlambda by enumerating all 2^S protonation states
    (Eq. "rek_ham_lambda"); dE/dlambda_s = E(lambda_s = 1) - E(lambda_s = 0)
    at fixed other lambdas (Eq. "ref_two_forms" for one site)."""
    x, qA, qB = sys["x"], np.asarray(sys["qA"]), np.asarray(sys["qB"])
    site_of, lam, L = np.asarray(sys["site_of"]), np.asarray(sys["lam"]), sys["L"]
    S = lam.shape[0]
    if S > 6:
        raise ValueError("brute force limited to S <= 6")
    EX = {}
    for X in itertools.product((0, 1), repeat=S):
        sel = np.array([X[s] if s >= 0 else 0 for s in site_of])
        q = np.where((site_of >= 0) & (sel == 1), qB, qA)
        EX[X] = energy(x, q, L, rc, f)

    def interp(lv):
        tot = 0.0
        for X, e in EX.items():
            w = 1.0
            for s in range(S):
                w *= lv[s] if X[s] else (1.0 - lv[s])
            tot += w * e
        return tot

    E = interp(lam)
    dEdl = np.zeros(S)
    for s in range(S):
        l1 = lam.copy(); l1[s] = 1.0
        l0 = lam.copy(); l0[s] = 0.0
        dEdl[s] = interp(l1) - interp(l0)
    return dict(E=E, dEdl=dEdl, states=EX)


# ---------------------------------------------------------------------------
# Sites with more than two forms (Sec. "Hamiltonian Interpolation Formulation",
# general formulation Eq. "iter_ham_lambda"; Appendix, Eqs. "lambda_list",
# "one_site_lambda").  A site with F = 2^m forms has m lambdas; form rho is the
# binary number whose bit l selects lambda_l (bit set) or 1 - lambda_l, so its
# weight is lambda~_rho = prod_l (lambda_l if bit l of rho else 1 - lambda_l).
# ---------------------------------------------------------------------------
def lambda_tilde(lams):
    """Weights of the 2^m forms of one site from its m lambdas (bit l <-> lambda_l)."""
    lams = np.asarray(lams, dtype=np.float64)
    m = lams.shape[0]
    w = np.ones(1 << m)
    for rho in range(1 << m):
        for l in range(m):
            w[rho] *= lams[l] if (rho >> l) & 1 else 1.0 - lams[l]
    return w


def dlambda_tilde(lams):
    """d lambda~_rho / d lambda_l as an (m, 2^m) array: the weight with factor l
    replaced by +1 (bit set) or -1 (bit clear)."""
    lams = np.asarray(lams, dtype=np.float64)
    m = lams.shape[0]
    d = np.ones((m, 1 << m))
    for l in range(m):
        for rho in range(1 << m):
            for k in range(m):
                if k == l:
                    d[l, rho] *= 1.0 if (rho >> k) & 1 else -1.0
                else:
                    d[l, rho] *= lams[k] if (rho >> k) & 1 else 1.0 - lams[k]
    return d


def multiform_eval(sys, rc=None, f=F_COULOMB):
    """HI energy, dE/dlambda and forces for sites with 2^m forms.

    ``sys`` holds x, q_env (charges of environment atoms; site entries unused),
    site_of, forms (list over sites of (F_s, n_s) arrays: charges of the site's
    atoms, in increasing atom index, in each form), lams (list over sites of
    m_s lambdas) and L.  With q~ = sum_rho lambda~_rho q^rho at site atoms, the
    general formulation equals the charge-scaled energy E(q~) plus, per site,
        C = f/2 [sum_rho lambda~_rho G_rho,rho - sum_rho,rho' lambda~_rho lambda~_rho' G_rho,rho']
    with G_rho,rho' = q^rho^T A q^rho' over the site (self term included):
    cross-site and environment terms are bilinear in the scaled charges and
    agree between the two.  Derivatives:
        dE/dlambda_l = sum_rho (d lambda~_rho / d lambda_l)
                       (q^rho . phi~ + f (1/2 G_rho,rho - (G lambda~)_rho)),
        F_i = -q~_i grad phi~_i - grad_i C,
        grad_i C = f [sum_rho lambda~_rho q_i^rho grad_i phi^rho - q~_i grad_i phi^q~]
    where phi^u is the potential of the site-only charge set u (f = 1)."""
    x, L = sys["x"], sys["L"]
    site_of = np.asarray(sys["site_of"])
    q = np.asarray(sys["q_env"], dtype=np.float64).copy()
    sites = site_lists(site_of, len(sys["forms"]))
    lt = [lambda_tilde(l) for l in sys["lams"]]
    for s, at in enumerate(sites):
        q[at] = lt[s] @ np.asarray(sys["forms"][s])
    phi, grad, e = ewald(x, q, L, rc)
    phi = phi * f
    grad = grad * f
    F = -q[:, None] * grad
    E = e * f
    dEdl = []
    for s, at in enumerate(sites):
        Q = np.asarray(sys["forms"][s], dtype=np.float64)      # (F, n)
        w = lt[s]
        xs = x[at]
        T = np.zeros_like(Q)                                   # A q^rho per form
        Gr = np.zeros(Q.shape + (3,))                          # grad of phi^rho
        for r in range(Q.shape[0]):
            p_r, g_r, _ = ewald(xs, Q[r], L, rc=0.5 * L)
            T[r] = p_r
            Gr[r] = g_r
        G = Q @ T.T
        E += 0.5 * f * (w @ np.diag(G) - w @ G @ w)
        pq, gq, _ = ewald(xs, q[at], L, rc=0.5 * L)
        gradC = f * (np.einsum("r,ri,rik->ik", w, Q, Gr) - q[at][:, None] * gq)
        F[at] -= gradC
        dl = dlambda_tilde(sys["lams"][s])
        per_form = Q @ phi[at] + f * (0.5 * np.diag(G) - G @ w)
        dEdl.append(dl @ per_form)
    return dict(E=E, F=F, dEdl=np.concatenate(dEdl) if dEdl else np.zeros(0), qt=q, phi=phi)


def multiform_charge_gradients(sys, rc=None, f=F_COULOMB, ref=None):
    """dE/dq_env and dE/dq^rho of the multi-form HI energy (the derivative of
    multiform_eval's E in the charges; the paper has no charge gradients).
    With E = E(q~) + sum_s f/2 [sum_rho w_rho G_rho,rho - w^T G w],
    q~ = sum_rho w_rho q^rho at site atoms and G_rho,rho' = q^rho^T A q^rho':
      dE/dq_env_i = phi~_i (environment atoms; 0 for site atoms, whose q_env
                    entries are not used),
      dE/dq^rho_i = w_rho (phi~_i + f (A q^rho)_i - f (A q~_s)_i)  (site atoms),
    A over the site's atoms with the self term (the same periodic kernel)."""
    ref = multiform_eval(sys, rc, f) if ref is None else ref
    x, L = sys["x"], sys["L"]
    site_of = np.asarray(sys["site_of"])
    sites = site_lists(site_of, len(sys["forms"]))
    dq_env = np.where(site_of < 0, ref["phi"], 0.0)
    dq_forms = []
    for s, at in enumerate(sites):
        Q = np.asarray(sys["forms"][s], dtype=np.float64)
        w = lambda_tilde(sys["lams"][s])
        xs = x[at]
        psi = np.array([ewald(xs, Q[r], L, rc=0.5 * L)[0] for r in range(Q.shape[0])]) * f   # f A q^rho
        psit = w @ psi
        dq_forms.append(w[:, None] * (ref["phi"][at][None, :] + psi - psit[None, :]))
    return dict(dq_env=dq_env, dq_forms=dq_forms)


def multiform_bruteforce(sys, rc=None, f=F_COULOMB):
    """The multilinear definition (Eq. "rek_ham_lambda" with Eq. "one_site_lambda"
    per site): E = sum over every choice of one form per site of the product of
    the forms' weights times the periodic energy of that charge set; dE/dlambda
    by the exact central difference of this multilinear function."""
    x, L = sys["x"], sys["L"]
    site_of = np.asarray(sys["site_of"])
    sites = site_lists(site_of, len(sys["forms"]))
    nf = [np.asarray(fm).shape[0] for fm in sys["forms"]]
    EX = {}
    for X in itertools.product(*[range(n) for n in nf]):
        q = np.asarray(sys["q_env"], dtype=np.float64).copy()
        for s, at in enumerate(sites):
            q[at] = np.asarray(sys["forms"][s])[X[s]]
        EX[X] = energy(x, q, L, rc, f)

    def interp(lams):
        lt = [lambda_tilde(l) for l in lams]
        tot = 0.0
        for X, e in EX.items():
            w = 1.0
            for s in range(len(X)):
                w *= lt[s][X[s]]
            tot += w * e
        return tot

    lams = [np.asarray(l, dtype=np.float64) for l in sys["lams"]]
    E = interp(lams)
    dEdl = []
    h = 0.25
    for s in range(len(lams)):
        for l in range(lams[s].shape[0]):
            lp = [v.copy() for v in lams]; lp[s][l] += h
            lm = [v.copy() for v in lams]; lm[s][l] -= h
            dEdl.append((interp(lp) - interp(lm)) / (2 * h))
    return dict(E=E, dEdl=np.array(dEdl))
