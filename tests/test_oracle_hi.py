"""Pins for the HI oracle: 2^S brute force vs closed form, multilinearity,
finite differences in lambda and x, the HI-QI difference (Eqs. DeltaFQIHI, Udiff)."""
import json
import os

import numpy as np
import pytest

import oracle
from oracle import hi

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def paper_random_system(seed=1, clustered=True):
    """1000 environment + 10 site particles, charges U(-1,1) (Sec. 'Random Systems').
    The site's second form draws fresh U(-1,1) charges."""
    g = json.load(open(os.path.join(GOLD, "paper_random_system.json")))
    rng = np.random.default_rng(seed)
    L = 3.0
    ne, ns = g["n_environment"], g["n_site"]
    x = rng.uniform(0, L, (ne + ns, 3))
    if clustered:
        c = rng.uniform(0, L, 3)
        x[ne:] = np.mod(c + rng.uniform(-0.25, 0.25, (ns, 3)), L)
    lo, hi_ = g["charge_range"]
    qA = rng.uniform(lo, hi_, ne + ns)
    qB = qA.copy()
    qB[ne:] = rng.uniform(lo, hi_, ns)
    site_of = np.full(ne + ns, -1, dtype=np.int32)
    site_of[ne:] = 0
    return dict(x=x, qA=qA, qB=qB, site_of=site_of, lam=np.array([g["lambda_two_forms"]]), L=L)


def small_multisite(seed=3, n=80, S=3, L=1.8):
    rng = np.random.default_rng(seed)
    x = rng.uniform(0, L, (n, 3))
    qA = rng.uniform(-1, 1, n)
    qB = qA.copy()
    site_of = np.full(n, -1, dtype=np.int32)
    for s in range(S):
        at = np.arange(s * 4, s * 4 + 4)
        site_of[at] = s
        qB[at] = qA[at] + rng.uniform(-0.5, 0.5, 4)
    return dict(x=x, qA=qA, qB=qB, site_of=site_of, lam=rng.uniform(0, 1, S), L=L)


def test_two_form_reference_lambda_force():
    """Eq. ref_two_forms: dH/dlambda = H_1 - H_0 for the paper's random system."""
    s = paper_random_system()
    out = hi.hi_eval(s)
    e0 = hi.energy(s["x"], s["qA"], s["L"])
    e1 = hi.energy(s["x"], s["qB"], s["L"])
    assert out["dEdl"][0] == pytest.approx(e1 - e0, rel=1e-10)
    lam = s["lam"][0]
    assert out["E"] == pytest.approx((1 - lam) * e0 + lam * e1, rel=1e-11)


def test_closed_form_equals_bruteforce():
    s = small_multisite()
    out = hi.hi_eval(s)
    bf = hi.hi_bruteforce(s)
    assert out["E"] == pytest.approx(bf["E"], rel=1e-11)
    np.testing.assert_allclose(out["dEdl"], bf["dEdl"], rtol=1e-9, atol=1e-9)


def test_hi_minus_qi_is_harmonic_in_lambda():
    """Eq. Udiff: E_QI - E_HI = k/2 (lambda^2 - lambda), with k from the brute force
    states: k = E(A) + E(B) - 2 E((A+B)/2) ... evaluated through the interpolation."""
    s = small_multisite(S=2)
    out = hi.hi_eval(s)
    bf = hi.hi_bruteforce(s)
    lam = s["lam"]
    diff = out["E_qi"] - bf["E"]
    assert diff == pytest.approx(float(np.sum(0.5 * out["k"] * (lam ** 2 - lam))), rel=1e-9)
    # Eq. DeltaFQIHI: dE_QI/dlambda = dE_HI/dlambda + (lambda - 1/2) k
    np.testing.assert_allclose(out["g"], out["dEdl"] + (lam - 0.5) * out["k"], rtol=1e-12)


def test_multilinear_in_each_lambda():
    s = small_multisite()
    base = hi.hi_eval(s)
    for sidx in range(3):
        s2 = dict(s); s2["lam"] = s["lam"].copy(); s2["lam"][sidx] = 0.9 - 0.7 * s["lam"][sidx]
        o2 = hi.hi_eval(s2)
        assert o2["dEdl"][sidx] == pytest.approx(base["dEdl"][sidx], rel=1e-10)
    # HI equals QI when every lambda sits at an end point
    s4 = dict(s); s4["lam"] = np.array([1.0, 0.0, 1.0])
    o4 = hi.hi_eval(s4)
    assert o4["E"] == pytest.approx(o4["E_qi"], rel=1e-14)
    assert np.all(o4["k"] != 0.0)


def test_lambda_central_difference_exact():
    s = small_multisite()
    base = hi.hi_eval(s)
    h = 0.05
    for sidx in range(3):
        sp = dict(s); sp["lam"] = s["lam"].copy(); sp["lam"][sidx] += h
        sm = dict(s); sm["lam"] = s["lam"].copy(); sm["lam"][sidx] -= h
        d = (hi.hi_eval(sp)["E"] - hi.hi_eval(sm)["E"]) / (2 * h)
        assert d == pytest.approx(base["dEdl"][sidx], rel=1e-9)


def test_forces_central_difference():
    s = small_multisite(n=40, S=2)
    base = hi.hi_eval(s)
    h = 1e-5
    for k in (0, 1, 5, 30):  # site atoms and environment atoms
        for ax in range(3):
            xp = s["x"].copy(); xp[k, ax] += h
            xm = s["x"].copy(); xm[k, ax] -= h
            ep = hi.hi_eval(dict(s, x=xp))["E"]
            em = hi.hi_eval(dict(s, x=xm))["E"]
            assert -(ep - em) / (2 * h) == pytest.approx(base["F"][k, ax], rel=2e-6, abs=1e-5)


def test_subset_targets_match_full():
    s = small_multisite()
    full = hi.hi_eval(s)
    part = hi.hi_eval(s, targets=np.array([20, 50, 70]))
    np.testing.assert_allclose(part["dEdl"], full["dEdl"], rtol=1e-12)
    for k, i in enumerate(part["targets"]):
        np.testing.assert_allclose(part["F"][k], full["F"][i], atol=1e-10)


def test_site_terms_match_pairwise_kernel():
    """k_s and the intra-site force sums through E(D) of the charge set D alone
    equal the explicit pair sums with A_ij (A_ii = xi)."""
    rng = np.random.default_rng(11)
    L = 2.6
    xs = np.mod(rng.uniform(0, 0.4, (6, 3)) + 1.1, L)
    D = rng.uniform(-0.4, 0.4, 6)
    kk, fc = hi.site_terms(xs, D, L)
    A, G = hi.site_kernel(xs, L)
    assert kk == pytest.approx(D @ A @ D, rel=1e-12)
    for a in range(6):
        ref = -sum(D[a] * D[b] * G[a, b] for b in range(6) if b != a)
        np.testing.assert_allclose(fc[a], ref, atol=1e-10)


def test_charge_gradients_central_difference_exact():
    """dE/dqA and dE/dqB against central differences of the HI energy.  E is a
    quadratic polynomial in the charges, so the central difference is exact up
    to rounding for any step.  Environment atoms use qA only (dE/dqB = 0)."""
    s = small_multisite(n=40, S=2)
    g = hi.hi_charge_gradients(s)
    h = 0.05
    for k in (0, 3, 5, 9, 30):  # atoms of site 0, of site 1 and of the environment
        for key in ("qA", "qB"):
            sp = dict(s); sp[key] = s[key].copy(); sp[key][k] += h
            sm = dict(s); sm[key] = s[key].copy(); sm[key][k] -= h
            d = (hi.hi_eval(sp)["E"] - hi.hi_eval(sm)["E"]) / (2 * h)
            assert d == pytest.approx(g["d" + key][k], rel=1e-9, abs=1e-9), (k, key)


def test_charge_gradients_match_bruteforce_states():
    """Through Eq. rek_ham_lambda: dE/dqB_i = sum over states with site s in form
    B of the state weight times that state's potential at i (and likewise for
    qA with form A); for one site these are lambda phi_B and (1 - lambda) phi_A."""
    s = paper_random_system()
    g = hi.hi_charge_gradients(s)
    lam = s["lam"][0]
    phiA = oracle.ewald(s["x"], s["qA"], s["L"])[0] * oracle.F_COULOMB
    phiB = oracle.ewald(s["x"], s["qB"], s["L"])[0] * oracle.F_COULOMB
    site = s["site_of"] == 0
    np.testing.assert_allclose(g["dqB"][site], lam * phiB[site], rtol=1e-9, atol=1e-9)
    np.testing.assert_allclose(g["dqA"][site], (1 - lam) * phiA[site], rtol=1e-9, atol=1e-9)
    # environment: one charge, weighted over both states
    env = ~site
    np.testing.assert_allclose(g["dqA"][env], (1 - lam) * phiA[env] + lam * phiB[env], rtol=1e-9, atol=1e-9)
    assert not g["dqB"][env].any()


def small_multiform(seed=7, n=60, L=1.9, nforms=(4, 2, 8)):
    """Environment charges plus sites of 3-4 atoms with 2^m forms each."""
    rng = np.random.default_rng(seed)
    x = rng.uniform(0, L, (n, 3))
    q_env = rng.uniform(-1, 1, n)
    site_of = np.full(n, -1, dtype=np.int32)
    forms, lams = [], []
    k = 0
    for s, F in enumerate(nforms):
        na = 3 + (s % 2)
        at = np.arange(k, k + na)
        k += na
        site_of[at] = s
        forms.append(q_env[at][None, :] + rng.uniform(-0.5, 0.5, (F, na)))
        lams.append(rng.uniform(0, 1, int(np.log2(F))))
    return dict(x=x, q_env=q_env, site_of=site_of, forms=forms, lams=lams, L=L)


def test_lambda_tilde_sums_to_one_and_matches_paper_example():
    """Eq. constraint (sum of the form weights is 1) and Eq. one_site_lambda for
    four forms: (1-l1)(1-l0), (1-l1) l0, l1 (1-l0), l1 l0."""
    l0, l1 = 0.3, 0.8
    w = hi.lambda_tilde([l0, l1])
    np.testing.assert_allclose(w, [(1 - l1) * (1 - l0), (1 - l1) * l0, l1 * (1 - l0), l1 * l0], rtol=1e-15)
    for m in range(1, 5):
        lams = np.random.default_rng(m).uniform(0, 1, m)
        assert hi.lambda_tilde(lams).sum() == pytest.approx(1.0, abs=1e-15)
        d = hi.dlambda_tilde(lams)
        np.testing.assert_allclose(d.sum(axis=1), 0.0, atol=1e-15)


def test_multiform_closed_form_equals_bruteforce():
    s = small_multiform()
    cf = hi.multiform_eval(s)
    bf = hi.multiform_bruteforce(s)
    assert cf["E"] == pytest.approx(bf["E"], rel=1e-11)
    np.testing.assert_allclose(cf["dEdl"], bf["dEdl"], rtol=1e-9, atol=1e-9)


def test_multiform_two_forms_reduce_to_two_form_path():
    s = small_multisite(n=50, S=2)
    sites = hi.site_lists(s["site_of"], 2)
    mf = dict(x=s["x"], q_env=s["qA"], site_of=s["site_of"], L=s["L"],
              forms=[np.stack([s["qA"][at], s["qB"][at]]) for at in sites], lams=[[v] for v in s["lam"]])
    a = hi.multiform_eval(mf)
    b = hi.hi_eval(s)
    assert a["E"] == pytest.approx(b["E"], rel=1e-12)
    np.testing.assert_allclose(a["dEdl"], b["dEdl"], rtol=1e-10)
    np.testing.assert_allclose(a["F"], b["F"], atol=1e-8)


def test_multiform_forces_central_difference():
    s = small_multiform(n=30, nforms=(4, 2))
    base = hi.multiform_eval(s)
    h = 1e-5
    for k in (0, 2, 4, 20):  # site atoms and an environment atom
        for ax in range(3):
            xp = s["x"].copy(); xp[k, ax] += h
            xm = s["x"].copy(); xm[k, ax] -= h
            ep = hi.multiform_eval(dict(s, x=xp))["E"]
            em = hi.multiform_eval(dict(s, x=xm))["E"]
            assert -(ep - em) / (2 * h) == pytest.approx(base["F"][k, ax], rel=2e-6, abs=1e-5)


def test_multiform_charge_gradients_central_difference_exact():
    """dE/dq_env and dE/dq^rho of the multi-form energy against central
    differences of multiform_eval's E: E is quadratic in every charge, so the
    central difference is exact up to rounding for any step."""
    s = small_multiform(n=30, nforms=(4, 2))
    g = hi.multiform_charge_gradients(s)
    h = 0.05
    for k in (20, 25):   # environment atoms
        sp = dict(s, q_env=s["q_env"].copy()); sp["q_env"][k] += h
        sm = dict(s, q_env=s["q_env"].copy()); sm["q_env"][k] -= h
        d = (hi.multiform_eval(sp)["E"] - hi.multiform_eval(sm)["E"]) / (2 * h)
        assert d == pytest.approx(g["dq_env"][k], rel=1e-9, abs=1e-9)
    assert not g["dq_env"][s["site_of"] >= 0].any()
    for si, (r, a) in ((0, (0, 0)), (0, (3, 2)), (1, (1, 1)), (1, (0, 3))):
        fp = [f.copy() for f in s["forms"]]; fp[si][r, a] += h
        fm = [f.copy() for f in s["forms"]]; fm[si][r, a] -= h
        d = (hi.multiform_eval(dict(s, forms=fp))["E"] - hi.multiform_eval(dict(s, forms=fm))["E"]) / (2 * h)
        assert d == pytest.approx(g["dq_forms"][si][r, a], rel=1e-9, abs=1e-9), (si, r, a)


def test_multiform_charge_gradients_reduce_to_two_forms():
    """With two forms per site the gradients are the two-form path's dE/dqA
    and dE/dqB at site atoms, and dE/dqA at environment atoms."""
    s = small_multisite(n=50, S=2)
    sites = hi.site_lists(s["site_of"], 2)
    mf = dict(x=s["x"], q_env=s["qA"], site_of=s["site_of"], L=s["L"],
              forms=[np.stack([s["qA"][at], s["qB"][at]]) for at in sites], lams=[[v] for v in s["lam"]])
    a = hi.multiform_charge_gradients(mf)
    b = hi.hi_charge_gradients(s)
    env = s["site_of"] < 0
    np.testing.assert_allclose(a["dq_env"][env], b["dqA"][env], rtol=1e-10, atol=1e-10)
    for si, at in enumerate(sites):
        np.testing.assert_allclose(a["dq_forms"][si][0], b["dqA"][at], rtol=1e-10, atol=1e-10)
        np.testing.assert_allclose(a["dq_forms"][si][1], b["dqB"][at], rtol=1e-10, atol=1e-10)
