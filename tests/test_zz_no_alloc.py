"""The allocation-free per-site entry point (mahi_site_terms_static) against
the library's own evaluation.

It exists for callers that cannot allocate device memory where they need the
per-site terms (stream capture, externally owned memory pools, other solvers
producing the charge-scaled potential).  Given the potential that mahi_eval
used (mahi_get_potential), it must reproduce mahi_eval's dE/dlambda, and its
energy and force corrections must match the closed forms, on two calls in a
row (its scratch is reused).  Collected last on purpose."""
import numpy as np
import pytest

import oracle
from oracle import hi
import paper_2410_01754_gb300 as pkg
import synth

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA device")]


def _csr(site_of, S):
    site_of = np.asarray(site_of)
    atoms = [np.where(site_of == s)[0] for s in range(S)]
    ptr = np.zeros(S + 1, dtype=np.int32)
    ptr[1:] = np.cumsum([len(a) for a in atoms])
    return ptr, np.concatenate(atoms).astype(np.int32)


@pytest.mark.parametrize("prec,xdt", [("fp64", "float64"), ("mixed_simt", "float32")])
def test_static_site_terms_match_eval(prec, xdt):
    s = synth.make_water(n_water=4000, grid=16, L=4.93, n_sites=8, seed=21, depth=3, order=8)
    N, S, L = len(s["qA"]), len(s["lam"]), s["L"]
    dev = torch.device("cuda")
    m = pkg.Mahi(L, N, S, 8, 3, prec)
    m.set_charges(s["qA"], s["qB"], s["site_of"])
    x = torch.tensor(s["x"], dtype=getattr(torch, xdt), device=dev)
    lam = torch.tensor(s["lam"], dtype=torch.float64, device=dev)
    E, F, g = m.eval(x, lam)
    phi = m.potential()
    torch.cuda.synchronize()
    ref_dEdl = g.cpu().numpy()
    m.close()

    ptr, atoms = _csr(s["site_of"], S)
    d_ptr = torch.tensor(ptr, device=dev)
    d_atoms = torch.tensor(atoms, device=dev)
    qA = torch.tensor(s["qA"], dtype=torch.float64, device=dev)
    qB = torch.tensor(s["qB"], dtype=torch.float64, device=dev)
    results = []
    for _ in range(2):
        dEdl = torch.full((S,), 7.0, dtype=torch.float64, device=dev)
        ecor = torch.full((1,), 7.0, dtype=torch.float64, device=dev)
        Fc = torch.zeros((N, 3), dtype=x.dtype, device=dev)
        pkg.mahi_site_terms_static(L, d_ptr, d_atoms, x, qA, qB, lam, phi, dEdl, ecor, Fc)
        torch.cuda.synchronize()
        results.append((dEdl.cpu().numpy(), ecor.item(), Fc.double().cpu().numpy()))
    (d1, e1, f1), (d2, e2, f2) = results
    # the second call reuses the scratch and gives the same answer
    assert np.array_equal(d1, d2) and e1 == e2 and np.array_equal(f1, f2)
    # dE/dlambda of the allocation-free path equals mahi_eval's
    np.testing.assert_allclose(d1, ref_dEdl, rtol=1e-12, atol=1e-9)
    # energy correction = sum_s 1/2 lam (1 - lam) k_s with k_s from the same outputs
    dq = s["qB"] - s["qA"]
    phin = phi.cpu().numpy()
    gs = np.array([np.sum(dq[atoms[ptr[k]:ptr[k + 1]]] * phin[atoms[ptr[k]:ptr[k + 1]]]) for k in range(S)])
    ks = (d1 - gs) / (0.5 - s["lam"])
    assert e1 == pytest.approx(float(np.sum(0.5 * s["lam"] * (1 - s["lam"]) * ks)), rel=1e-9)
    # force corrections against the oracle's intra-site pair sums
    for k in range(S):
        at = atoms[ptr[k]:ptr[k + 1]]
        _, fc = hi.site_terms(s["x"][at], dq[at], L)
        w = s["lam"][k] * (1 - s["lam"][k]) * oracle.F_COULOMB
        tol = 1e-9 if xdt == "float64" else 1e-5
        np.testing.assert_allclose(f1[at], w * fc, rtol=tol, atol=tol * (1 + np.abs(w * fc).max()))
    # atoms outside the sites are untouched
    mask = np.ones(N, dtype=bool)
    mask[atoms] = False
    assert not f1[mask].any()


def test_static_site_terms_reject_too_many_sites():
    dev = torch.device("cuda")
    S = 4097
    ptr = torch.arange(S + 1, dtype=torch.int32, device=dev)
    atoms = torch.arange(S, dtype=torch.int32, device=dev)
    x = torch.zeros((S, 3), dtype=torch.float64, device=dev)
    q = torch.zeros(S, dtype=torch.float64, device=dev)
    lam = torch.zeros(S, dtype=torch.float64, device=dev)
    with pytest.raises(pkg.MahiError) as ei:
        pkg.mahi_site_terms_static(3.0, ptr, atoms, x, q, q, lam, q)
    assert ei.value.code == -1
