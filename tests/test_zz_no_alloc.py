"""The allocation-free per-site entry point (mahi_site_terms_static) against
the library's own evaluation and the oracle.

It exists for callers that cannot allocate device memory where they need the
per-site terms (stream capture, externally owned memory pools, other solvers
producing the charge-scaled potential).  Given the potential that mahi_eval
used (mahi_get_potential), it must reproduce mahi_eval's dE/dlambda, and its
energy and force corrections must match the oracle's intra-site terms
(k_s = f D^T A D over the site's atoms and their pair forces), on two calls
in a row (its scratch is reused).  A call captured into a CUDA graph must give
the same bits (nothing on its path may allocate or synchronise), and a site
with an atom index out of range must come back as NaN without any access.
Collected last on purpose."""
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
    # energy and force corrections against the oracle's intra-site terms:
    # sum_s 1/2 lam (1 - lam) f k_s, and the pair forces of each site
    dq = s["qB"] - s["qA"]
    e_ref = 0.0
    tol = 1e-9 if xdt == "float64" else 1e-5   # float32 positions enter the pair distances
    for k in range(S):
        at = atoms[ptr[k]:ptr[k + 1]]
        xs = np.asarray(x[at.tolist()].double().cpu().numpy())
        ks, fc = hi.site_terms(xs, dq[at], L)
        w = s["lam"][k] * (1 - s["lam"][k]) * oracle.F_COULOMB
        e_ref += 0.5 * w * ks
        np.testing.assert_allclose(f1[at], w * fc, rtol=tol, atol=tol * (1 + np.abs(w * fc).max()))
    assert e1 == pytest.approx(e_ref, rel=1e-9, abs=1e-9)
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


def test_static_site_terms_in_a_captured_graph():
    """One call captured into a CUDA graph on a side stream (after the set-up
    call): the replay must give the uncaptured call's bits."""
    s = synth.make_water(n_water=2000, grid=16, L=3.9, n_sites=6, seed=22, depth=3, order=8)
    N, S, L = len(s["qA"]), len(s["lam"]), s["L"]
    dev = torch.device("cuda")
    ptr, atoms = _csr(s["site_of"], S)
    d_ptr, d_atoms = torch.tensor(ptr, device=dev), torch.tensor(atoms, device=dev)
    x = torch.tensor(s["x"], dtype=torch.float64, device=dev)
    qA = torch.tensor(s["qA"], dtype=torch.float64, device=dev)
    qB = torch.tensor(s["qB"], dtype=torch.float64, device=dev)
    lam = torch.tensor(s["lam"], dtype=torch.float64, device=dev)
    phi = torch.linspace(-300.0, 300.0, N, dtype=torch.float64, device=dev)
    outs = [(torch.zeros(S, dtype=torch.float64, device=dev), torch.zeros(1, dtype=torch.float64, device=dev),
             torch.zeros((N, 3), dtype=torch.float64, device=dev)) for _ in range(2)]
    pkg.mahi_site_terms_static(L, d_ptr, d_atoms, x, qA, qB, lam, phi, *outs[0])   # set-up call, uncaptured
    torch.cuda.synchronize()
    side = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=side):
        pkg.mahi_site_terms_static(L, d_ptr, d_atoms, x, qA, qB, lam, phi, *outs[1], stream=side)
    g.replay()
    torch.cuda.synchronize()
    for a, b in zip(outs[0], outs[1]):
        assert torch.equal(a, b)


def test_static_site_terms_flag_an_out_of_range_atom():
    """A site naming an atom beyond n_atoms gets NaN and is not touched; the
    other sites are evaluated as usual."""
    dev = torch.device("cuda")
    N, L = 40, 3.0
    rng = np.random.default_rng(3)
    x = torch.tensor(rng.uniform(0, L, (N, 3)), dtype=torch.float64, device=dev)
    qA = torch.tensor(rng.uniform(-0.5, 0.5, N), dtype=torch.float64, device=dev)
    qB = qA + 0.25
    lam = torch.tensor([0.3, 0.6], dtype=torch.float64, device=dev)
    phi = torch.zeros(N, dtype=torch.float64, device=dev)
    ptr = torch.tensor([0, 3, 6], dtype=torch.int32, device=dev)
    atoms = torch.tensor([1, 2, 3, 4, N + 7, 5], dtype=torch.int32, device=dev)   # site 1 is malformed
    dEdl = torch.zeros(2, dtype=torch.float64, device=dev)
    ecor = torch.zeros(1, dtype=torch.float64, device=dev)
    F = torch.zeros((N, 3), dtype=torch.float64, device=dev)
    pkg.mahi_site_terms_static(L, ptr, atoms, x, qA, qB, lam, phi, dEdl, ecor, F)
    torch.cuda.synchronize()
    d = dEdl.cpu().numpy()
    assert np.isfinite(d[0]) and np.isnan(d[1]) and np.isnan(ecor.item())
    Fh = F.cpu().numpy()
    assert not Fh[[4, 5]].any()             # atoms of the malformed site untouched
    assert Fh[[1, 2, 3]].any()
