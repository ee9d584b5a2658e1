"""Batched replicas in one CUDA graph (mahi_batch_*) and the launch-shape
autotuner (mahi_autotune): the graph reproduces one mahi_eval per replica
bit for bit, follows in-place input updates between launches, and tuning
changes results only at the rounding level of reordered sums."""
import numpy as np
import pytest

import paper_2410_01754_gb300 as pkg
import synth

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA device")]

# uneven replicas: (waters, lattice side, box nm, sites, depth)
REPLICAS = [(1000, 11, 3.38, 2, 2), (3000, 15, 4.61, 4, 3), (10000, 22, 6.76, 7, 3)]


def _replica(k, spec, prec):
    nw, grid, L, S, d = spec
    s = synth.make_water(n_water=nw, grid=grid, L=L, n_sites=S, seed=30 + k, depth=d, order=10)
    h = pkg.mahi_create(L, len(s["qA"]), S, 10, d, prec)
    pkg.mahi_set_charges(h, s["qA"], s["qB"], s["site_of"])
    dev = torch.device("cuda")
    x = torch.tensor(s["x"], dtype=torch.float32, device=dev)
    lam = torch.tensor(s["lam"], dtype=torch.float64, device=dev)
    return s, h, x, lam


def _outputs(x, S):
    dev = x.device
    return (torch.zeros(1, dtype=torch.float64, device=dev), torch.zeros_like(x),
            torch.zeros(max(1, S), dtype=torch.float64, device=dev))


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_graph_matches_individual_evaluations(prec):
    stream = torch.cuda.Stream()
    reps = [_replica(k, spec, prec) for k, spec in enumerate(REPLICAS)]
    ref = []
    for s, h, x, lam in reps:
        pkg.mahi_set_stream(h, stream)
        E, F, g = _outputs(x, len(s["lam"]))
        pkg.mahi_eval(h, x, lam, E, F, g)
        stream.synchronize()
        ref.append((E.item(), F.cpu().numpy().copy(), g.cpu().numpy().copy()))
    outs = [_outputs(x, len(s["lam"])) for s, h, x, lam in reps]
    b = pkg.MahiBatch([r[1] for r in reps], stream, [r[2] for r in reps], [r[3] for r in reps],
                      [o[0] for o in outs], [o[1] for o in outs], [o[2] for o in outs])
    for o in outs:  # clear what the capture pass wrote
        for t in o:
            t.zero_()
    torch.cuda.synchronize()
    b.launch()
    stream.synchronize()
    for (E0, F0, g0), (E, F, g) in zip(ref, outs):
        assert E.item() == E0
        assert np.array_equal(F.cpu().numpy(), F0) and np.array_equal(g.cpu().numpy(), g0)
    # in-place update of the inputs: move every replica by one box edge (same
    # physics after wrapping) and one lambda; the graph follows
    for k, (s, h, x, lam) in enumerate(reps):
        x.add_(float(s["L"]))
        lam[0] = 0.25
    torch.cuda.synchronize()
    b.launch()
    stream.synchronize()
    for k, (s, h, x, lam) in enumerate(reps):
        E, F, g = _outputs(x, len(s["lam"]))
        pkg.mahi_eval(h, x, lam, E, F, g)
        stream.synchronize()
        assert outs[k][0].item() == E.item()
        assert np.array_equal(outs[k][2].cpu().numpy(), g.cpu().numpy())
    b.close()
    for s, h, x, lam in reps:
        pkg.mahi_destroy(h)


def test_batch_rejects_null_stream():
    s, h, x, lam = _replica(0, REPLICAS[0], "mixed")
    E, F, g = _outputs(x, len(s["lam"]))
    with pytest.raises(pkg.MahiError) as ei:
        pkg.MahiBatch([h], None, [x], [lam], [E], [F], [g])
    assert ei.value.code == -1
    pkg.mahi_destroy(h)


def test_autotune_keeps_results():
    s = synth.make_water(n_water=20000, grid=28, L=8.6, n_sites=16, seed=41, depth=4, order=12)
    N, S = len(s["qA"]), 16
    m = pkg.Mahi(s["L"], N, S, 12, 4, "mixed")
    m.set_charges(s["qA"], s["qB"], s["site_of"])
    x = torch.tensor(s["x"], dtype=torch.float32, device="cuda")
    lam = torch.tensor(s["lam"], dtype=torch.float64, device="cuda")
    E0, F0, g0 = m.eval(x, lam)
    torch.cuda.synchronize()
    pkg.mahi_autotune(m.h, x, lam, 2)
    p2p, blocks = pkg.mahi_get_tuning(m.h)
    assert p2p in (64, 128, 256) and blocks in range(0, 17)
    assert m.get_option("p2p_threads") == p2p and m.get_option("site_blocks") == blocks
    assert m.get_option("p2p_targets") in (8, 4, -1)
    assert m.get_option("m2l_single_tile") in (0, 1) and m.get_option("m2l_b_stages") in (0, 2, 3)
    E1, F1, g1 = m.eval(x, lam)
    torch.cuda.synchronize()
    m.close()
    a, b = F0.double().cpu().numpy(), F1.double().cpu().numpy()
    # the M2L's tile choice changes which rows share an accumulator's rounding
    # history only through the order of the items (the same per unit), so the
    # results move at the single-precision rounding level
    assert np.sqrt(((a - b) ** 2).sum() / (a ** 2).sum()) < 1e-6
    assert abs(E0.item() - E1.item()) < 1e-8 * abs(E0.item())
    assert np.abs(g0.cpu().numpy() - g1.cpu().numpy()).max() < 1e-6
