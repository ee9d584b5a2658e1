"""Helpers shared by the GPU tests: run the library on a seeded system."""
import numpy as np

import paper_2410_01754_gb300 as pkg


def run_gpu(s, prec, p=None, d=None, x_dtype="float64", evals=1, options=None):
    import torch
    p = s["order"] if p is None else p
    d = s["depth"] if d is None else d
    N, S = len(s["qA"]), len(s["lam"])
    m = pkg.Mahi(s["L"], N, S, p, d, prec)
    try:
        m.set_charges(s["qA"], s["qB"], s["site_of"])
        for k, v in (options or {}).items():
            m.set_option(k, v)
        x = torch.tensor(s["x"], dtype=getattr(torch, x_dtype), device="cuda")
        lam = torch.tensor(s["lam"], dtype=torch.float64, device="cuda")
        for _ in range(evals):
            E, F, g = m.eval(x, lam)
        phi = m.potential()
        torch.cuda.synchronize()
        return dict(E=E.item(), F=F.double().cpu().numpy(), dEdl=g.cpu().numpy(), phi=phi.cpu().numpy(),
                    launches=pkg.mahi_launch_count(m.h))
    finally:
        m.close()


def errors(res, ref, idx=None):
    """Force error as relative RMS (Frel) and as the worst single atom,
    |F_i - F_ref,i| / rms_i |F_ref,i| (Fmax, at atom Fmax_atom, an index into
    the compared atoms); worst |d dE/dlambda| in kJ/mol; relative energy."""
    F = res["F"] if idx is None else res["F"][idx]
    Fr = ref["F"]
    per = np.sqrt(((F - Fr) ** 2).sum(axis=1))
    rms = np.sqrt((Fr ** 2).sum(axis=1).mean())
    out = dict(
        Frel=float(np.sqrt(((F - Fr) ** 2).sum() / (Fr ** 2).sum())),
        Fmax=float(per.max() / rms), Fmax_atom=int(per.argmax()),
        dEdl=float(np.abs(res["dEdl"] - ref["dEdl"]).max()) if len(ref["dEdl"]) else 0.0,
    )
    if ref.get("E") is not None:
        out["Erel"] = abs(res["E"] - ref["E"]) / abs(ref["E"])
    if idx is None and "phi" in ref and ref["phi"] is not None and len(ref["phi"]) == len(res["phi"]):
        out["phi"] = float(np.abs(res["phi"] - ref["phi"]).max())
    return out
