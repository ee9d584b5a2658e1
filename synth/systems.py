"""Seeded synthetic constant-pH test systems.

Random numbers come from SplitMix64 (Steele, Lea & Flood, OOPSLA 2014) used as
a counter-based generator: draw i of stream s under seed k is
splitmix64(key(k, s) + i * 0x9E3779B97F4A7C15).  Only integer arithmetic and
correctly rounded IEEE operations (+ - * / sqrt) are used, so the same seed gives
bit-identical systems on x86 and Arm.  Positions are rounded to float32 so that
float32 and float64 callers see the same coordinates.

Workload shapes follow the paper's benchmark systems (random charges with
clustered sites, Sec. "Random Systems"; water boxes of ~1e5-1e6 atoms with
hundreds of titratable sites, Sec. "Scaling with Increasing Number of Sites").
"""
from __future__ import annotations

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

# TIP3P-like rigid water: O-H 0.09572 nm, H-O-H 104.52 deg.  The hydrogen offsets
# in the molecular frame (x: in-plane, z: bisector) are written out as decimal
# literals (computed once at 30 digits) so no libm call enters the generator.
_HX = 0.0756950327263661161743181192209
_HZ = 0.0585882276618294936567420906481
Q_O, Q_H = -0.834, 0.417

CONFIGS = {
    # 3,000 point charges, S=4 sites of 4 atoms, L=3.2 nm, d=3, p=8
    "A": dict(kind="charges", n=3000, L=3.2, n_sites=4, atoms_per_site=4, dmin=0.1,
              depth=3, order=8),
    # 32,000 waters on a jittered 32^3 lattice, L=9.86 nm, S=32, d=4, p=10
    "B": dict(kind="water", n_water=32000, grid=32, L=9.86, n_sites=32,
              waters_per_site=(2, 4), depth=4, order=10),
    # 333,334 waters (1,000,002 atoms) on a 70^3 lattice, L=21.5 nm, S=512, d=5, p=12
    "C": dict(kind="water", n_water=333334, grid=70, L=21.5, n_sites=512,
              waters_per_site=(2, 4), depth=5, order=12),
    # 66,667 waters (200,001 atoms) at C's density, L=12.57 nm, S=128, d=4, p=12
    # (the differentiation workload)
    "D": dict(kind="water", n_water=66667, grid=41, L=12.57, n_sites=128,
              waters_per_site=(2, 4), depth=4, order=12),
    # profiler case: a quarter of C's waters (250,002 atoms) in the same box and
    # tree, S=128; the M2L, M2M and L2L work is identical to C's
    "C_quarter": dict(kind="water", n_water=83334, grid=70, L=21.5, n_sites=128,
                      waters_per_site=(2, 4), depth=5, order=12),
}


def splitmix64(z: np.ndarray) -> np.ndarray:
    """SplitMix64 output function applied elementwise to uint64 counters."""
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = z + _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def _key(seed: int, stream: int) -> np.uint64:
    k = splitmix64(np.array([seed], dtype=np.uint64))[0]
    return splitmix64(np.array([k ^ np.uint64(stream * 0x632BE59BD9B4E019 % (1 << 64))],
                               dtype=np.uint64))[0]


def bits(seed: int, stream: int, n: int, offset: int = 0) -> np.ndarray:
    ctr = np.arange(offset, offset + n, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return splitmix64(_key(seed, stream) + ctr * _GOLDEN)


def uniform01(seed: int, stream: int, n: int, offset: int = 0) -> np.ndarray:
    """Doubles in [0, 1) with 53 random bits."""
    return (bits(seed, stream, n, offset) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def _uniform(seed, stream, n, lo, hi, offset=0):
    return lo + (hi - lo) * uniform01(seed, stream, n, offset)


def _to_f32_box(x: np.ndarray, L: float) -> np.ndarray:
    x = np.mod(x, L)
    x = x.astype(np.float32).astype(np.float64)
    x[x >= L] = 0.0
    return x


def _min_image(d: np.ndarray, L: float) -> np.ndarray:
    return d - L * np.round(d / L)


def _random_unit_quaternions(seed: int, stream: int, n: int) -> np.ndarray:
    """Uniform rotations by Marsaglia's (1972) disk method (sqrt only)."""
    out = np.zeros((n, 4))
    todo = np.arange(n)
    rnd = 0
    pts = {}
    for half in (0, 1):
        todo = np.arange(n)
        xy = np.zeros((n, 2))
        s = np.zeros(n)
        rnd = 0
        while todo.size:
            u = _uniform(seed, stream * 8 + half, 2 * n, -1.0, 1.0, offset=2 * n * rnd).reshape(n, 2)
            cand = u[todo]
            ss = (cand ** 2).sum(1)
            ok = (ss < 1.0) & (ss > 0.0)
            xy[todo[ok]] = cand[ok]
            s[todo[ok]] = ss[ok]
            todo = todo[~ok]
            rnd += 1
        pts[half] = (xy, s)
    (a, s1), (b, s2) = pts[0], pts[1]
    f = np.sqrt((1.0 - s1) / s2)
    out[:, 0] = a[:, 0]
    out[:, 1] = a[:, 1]
    out[:, 2] = b[:, 0] * f
    out[:, 3] = b[:, 1] * f
    return out


def _rotmat(qt: np.ndarray) -> np.ndarray:
    w, x, y, z = qt[:, 0], qt[:, 1], qt[:, 2], qt[:, 3]
    R = np.empty((qt.shape[0], 3, 3))
    R[:, 0, 0] = 1 - 2 * (y * y + z * z)
    R[:, 0, 1] = 2 * (x * y - w * z)
    R[:, 0, 2] = 2 * (x * z + w * y)
    R[:, 1, 0] = 2 * (x * y + w * z)
    R[:, 1, 1] = 1 - 2 * (x * x + z * z)
    R[:, 1, 2] = 2 * (y * z - w * x)
    R[:, 2, 0] = 2 * (x * z - w * y)
    R[:, 2, 1] = 2 * (y * z + w * x)
    R[:, 2, 2] = 1 - 2 * (x * x + y * y)
    return R


def _site_deltas(seed, stream, sizes, signs):
    """Per-atom charge changes U(-0.3,0.3), recentred so each site changes by signs[s] e."""
    total = int(sum(sizes))
    u = _uniform(seed, stream, total, -0.3, 0.3)
    out = []
    pos = 0
    for n, sg in zip(sizes, signs):
        d = u[pos:pos + n]
        d = d - d.mean() + sg / n
        out.append(d)
        pos += n
    return out


def make_charges(n: int, L: float, n_sites: int, atoms_per_site: int, seed: int,
                 dmin: float = 0.1, depth: int = 3, order: int = 8, name: str = "charges"):
    """Random point charges with clustered ("typical case") sites.

    Positions uniform in the periodic cube with rejection to a minimum periodic
    pair distance dmin; charges +-U(0.2,0.8) with random sign, shifted to sum to
    zero.  Each site is a random atom plus its (atoms_per_site-1) nearest periodic
    neighbours; sites are disjoint.  qB = qA + Delta with sum(Delta) = +1 e."""
    acc = np.zeros((0, 3))
    rnd = 0
    while acc.shape[0] < n:
        cand = _uniform(seed, 1, 3 * 4096, 0.0, L, offset=3 * 4096 * rnd).reshape(-1, 3)
        cand = _to_f32_box(cand, L)
        for c in cand:
            if acc.shape[0] >= n:
                break
            if acc.shape[0]:
                dd = _min_image(acc - c, L)
                if ((dd * dd).sum(1) < dmin * dmin).any():
                    continue
            acc = np.vstack([acc, c[None]])
        rnd += 1
    x = acc
    mag = _uniform(seed, 2, n, 0.2, 0.8)
    sgn = np.where(uniform01(seed, 3, n) < 0.5, -1.0, 1.0)
    q = sgn * mag
    q = q - q.mean()
    site_of = np.full(n, -1, dtype=np.int32)
    pick = uniform01(seed, 4, 64 * n_sites)
    sites = []
    k = 0
    while len(sites) < n_sites:
        c = int(pick[k] * n)
        k += 1
        if site_of[c] >= 0:
            continue
        dd = _min_image(x - x[c], L)
        r2 = (dd * dd).sum(1)
        order_ = np.argsort(r2, kind="stable")
        members = [j for j in order_ if site_of[j] < 0][:atoms_per_site]
        if c not in members:
            continue
        for j in members:
            site_of[j] = len(sites)
        sites.append(np.array(sorted(members), dtype=np.int64))
    deltas = _site_deltas(seed, 5, [len(s) for s in sites], [1.0] * n_sites)
    qA = q.copy()
    qB = q.copy()
    for s, dl in zip(sites, deltas):
        qB[s] = qA[s] + dl
    lam = uniform01(seed, 6, n_sites)
    return dict(name=name, seed=seed, L=float(L), x=x, qA=qA, qB=qB, site_of=site_of,
                lam=lam, depth=depth, order=order)


def make_water(n_water: int, grid: int, L: float, n_sites: int, seed: int,
               waters_per_site=(2, 4), depth: int = 4, order: int = 10, name: str = "water"):
    """Rigid 3-site waters (O -0.834 e, H +0.417 e) on a jittered lattice.

    n_water distinct sites of the grid^3 lattice (spacing L/grid) are chosen at
    random; each O gets a U(+-0.02 nm) jitter and each molecule a uniform random
    orientation.  A titratable site is a random water together with its nearest
    unused neighbours (waters_per_site inclusive range); its per-atom charge
    changes are recentred to a net +-1 e (random sign)."""
    if n_water > grid ** 3:
        raise ValueError("more waters than lattice sites")
    keys = bits(seed, 11, grid ** 3)
    cells = np.argsort(keys, kind="stable")[:n_water]
    ix = cells % grid
    iy = (cells // grid) % grid
    iz = cells // (grid * grid)
    h = L / grid
    O = np.stack([ix, iy, iz], 1).astype(np.float64) * h + 0.5 * h
    O = O + _uniform(seed, 12, 3 * n_water, -0.02, 0.02).reshape(-1, 3)
    R = _rotmat(_random_unit_quaternions(seed, 13, n_water))
    h1 = np.array([_HX, 0.0, _HZ])
    h2 = np.array([-_HX, 0.0, _HZ])
    H1 = O + R @ h1
    H2 = O + R @ h2
    x = np.empty((3 * n_water, 3))
    x[0::3] = O
    x[1::3] = H1
    x[2::3] = H2
    x = _to_f32_box(x, L)
    n = 3 * n_water
    q = np.empty(n)
    q[0::3] = Q_O
    q[1::3] = Q_H
    q[2::3] = Q_H
    site_of = np.full(n, -1, dtype=np.int32)
    used = np.zeros(n_water, dtype=bool)
    Ox = x[0::3]
    lo, hi = waters_per_site
    pick = uniform01(seed, 14, 64 * n_sites)
    cnt = uniform01(seed, 15, 64 * n_sites)
    sites = []
    k = 0
    while len(sites) < n_sites:
        w = int(pick[k] * n_water)
        nw = lo + int(cnt[k] * (hi - lo + 1))
        k += 1
        if used[w]:
            continue
        dd = _min_image(Ox - Ox[w], L)
        r2 = (dd * dd).sum(1)
        r2[used] = np.inf
        part = np.argpartition(r2, nw)[:nw + 1]
        part = part[np.argsort(r2[part], kind="stable")][:nw]
        if w not in part:
            continue
        used[part] = True
        atoms = np.sort(np.concatenate([3 * part, 3 * part + 1, 3 * part + 2]))
        site_of[atoms] = len(sites)
        sites.append(atoms.astype(np.int64))
    signs = np.where(uniform01(seed, 16, n_sites) < 0.5, -1.0, 1.0)
    deltas = _site_deltas(seed, 17, [len(s) for s in sites], signs)
    qA = q.copy()
    qB = q.copy()
    for s, dl in zip(sites, deltas):
        qB[s] = qA[s] + dl
    lam = uniform01(seed, 18, n_sites)
    return dict(name=name, seed=seed, L=float(L), x=x, qA=qA, qB=qB, site_of=site_of,
                lam=lam, depth=depth, order=order)


def make_e1(layout: str = "typical", forms: int = 2, seed: int = 1, L: float = 2.2, depth: int = 2, order: int = 8):
    """The paper's accuracy test system (Sec. "Random Systems"): 1,000
    background particles and 10 site particles, all charges U(-1, 1), in a
    periodic cube (edge L; the paper gives none, 2.2 nm puts the particles at
    config A's density), positions uniform with rejection to a minimum
    periodic pair distance of 0.1 nm.  The 10 site particles form one site with
    `forms` forms (2 or 4), each form its own U(-1, 1) charge set:
    layout "typical" takes a random particle and its 9 nearest periodic
    neighbours (clustered, like the atoms of one residue), "worst" 10 particles
    drawn uniformly from the whole box.  lambda = 0.345 (two forms) or
    (0.345, 0.721) (four forms), as in the paper.  Returns the multi-form
    layout (q_env, site_of, forms, lams) and, for two forms, also qA, qB, lam."""
    assert layout in ("typical", "worst") and forms in (2, 4)
    n, nsite = 1010, 10
    base = make_charges(n=n, L=L, n_sites=0, atoms_per_site=1, seed=seed, dmin=0.1, depth=depth, order=order)
    x = base["x"]
    q = _uniform(seed, 11, n, -1.0, 1.0)
    pick = uniform01(seed, 12, 4 * nsite * 16)
    if layout == "typical":
        c = int(pick[0] * n)
        dd = _min_image(x - x[c], L)
        members = np.argsort((dd * dd).sum(1), kind="stable")[:nsite]
    else:
        members, k = [], 0
        while len(members) < nsite:
            j = int(pick[k] * n)
            k += 1
            if j not in members:
                members.append(j)
        members = np.array(members)
    members = np.array(sorted(int(j) for j in members), dtype=np.int64)
    site_of = np.full(n, -1, dtype=np.int32)
    site_of[members] = 0
    fq = _uniform(seed, 13, forms * nsite, -1.0, 1.0).reshape(forms, nsite)
    lams = [np.array([0.345])] if forms == 2 else [np.array([0.345, 0.721])]
    out = dict(name=f"e1_{layout}_{forms}forms", seed=seed, L=float(L), x=x, q_env=q, site_of=site_of,
               forms=[fq], lams=lams, depth=depth, order=order)
    if forms == 2:
        qA, qB = q.copy(), q.copy()
        qA[members] = fq[0]
        qB[members] = fq[1]
        out.update(qA=qA, qB=qB, lam=lams[0].copy())
    return out


def make(config: str, seed: int = 1):
    """Build one of the named workloads ("A", "B", "C", "D", "C_quarter") for a seed."""
    c = dict(CONFIGS[config])
    kind = c.pop("kind")
    if kind == "charges":
        return make_charges(seed=seed, name=config, **c)
    return make_water(seed=seed, name=config, **c)
