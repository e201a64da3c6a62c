"""Seeded synthetic inputs for CFNEB workloads.

This module builds crystal structures and random draws only: lattices,
vacancies, tilings, strains, seeded Gaussian displacements and request
streams.  It holds none of the method's arithmetic (no cell filter, no
interpolation, no forces) and serves the CUDA library, the oracle, the tests
and the benchmark alike.

Structures are (R, h): Cartesian positions (n, 3) and the lattice matrix h
with the lattice vectors as rows.  All generators are deterministic for a
given seed.
"""
import itertools
import json
import math
import os

import numpy as np

_DATA = os.path.join(os.path.dirname(os.path.abspath(__file__)), "data")

# ---------------------------------------------------------------------------
# Lennard-Jones FCC
# ---------------------------------------------------------------------------

FCC_BASIS = np.array([[0.0, 0.0, 0.0], [0.5, 0.5, 0.0], [0.5, 0.0, 0.5], [0.0, 0.5, 0.5]])
LJ_A = 1.5496  # FCC lattice constant (sigma units) used by the LJ workloads


def _lattice(basis, a, n1, n2, n3):
    """Cubic supercell: cells in (i, j, k) order, basis sites within each."""
    ijk = np.array(list(itertools.product(range(n1), range(n2), range(n3))), dtype=np.float64)
    R = ((ijk[:, None, :] + basis[None, :, :]) * a).reshape(-1, 3)
    h = np.diag([n1 * a, n2 * a, n3 * a]).astype(np.float64)
    return R, h


def fcc(a, n1, n2, n3):
    """Conventional FCC supercell n1 x n2 x n3 (4 atoms per cell)."""
    return _lattice(FCC_BASIS, a, n1, n2, n3)


def _nearest_neighbour(R, h, i, exclude=()):
    """Index of the atom nearest to atom i (minimum image; ties: lowest
    index).  Used only to pick which atom hops."""
    hinv = np.linalg.inv(h)
    ds = (R - R[i]) @ hinv
    ds -= np.round(ds)
    d = np.linalg.norm(ds @ h, axis=1)
    d[i] = np.inf
    for e in exclude:
        d[e] = np.inf
    m = d.min()
    return int(np.flatnonzero(np.isclose(d, m, rtol=0, atol=1e-9))[0])


def lj_vacancy_hop(a=LJ_A, reps=(2, 2, 2), divacancy=False):
    """Vacancy hop in FCC: atom 0 is removed; in the final state its nearest
    neighbour (lowest index) sits on the vacant site.  With ``divacancy`` a
    second neighbour of site 0 is removed too and the next neighbour hops.

    Returns (R0, h, R1, h) with matched atom order.
    """
    R, h = fcc(a, *reps)
    site = R[0].copy()
    removed = [0]
    if divacancy:
        removed.append(_nearest_neighbour(R, h, 0))
    hop = _nearest_neighbour(R, h, 0, exclude=removed)
    keep = [i for i in range(len(R)) if i not in removed]
    R0 = R[keep].copy()
    R1 = R0.copy()
    R1[keep.index(hop)] = site
    return R0, h.copy(), R1, h.copy()


# cubic diamond: FCC sites plus the same sites shifted by (1/4, 1/4, 1/4)
DIAMOND_BASIS = np.vstack([FCC_BASIS, FCC_BASIS + 0.25])
DIAMOND_A = 3.5656  # cubic diamond lattice constant (Angstrom), Tersoff C workloads


def diamond(a, n1, n2, n3):
    """Conventional cubic-diamond supercell n1 x n2 x n3 (8 atoms per cell)."""
    return _lattice(DIAMOND_BASIS, a, n1, n2, n3)


def diamond_vacancy_hop(a=DIAMOND_A, reps=(2, 2, 2)):
    """Vacancy hop in cubic diamond: atom 0 is removed and, in the final
    state, its nearest neighbour (lowest index) sits on the vacant site.
    Unrelaxed lattice sites.  Returns (R0, h, R1, h) with matched order."""
    R, h = diamond(a, *reps)
    site = R[0].copy()
    hop = _nearest_neighbour(R, h, 0)
    keep = list(range(1, len(R)))
    R0 = R[keep].copy()
    R1 = R0.copy()
    R1[keep.index(hop)] = site
    return R0, h.copy(), R1, h.copy()


def diamond_vacancy_hop_relaxed(reps=(4, 4, 4)):
    """Vacancy hop in cubic diamond (Tersoff carbon) between relaxed
    endpoints, in an n1 x n2 x n3 conventional supercell (each n >= 4).

    The displacement field of both endpoints, relaxed around the vacancy in
    a 4 x 4 x 4 cell by oracle/make_diamond_vacancy_endpoints.py, is placed
    around site 0 of the supercell: every atom within the 4 x 4 x 4 box
    centred on the vacancy (boundary included) takes the stored displacement
    of its site, atoms farther out stay on their ideal sites.  At 4 x 4 x 4
    the endpoints are the stored relaxed ones.  Atom order: the supercell's
    sites in lattice order without site 0; the hopping atom is the nearest
    neighbour the stored hop names.  Returns (R0, h, R1, h).
    """
    with open(os.path.join(_DATA, "tersoff_c_diamond_vacancy_4x4x4.json")) as f:
        d = json.load(f)
    a = d["a"]
    small = np.array(d["reps"]) * 4  # box side in units of a/4
    half = small // 2
    off_s = np.array(d["offset"])
    key = lambda u: tuple(int(x) for x in (np.asarray(u) + half) % small - half)
    field = {key(u): (np.array(p0), np.array(p1))
             for u, p0, p1 in zip(off_s, d["d0"], d["d1"])}
    hop_key = key(off_s[d["hop"]])
    R, h = diamond(a, *reps)
    if any(r < s // 4 for r, s in zip(reps, small)):
        raise ValueError("supercell smaller than the stored relaxed cell")
    site = R[0]
    s = (R - site) @ np.linalg.inv(h)
    s -= np.round(s)
    off = np.rint(s @ h / (a / 4.0)).astype(int)
    off = off[1:]
    R0 = R[1:].copy()
    R1 = R0.copy()
    hop = None
    for m in np.flatnonzero(np.all(np.abs(off) <= half, axis=1)):
        ku = key(off[m])
        d0, d1 = field[ku]
        R0[m] += d0
        if ku == hop_key and hop is None:
            hop = m
            R1[m] = site + d1
        else:
            R1[m] += d1
    if hop is None:
        raise ValueError("hopping atom not found")
    return R0, h.copy(), R1, h.copy()


def strained_cell(h, seed, amplitude=0.02):
    """h (I + eps) with eps symmetric, entries uniform in [-amplitude, amplitude]."""
    rng = np.random.default_rng(seed)
    e = rng.uniform(-amplitude, amplitude, size=(3, 3))
    e = np.triu(e) + np.triu(e, 1).T
    return h @ (np.eye(3) + e)


def affine(R, h_from, h_to):
    """Positions carried along by a change of cell (same fractional coords)."""
    return (R @ np.linalg.inv(h_from)) @ h_to


# ---------------------------------------------------------------------------
# Carbon: AB graphite and hexagonal diamond in one orthohexagonal setting
# ---------------------------------------------------------------------------

# in-plane fractional sites of a honeycomb layer in the (a, sqrt(3) a) cell
_ALPHA = [(0.0, 0.0), (0.5, 0.5)]
_BETA = [(0.5, 1.0 / 6.0), (0.0, 2.0 / 3.0)]
_LAYER_A = [(0.0, 0.0), (0.5, 1.0 / 6.0), (0.5, 0.5), (0.0, 2.0 / 3.0)]
_LAYER_B = [(0.5, 1.0 / 6.0), (0.0, 1.0 / 3.0), (0.0, 2.0 / 3.0), (0.5, 5.0 / 6.0)]


def _is_alpha(xy):
    return any(abs(xy[0] - p[0]) < 1e-9 and abs(xy[1] - p[1]) < 1e-9 for p in _ALPHA)


def graphite_hexdiamond_cells(a_g=2.46, c_g=6.70, a_d=2.52, c_d=4.12, delta=1.0 / 16.0):
    """8-atom orthohexagonal cells of AB graphite and hexagonal diamond with
    matched atom order.

    Graphite: layer A at z=0, layer B at z=1/2 (Bernal stacking).  Diamond
    target of each atom: layer-A atoms keep their in-plane site; layer-B atoms
    slide by (0, 1/3) (one bond length along the armchair direction) into
    A registry; every layer buckles by +-delta (alpha sites up in the lower
    layer, down in the upper one), which closes the interlayer bonds of
    lonsdaleite.  Returns (s_g, h_g, s_d, h_d) with fractional coordinates.
    """
    s_g, s_d = [], []
    for (x, y) in _LAYER_A:
        s_g.append((x, y, 0.0))
        s_d.append((x, y, delta if _is_alpha((x, y)) else -delta))
    for (x, y) in _LAYER_B:
        s_g.append((x, y, 0.5))
        t = (x, (y + 1.0 / 3.0) % 1.0)
        t = (t[0], 0.0 if abs(t[1] - 1.0) < 1e-12 else t[1])
        s_d.append((t[0], t[1], 0.5 - delta if _is_alpha(t) else 0.5 + delta))
    h_g = np.diag([a_g, math.sqrt(3.0) * a_g, c_g])
    h_d = np.diag([a_d, math.sqrt(3.0) * a_d, c_d])
    return np.array(s_g), h_g, np.array(s_d), h_d


def tile(R, h, reps):
    """Replicate a periodic structure reps = (n1, n2, n3) times."""
    n1, n2, n3 = reps
    ijk = np.array(list(itertools.product(range(n1), range(n2), range(n3))), dtype=np.float64)
    shift = ijk[:, 0:1] * h[0] + ijk[:, 1:2] * h[1] + ijk[:, 2:3] * h[2]
    out = (R[None, :, :] + shift[:, None, :]).reshape(-1, 3)
    return out, np.array([h[0] * n1, h[1] * n2, h[2] * n3])


def tersoff_endpoint_cells():
    """Relaxed 8-atom graphite and hexagonal-diamond cells (Tersoff 1988 C).

    Stored in data/tersoff_c_endpoints_8atom.json; the file is written by
    oracle/make_tersoff_endpoints.py, which relaxes the cells built by
    graphite_hexdiamond_cells() with the FP64 CPU reference.
    Returns (R_g, h_g, R_d, h_d).
    """
    with open(os.path.join(_DATA, "tersoff_c_endpoints_8atom.json")) as f:
        d = json.load(f)
    return (np.array(d["R_graphite"]), np.array(d["h_graphite"]),
            np.array(d["R_hexdiamond"]), np.array(d["h_hexdiamond"]))


def unwrap_cell(R_init, h_init, R_final, h_final):
    """Final positions of a matched cell (same atom order), each shifted by
    the lattice vector of the final cell that brings its fractional
    coordinate nearest to the initial one, within the cell itself."""
    s0 = np.asarray(R_init) @ np.linalg.inv(h_init)
    s1 = np.asarray(R_final) @ np.linalg.inv(h_final)
    return (s1 - np.round(s1 - s0)) @ h_final


def graphite_hexdiamond_path(reps):
    """Endpoints of the graphite -> hexagonal-diamond band at a tiling.

    The matched final cell is unwrapped against the initial one in the
    8-atom cell before both are tiled, so that every tile carries the same
    per-atom displacement.  (Unwrapping after tiling would send an atom whose
    target wrapped across the 8-atom cell boundary to the site in its own
    tile, 2.9 A through the layer, instead of the neighbouring tile's site
    1.46 A away.)"""
    Rg, hg, Rd, hd = tersoff_endpoint_cells()
    Rd = unwrap_cell(Rg, hg, Rd, hd)
    R0, h0 = tile(Rg, hg, reps)
    R1, h1 = tile(Rd, hd, reps)
    return R0, h0, R1, h1


# ---------------------------------------------------------------------------
# Random draws passed to both implementations
# ---------------------------------------------------------------------------

def interior_noise(seed, n_images, n_atoms, sigma):
    """Gaussian displacements (n_images-2, n_atoms, 3), numpy PCG64 stream."""
    rng = np.random.default_rng(seed)
    return rng.normal(0.0, sigma, size=(n_images - 2, n_atoms, 3))


# ---------------------------------------------------------------------------
# Workloads (sizes of the benchmarked configurations)
# ---------------------------------------------------------------------------

def lj_vacancy_31():
    """31-atom LJ FCC vacancy hop (2x2x2 conventional cells, a = 1.5496)."""
    return dict(name="lj_fcc_vacancy_31", potential="lj", endpoints=lj_vacancy_hop(LJ_A, (2, 2, 2)),
                n_images=7, k=1.0, climb=True, dt=0.01, fmax=1e-4, cell_filter=False,
                precision="fp64")


def tersoff_graphite_hexdiamond(reps=(6, 4, 3), n_images=9, seed=2510, jitter=0.01,
                                precision="fp64"):
    """Graphite -> hexagonal diamond, Tersoff C, cell filter on."""
    R0, h0, R1, h1 = graphite_hexdiamond_path(reps)
    n = len(R0)
    return dict(name="tersoff_graphite_hexdiamond_%d" % n, potential="tersoff",
                endpoints=(R0, h0, R1, h1), n_images=n_images, k=0.1, climb=True, dt=0.1,
                fmax=0.05, cell_filter=True, precision=precision,
                noise=interior_noise(seed, n_images, n, jitter) if jitter else None)


TERSOFF_LARGE_REPS = (32, 24, 16)  # 8 * 32 * 24 * 16 = 98,304 atoms


def near_cubic_factors(m):
    """(n1, n2, n3) with n1 n2 n3 = m, as close to cubic as possible."""
    best = None
    for n1 in range(1, int(round(m ** (1 / 3))) + 2):
        if m % n1:
            continue
        r = m // n1
        for n2 in range(n1, int(math.isqrt(r)) + 1):
            if r % n2:
                continue
            n3 = r // n2
            key = max(n1, n2, n3) - min(n1, n2, n3)
            if best is None or key < best[0]:
                best = (key, (n1, n2, n3))
    return best[1] if best else (1, 1, m)


def lj_batch(seed=4, n_bands=64, n_lo=256, n_hi=32768, img_lo=5, img_hi=15, strain=0.02):
    """Uneven LJ vacancy / divacancy bands with strained end cells."""
    rng = np.random.default_rng(seed)
    bands = []
    for b in range(n_bands):
        target = math.exp(rng.uniform(math.log(n_lo), math.log(n_hi)))
        m = max(1, int(round(target / 4.0)))
        reps = near_cubic_factors(m)
        while min(reps) < 2:  # a vacancy hop needs at least 2 cells per side
            m += 1
            reps = near_cubic_factors(m)
        div = bool(rng.integers(0, 2))
        n_images = int(rng.integers(img_lo, img_hi + 1))
        R0, h0, R1, h1 = lj_vacancy_hop(LJ_A, reps, divacancy=div)
        h1s = strained_cell(h1, seed * 1000 + b, strain)
        R1s = affine(R1, h1, h1s)
        bands.append(dict(name="lj_%s_%d" % ("divac" if div else "vac", len(R0)),
                          potential="lj", endpoints=(R0, h0, R1s, h1s), n_images=n_images,
                          k=1.0, climb=True, dt=0.01, fmax=0.05, cell_filter=True))
    return bands


def poisson_arrivals(seed, rate, window):
    """Arrival times of a Poisson process on [0, window)."""
    rng = np.random.default_rng(seed)
    t, out = 0.0, []
    while True:
        t += rng.exponential(1.0 / rate)
        if t >= window:
            return np.array(out)
        out.append(t)


def _orthohex_reps(n_target):
    """Tiling of the 8-atom orthohexagonal carbon cell with about n_target
    atoms and a near-cubic box (at least 2 cells per side)."""
    lens = (2.46, 4.26, 6.70)
    L = (n_target / 8.0 * lens[0] * lens[1] * lens[2]) ** (1.0 / 3.0)
    return tuple(max(2, int(round(L / x))) for x in lens)


def serve_requests(seed=5, rate=20.0, window=60.0, n_lo=500, n_hi=50000, img_lo=7, img_hi=16,
                   fmax=0.05, lj_strain=0.003):
    """Request stream for the serving loop: Poisson arrivals at `rate` per
    second over `window` seconds; each request is an LJ or a Tersoff carbon
    band (even odds).  LJ: FCC vacancy hop, end cell strained by up to
    lj_strain, image counts (endpoints included) uniform in [img_lo, img_hi],
    FIRE dt 0.01 with dt_max 0.03 (3 dt: the large strained bands overshoot
    into atom overlaps more often at 10 dt).
    Tersoff: cubic-diamond vacancy hop between relaxed endpoints
    (diamond_vacancy_hop_relaxed, at least 4 x 4 x 4 cells), an odd image
    count in the same range (the hop is mirror-symmetric: an odd count puts
    one image on the saddle), FIRE dt 0.05, dt_max 0.2, maxstep 0.1.  Atom
    counts log-uniform in [n_lo, n_hi].  Returns specs; build_request()
    makes the structures.
    """
    rng = np.random.default_rng(seed)
    arrivals = poisson_arrivals(seed, rate, window)
    specs = []
    for q, t in enumerate(arrivals):
        target = math.exp(rng.uniform(math.log(n_lo), math.log(n_hi)))
        n_images = int(rng.integers(img_lo, img_hi + 1))
        if rng.integers(0, 2) == 0:
            m = max(8, int(round(target / 4.0)))
            reps = near_cubic_factors(m)
            while min(reps) < 2:
                m += 1
                reps = near_cubic_factors(m)
            specs.append(dict(id=q, arrival=float(t), kind="lj_vacancy", reps=reps,
                              n_images=n_images, k=1.0, dt=0.01, dt_max=0.03, fmax=fmax,
                              strain_seed=seed * 100000 + q, strain=lj_strain))
        else:
            m = max(64, int(round(target / 8.0)))
            reps = near_cubic_factors(m)
            while min(reps) < 4:
                m += 1
                reps = near_cubic_factors(m)
            if n_images % 2 == 0:
                n_images = n_images + 1 if n_images < img_hi else n_images - 1
            specs.append(dict(id=q, arrival=float(t), kind="tersoff_diamond_vacancy", reps=reps,
                              n_images=n_images, k=0.1, dt=0.05, dt_max=0.2, maxstep=0.1,
                              fmax=fmax))
    return specs


def build_request(spec):
    """Endpoints (R0, h0, R1, h1) and potential name of a serve_requests spec."""
    if spec["kind"] == "lj_vacancy":
        R0, h0, R1, h1 = lj_vacancy_hop(LJ_A, spec["reps"])
        h1s = strained_cell(h1, spec["strain_seed"], spec["strain"])
        return (R0, h0, affine(R1, h1, h1s), h1s), "lj"
    if spec["kind"] == "tersoff_graphite_hexdiamond":
        return graphite_hexdiamond_path(spec["reps"]), "tersoff"
    if spec["kind"] == "tersoff_diamond_vacancy":
        return diamond_vacancy_hop_relaxed(spec["reps"]), "tersoff"
    return diamond_vacancy_hop(DIAMOND_A, spec["reps"]), "tersoff"


def nep_weights(seed=2510, scale=0.3):
    """Synthetic weights for the NEP-style potential (no trained model is
    available): N(0, scale^2) entries in the order the potential reads them
    (radial and angular basis coefficients, hidden-layer weights and biases,
    output weights and bias), from numpy's PCG64 with the given seed.  The
    count follows the fixed sizes K = 6, NR = 4, NA = 2, L = 4, H = 16."""
    K, NR, NA, L, H = 6, 4, 2, 4, 16
    n = NR * K + NA * K + H * (NR + NA * L) + H + H + 1
    return np.random.default_rng(seed).normal(0.0, scale, n)
