"""Oracle: plain FP64 cell-filter nudged elastic band (CFNEB).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the cpu_baseline / reference legs of ``bench.py`` may import this module; the
CUDA library never does, and the two share no code.

Every function restates one step of the method, in the paper's notation, with
numpy primitives (matrix products, ``eigh``) as the only library steps:

* potentials -- brute-force FP64 energies, forces and virials (Sec. II.B),
  in ``potentials.c``;
* cell filter -- deformation gradient D = h0^-1 h, R~ = R D^-1, rotation-free
  lattice coordinate B = D D^T and the conjugate forces F D^T and
  D^-T V D^-1 (Sec. II.C);
* NEB -- f_NEB = f_real(perp) + f_spring (Sec. II.A) with the improved (upwind)
  tangent and the climbing image that Sec. I cites;
* FIRE -- the optimiser (Sec. III relies on standard optimisers of the
  host package without naming one);
* adaptive refinement -- images inserted or removed from the spacing of the
  images in configuration space after NEB iterations (Sec. III).

Readings where the paper is silent or garbled:

1. f^{ij} = dU_i/dr^{ij} - dU_j/dr^{ji} (derivation of Eq. V2).
2. The rotation-free lattice force carries a factor 1/2:
   Phi = 1/2 D^-T V_sym D^-1.  The chain of equalities in Sec. II.C calls
   1/2 (D dD^T + dD D^T) "dB", but dB = D dD^T + dD D^T; with the 1/2 the
   generalised force is the exact negative gradient of E (pinned by finite
   differences in the tests).  ``paper_factor=True`` drops the 1/2.
3. h0 is the cell of the initial endpoint, shared by every image.
4. D is recovered from B as the symmetric positive square root.
5. The lattice coordinate is scaled: X_lat = c B, F_lat = Phi / c,
   c = number of atoms unless given; c = "J" selects J = Omega0^(1/3) n^(1/6)
   (the scale of the generalized solid-state NEB, Omega0 the initial cell's
   volume), which keeps the lattice rows' stiffness per unit of X at that of
   the atom rows for any n.
6. B is stored as 9 entries (a symmetric 3x3 block of 3 "atoms").
7. The virial is symmetrised in the rotation-free filter.
8. Tangent: Henkelman-Jonsson upwind rule (exact ties fall to the energy
   weighted branch); if both energy weights vanish the tangent is the sum of
   the two neighbour differences.
9. Spring k (|X_{i+1}-X_i| - |X_i-X_{i-1}|) tau^; climbing image = argmax E
   of the interior images (lowest index on ties), chosen at every step.
10. The image count includes both endpoints.
11. FIRE (Bitzek et al. 2006) with band-global power, N_min=5, f_inc=1.1,
    f_dec=0.5, alpha0=0.1, f_alpha=0.99, unit masses, per-row step clamp.
12. fmax = the largest row norm of f_NEB over moving images (atom rows and the
    three lattice rows).
13. Refinement every K_ref steps after a cooldown: insert the midpoint of the
    longest segment if it exceeds alpha_ins times the mean, else delete the
    interior non-climbing image with the smallest sum of adjacent segments if
    that sum is below alpha_del times the mean; at most one change, FIRE reset.
16. External pressure enters as H = U + P Omega, V_eff = V - P Omega I.
"""
import numpy as np

from . import _native

# ---------------------------------------------------------------------------
# Potentials (Sec. II.B)
# ---------------------------------------------------------------------------

# Tersoff, Phys. Rev. Lett. 61, 2879 (1988), carbon; lambda3 = 0.
TERSOFF_C1988 = dict(A=1393.6, B=346.74, lambda1=3.4879, lambda2=2.2119, beta=1.5724e-7,
                     n=0.72751, c=38049.0, d=4.3484, h=-0.57058, R=1.95, D=0.15)
_TERSOFF_ORDER = ("A", "B", "lambda1", "lambda2", "beta", "n", "c", "d", "h", "R", "D")


class LJ:
    """phi(r) = 4 eps [(sigma/r)^12 - (sigma/r)^6] (- phi(rc) if shift)."""

    def __init__(self, eps=1.0, sigma=1.0, rc=2.5, shift=True):
        self.eps, self.sigma, self.rc, self.shift = eps, sigma, rc, bool(shift)

    def evaluate(self, R, h):
        """Per-atom energies, forces (n,3), virial (3,3) by brute force."""
        return _native.lj(R, h, self.eps, self.sigma, self.rc, self.shift)

    def forces_sampled(self, R, h, idx):
        return _native.lj_sampled(R, h, self.eps, self.sigma, self.rc, idx)


class Tersoff:
    """Tersoff 1988 three-body bond-order potential (lambda3 = 0)."""

    def __init__(self, params=None):
        p = dict(TERSOFF_C1988)
        if params:
            p.update(params)
        self.params = p
        self._vec = np.array([p[k] for k in _TERSOFF_ORDER], dtype=np.float64)
        self.rc = p["R"] + p["D"]

    def evaluate(self, R, h):
        return _native.tersoff(R, h, self._vec)

    def forces_sampled(self, R, h, idx):
        return _native.tersoff_sampled(R, h, self._vec, idx)


def energy_forces_virial(pot, R, h):
    """Total energy U = sum_i U_i, forces F (n,3), virial V (3,3)."""
    e, F, V = pot.evaluate(R, h)
    return float(np.sum(e)), e, F, V


# ---------------------------------------------------------------------------
# Cell filter (Sec. II.C)
# ---------------------------------------------------------------------------

ROTFREE_B = 0   # generalised lattice coordinate B = D D^T (default)
DEFGRAD_D = 1   # generalised lattice coordinate D itself


class NotSPD(ValueError):
    pass


def sym_sqrt(B):
    """Symmetric positive square root of a symmetric 3x3 matrix (eigh)."""
    B = 0.5 * (B + B.T)
    w, Q = np.linalg.eigh(B)
    if np.any(w <= 0.0):
        raise NotSPD("B is not positive definite: eigenvalues %r" % (w,))
    return (Q * np.sqrt(w)) @ Q.T


def to_generalized(R, h, h0, c, variant=ROTFREE_B):
    """Generalised coordinates of one structure: (n+3, 3) array.

    s = R h^-1, D = h0^-1 h, R~ = s h0 = R D^-1; lattice rows c B (B = D D^T)
    or c D (deformation-gradient variant).
    """
    R = np.asarray(R, dtype=np.float64)
    s = R @ np.linalg.inv(h)
    Rt = s @ h0
    D = np.linalg.inv(h0) @ h
    lat = D @ D.T if variant == ROTFREE_B else D
    return np.vstack([Rt, c * lat])


def from_generalized(X, h0, c, variant=ROTFREE_B):
    """Map generalised coordinates back to Cartesian positions and cell.

    Returns (R, h, D) with D = sqrt(B) (rotation-free) or D = X_lat / c,
    h = h0 D, R = R~ D.
    """
    n = X.shape[0] - 3
    lat = X[n:] / c
    D = sym_sqrt(lat) if variant == ROTFREE_B else lat.copy()
    h = h0 @ D
    R = X[:n] @ D
    return R, h, D


def generalized_force(F, V, D, c, variant=ROTFREE_B, paper_factor=False):
    """Conjugate generalised forces: atom rows F D^T, lattice rows

    rotation-free: (1/c) * 1/2 * D^-T V_sym D^-1  (paper_factor: without 1/2)
    deformation gradient: (1/c) * D^-T V
    """
    Dinv = np.linalg.inv(D)
    Fat = F @ D.T
    if variant == ROTFREE_B:
        Vs = 0.5 * (V + V.T)
        Phi = Dinv.T @ Vs @ Dinv
        if not paper_factor:
            Phi = 0.5 * Phi
    else:
        Phi = Dinv.T @ V
    return np.vstack([Fat, Phi / c])


class AtomicImage:
    """Energy and generalised force of one image of an atomic band."""

    def __init__(self, pot, h0, c, cell_filter=True, variant=ROTFREE_B, pressure=0.0,
                 paper_factor=False):
        self.pot, self.h0, self.c = pot, np.asarray(h0, dtype=np.float64), float(c)
        self.cell_filter, self.variant = bool(cell_filter), variant
        self.pressure, self.paper_factor = float(pressure), paper_factor

    def __call__(self, X):
        """X (n+3, 3) -> (E, F_gen (n+3, 3), info dict)."""
        R, h, D = from_generalized(X, self.h0, self.c, self.variant)
        U, e, F, V = energy_forces_virial(self.pot, R, h)
        omega = abs(np.linalg.det(h))
        E = U
        if self.pressure != 0.0:
            E = U + self.pressure * omega
            V = V - self.pressure * omega * np.eye(3)
        if self.cell_filter:
            Fg = generalized_force(F, V, D, self.c, self.variant, self.paper_factor)
        else:
            Fg = np.vstack([F @ D.T, np.zeros((3, 3))])
        return E, Fg, dict(R=R, h=h, D=D, V=V, U=U)


# ---------------------------------------------------------------------------
# NEB (Sec. II.A) with the upwind tangent and climbing image (Sec. I)
# ---------------------------------------------------------------------------

def upwind_tangent(Xm, X0, Xp, Em, E0, Ep):
    """Henkelman-Jonsson improved tangent (unnormalised)."""
    tp = Xp - X0
    tm = X0 - Xm
    if Ep > E0 > Em:
        return tp
    if Ep < E0 < Em:
        return tm
    dmax = max(abs(Ep - E0), abs(Em - E0))
    dmin = min(abs(Ep - E0), abs(Em - E0))
    if dmax == 0.0:
        return tp + tm
    if Ep > Em:
        return tp * dmax + tm * dmin
    return tp * dmin + tm * dmax


def climbing_index(E):
    """argmax of E over the interior images (lowest index on ties)."""
    inner = np.asarray(E[1:-1])
    return 1 + int(np.argmax(inner))


def neb_forces(X, E, F, k, climb, ci=None):
    """f_NEB for the interior images.  X, F: (N, d); E: (N,).  ``ci``, when
    given, names the climbing image instead of the argmax of E (a range of
    a band whose climbing image lies elsewhere passes -1)."""
    N = X.shape[0]
    out = np.zeros_like(X)
    if ci is None:
        ci = climbing_index(E) if climb else -1
    for i in range(1, N - 1):
        tau = upwind_tangent(X[i - 1], X[i], X[i + 1], E[i - 1], E[i], E[i + 1])
        that = tau / np.linalg.norm(tau)
        fpar = float(np.dot(F[i], that))
        if i == ci:
            out[i] = F[i] - 2.0 * fpar * that
        else:
            spring = k * (np.linalg.norm(X[i + 1] - X[i]) - np.linalg.norm(X[i] - X[i - 1]))
            out[i] = F[i] - fpar * that + spring * that
    return out, ci


# ---------------------------------------------------------------------------
# FIRE (Bitzek, Koskinen, Gahler, Moseler, Gumbsch, PRL 97, 170201 (2006))
# ---------------------------------------------------------------------------

class Fire:
    def __init__(self, dt=0.1, dt_max=None, maxstep=0.2, n_min=5, f_inc=1.1, f_dec=0.5,
                 alpha0=0.1, f_alpha=0.99, row_dim=3, global_clamp=False):
        self.dt0 = dt
        self.dt_max = 10.0 * dt if dt_max is None else dt_max
        self.maxstep, self.n_min, self.f_inc, self.f_dec = maxstep, n_min, f_inc, f_dec
        self.alpha0, self.f_alpha, self.row_dim = alpha0, f_alpha, row_dim
        self.global_clamp = global_clamp
        self.reset(None)

    def reset(self, shape):
        self.v = None if shape is None else np.zeros(shape)
        self.dt, self.alpha, self.n_pos = self.dt0, self.alpha0, 0
        self.fresh = True

    def step(self, F, sums=None):
        """One FIRE move for the stacked vector F (moving images only).

        Returns the displacement dX.  Velocity mixing uses band-global
        quantities P = F.v, |F|^2, |v|^2; ``sums`` = (P, |F|^2, |v|^2), when
        given, are those of the whole band (F and v here being a part of it).
        """
        if self.v is None or self.v.shape != F.shape:
            self.v = np.zeros_like(F)
            self.fresh = True
        if not self.fresh:
            P = float(np.sum(F * self.v)) if sums is None else float(sums[0])
            if P > 0.0:
                fn = np.sqrt(float(np.sum(F * F)) if sums is None else float(sums[1]))
                vn = np.sqrt(float(np.sum(self.v * self.v)) if sums is None else float(sums[2]))
                if fn > 0.0:
                    self.v = (1.0 - self.alpha) * self.v + self.alpha * vn * F / fn
                if self.n_pos > self.n_min:
                    self.dt = min(self.dt * self.f_inc, self.dt_max)
                    self.alpha *= self.f_alpha
                self.n_pos += 1
            else:
                self.v = np.zeros_like(F)
                self.alpha = self.alpha0
                self.dt *= self.f_dec
                self.n_pos = 0
        self.fresh = False
        self.v = self.v + self.dt * F
        dX = self.dt * self.v
        if self.global_clamp:
            nrm = np.sqrt(float(np.sum(dX * dX)))
            if nrm > self.maxstep:
                dX = dX * (self.maxstep / nrm)
        else:
            rows = dX.reshape(-1, self.row_dim)
            nr = np.sqrt(np.sum(rows * rows, axis=1))
            scale = np.where(nr > self.maxstep, self.maxstep / np.where(nr > 0, nr, 1.0), 1.0)
            dX = (rows * scale[:, None]).reshape(dX.shape)
        return dX


def row_fmax(Fneb_interior, row_dim=3):
    rows = np.asarray(Fneb_interior).reshape(-1, row_dim)
    return float(np.sqrt(np.max(np.sum(rows * rows, axis=1)))) if rows.size else 0.0


# ---------------------------------------------------------------------------
# Band: interpolation, step, relax, adaptive refinement (Sec. III)
# ---------------------------------------------------------------------------

class Band:
    """A chain of N images X[0..N-1] (endpoints fixed) relaxed by NEB + FIRE.

    ``image_fn(X_img) -> (E, F_gen, info)`` gives the energy and generalised
    force of one image; X_img has shape ``shape`` (e.g. (n+3, 3)).
    """

    def __init__(self, X, image_fn, k=0.1, climb=True, fire=None, row_dim=3,
                 adaptive=False, n_min=3, n_max=64, k_ref=10, cooldown=20,
                 alpha_ins=1.5, alpha_del=0.5):
        self.X = [np.array(x, dtype=np.float64) for x in X]
        self.shape = self.X[0].shape
        self.image_fn, self.k, self.climb, self.row_dim = image_fn, k, climb, row_dim
        self.fire = fire if fire is not None else Fire(row_dim=row_dim)
        self.adaptive, self.n_min, self.n_max = adaptive, n_min, n_max
        self.k_ref, self.cooldown = k_ref, cooldown
        self.alpha_ins, self.alpha_del = alpha_ins, alpha_del
        self.E = [None] * len(self.X)
        self.F = [None] * len(self.X)
        self.info = [None] * len(self.X)
        for i in (0, len(self.X) - 1):
            self._evaluate(i)
        self.steps = 0
        self.last_change = 0
        self.fmax = np.inf
        self.ci = -1
        self.fneb = None
        self.events = []

    @property
    def N(self):
        return len(self.X)

    def _evaluate(self, i):
        E, Fg, info = self.image_fn(self.X[i])
        self.E[i], self.F[i], self.info[i] = float(E), np.asarray(Fg, dtype=np.float64), info

    def compute(self):
        """Energies/forces of the interior images, f_NEB and fmax."""
        for i in range(1, self.N - 1):
            self._evaluate(i)
        Xs = np.array([x.ravel() for x in self.X])
        Fs = np.array([f.ravel() for f in self.F])
        Fneb, self.ci = neb_forces(Xs, np.array(self.E), Fs, self.k, self.climb)
        self.fneb = Fneb[1:-1]
        self.fmax = row_fmax(self.fneb, self.row_dim)
        return self.fmax

    def update(self):
        """FIRE move of the interior images with the current f_NEB."""
        dX = self.fire.step(self.fneb)
        for i in range(1, self.N - 1):
            self.X[i] = self.X[i] + dX[i - 1].reshape(self.shape)
        self.steps += 1
        if (self.adaptive and self.steps % self.k_ref == 0
                and self.steps - self.last_change >= self.cooldown):
            self.refine()

    def step(self, n=1):
        for _ in range(n):
            self.compute()
            self.update()

    def relax(self, fmax, max_steps):
        """Iterate until fmax < tolerance; returns (steps_done, converged)."""
        start = self.steps
        while self.steps - start < max_steps:
            if self.compute() < fmax:
                return self.steps - start, True
            self.update()
        return self.steps - start, self.compute() < fmax

    # -- adaptive refinement -------------------------------------------------
    def spacings(self):
        return np.array([np.linalg.norm(self.X[i + 1] - self.X[i]) for i in range(self.N - 1)])

    def insert_image(self, after):
        """Insert the linear midpoint between images after and after+1."""
        if after < 0 or after >= self.N - 1:
            raise IndexError("insert position out of range")
        Xm = 0.5 * (self.X[after] + self.X[after + 1])
        self.X.insert(after + 1, Xm)
        self.E.insert(after + 1, None)
        self.F.insert(after + 1, None)
        self.info.insert(after + 1, None)
        self.fire.reset(None)

    def delete_image(self, index):
        """Remove interior image ``index`` (endpoints cannot be removed)."""
        if index <= 0 or index >= self.N - 1:
            raise IndexError("only interior images can be deleted")
        for lst in (self.X, self.E, self.F, self.info):
            del lst[index]
        self.fire.reset(None)

    def refine(self):
        """One adaptive check: at most one insertion or deletion."""
        ell = self.spacings()
        mean = float(np.mean(ell))
        s = int(np.argmax(ell))
        if ell[s] > self.alpha_ins * mean and self.N < self.n_max:
            self.insert_image(s)
            self.last_change = self.steps
            self.events.append(("insert", self.steps, s))
            return "insert"
        if self.N > self.n_min:
            best, best_j = None, -1
            for j in range(1, self.N - 1):
                if self.climb and j == self.ci:
                    continue
                pair = ell[j - 1] + ell[j]
                if best is None or pair < best:
                    best, best_j = pair, j
            if best is not None and best < self.alpha_del * mean:
                self.delete_image(best_j)
                self.last_change = self.steps
                self.events.append(("delete", self.steps, best_j))
                return "delete"
        return None

    def barrier(self):
        return max(self.E) - self.E[0]


def interpolate(X0, X1, n_images, noise=None):
    """Linear interpolation of the generalised coordinates; ``noise``
    ((n_images-2, n, 3) or None) is added to the interior atom rows."""
    X = []
    for k in range(n_images):
        t = k / (n_images - 1)
        X.append(X0 + t * (X1 - X0))
    if noise is not None:
        n = X0.shape[0] - 3
        for k in range(1, n_images - 1):
            X[k] = X[k].copy()
            X[k][:n] += noise[k - 1]
    return X


def unwrap_final(R_init, h_init, R_final, h_final):
    """Shift each final atom by a lattice vector so that its fractional
    coordinate is the nearest to the initial one."""
    s0 = np.asarray(R_init) @ np.linalg.inv(h_init)
    s1 = np.asarray(R_final) @ np.linalg.inv(h_final)
    s1 = s1 - np.round(s1 - s0)
    return s1 @ h_final


def make_band(pot, R0, h0, R1, h1, n_images, k=0.1, climb=True, cell_filter=True,
              variant=ROTFREE_B, c=None, pressure=0.0, fire=None, noise=None, **kw):
    """Set up an atomic CFNEB band between two endpoints (h0 is the reference)."""
    R0 = np.asarray(R0, dtype=np.float64)
    h0 = np.asarray(h0, dtype=np.float64)
    h1 = np.asarray(h1, dtype=np.float64)
    R1 = unwrap_final(R0, h0, R1, h1)
    n = R0.shape[0]
    if c == "J":  # J = Omega0^(1/3) n^(1/6) (generalized solid-state NEB scale)
        c = abs(np.linalg.det(h0)) ** (1.0 / 3.0) * n ** (1.0 / 6.0)
    c = float(n) if c is None or c <= 0 else float(c)
    if not cell_filter:
        h1 = h0
    X0 = to_generalized(R0, h0, h0, c, variant)
    X1 = to_generalized(R1, h1, h0, c, variant)
    img = AtomicImage(pot, h0, c, cell_filter, variant, pressure)
    X = interpolate(X0, X1, n_images, noise)
    return Band(X, img, k=k, climb=climb, fire=fire, row_dim=3, **kw)


def relax_single(image_fn, X, fmax, max_steps, fire=None):
    """Relax one structure in generalised coordinates (endpoint relaxation)."""
    fire = fire if fire is not None else Fire()
    X = np.array(X, dtype=np.float64)
    for step in range(max_steps):
        E, Fg, _ = image_fn(X)
        f = row_fmax(Fg)
        if f < fmax:
            return X, E, step, True
        X = X + fire.step(Fg.ravel()).reshape(X.shape)
    E, Fg, _ = image_fn(X)
    return X, E, max_steps, row_fmax(Fg) < fmax
