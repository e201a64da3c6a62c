"""Oracle: NEP-style descriptor + neural-network site energy (single species).

TEST INFRASTRUCTURE ONLY (same callers as the rest of ``oracle/``).

The paper's examples run a neuroevolution potential (NEP, the force field of
the GPUMD package it builds on, Sec. IV); its trained weights are not
available, so this restates the NEP construction with synthetic weights
passed in by the caller.  Site energy of atom i (Sec. II.B's per-atom split):

* cutoff f_c(r) = (1 + cos(pi r / rc)) / 2 for r < rc, 0 beyond;
* radial basis f_k(r) = (T_k(x) + 1) / 2 f_c(r), x = 2 (r / rc - 1)^2 - 1,
  T_k the Chebyshev polynomials of the first kind, k < K;
* radial functions g^R_n = sum_k cR[n, k] f_k and g^A_n = sum_k cA[n, k] f_k;
* descriptors q_n = sum_j g^R_n(r_ij) (n < NR) and
  q_nl = sum_j sum_k g^A_n(r_ij) g^A_n(r_ik) P_l(cos theta_jk) (n < NA,
  1 <= l <= L, j and k over all neighbours of i within rc, j = k included),
  P_l the Legendre polynomials;
* U_i = sum_h w1[h] tanh(sum_d W0[h, d] q_d - b0[h]) - b1, descriptors
  ordered (q_0 .. q_{NR-1}, q_{0,1} .. q_{0,L}, q_{1,1} .. ).

Every derivative comes from torch autograd in FP64 on the pair vectors
r^ij = R_j + t h - R_i: P_ij = dU_i/dr^ij, F_i = sum_j (P_ij - P_ji)
(derivation of Eq. V2) and V = -sum_ij r^ij (x) P_ij.  Neighbours by brute
force over every periodic image within rc.  Pinned by finite differences of
the energy (forces, strain derivative), invariances, the spherical-harmonic
form of the angular descriptors and numpy's Chebyshev series.
"""
import math

import numpy as np

K, NR, NA, L, H = 6, 4, 2, 4, 16        # basis, radial, angular functions, l_max, hidden
ND = NR + NA * L                         # descriptors
N_WEIGHTS = NR * K + NA * K + H * ND + H + H + 1


def unpack(w):
    """Weights in the order cR (NR x K), cA (NA x K), W0 (H x ND), b0 (H),
    w1 (H), b1."""
    w = np.asarray(w, dtype=np.float64).ravel()
    if w.size != N_WEIGHTS:
        raise ValueError("expected %d weights, got %d" % (N_WEIGHTS, w.size))
    o = 0
    out = {}
    for name, shape in (("cR", (NR, K)), ("cA", (NA, K)), ("W0", (H, ND)), ("b0", (H,)),
                        ("w1", (H,)), ("b1", ())):
        size = int(np.prod(shape)) if shape else 1
        out[name] = w[o:o + size].reshape(shape) if shape else float(w[o])
        o += size
    return out


def periodic_pairs(R, h, rc):
    """Every (i, j, r^ij) with 0 < |r^ij| < rc over all periodic images."""
    R = np.asarray(R, dtype=np.float64)
    h = np.asarray(h, dtype=np.float64)
    vol = abs(np.linalg.det(h))
    widths = [vol / np.linalg.norm(np.cross(h[(a + 1) % 3], h[(a + 2) % 3])) for a in range(3)]
    m = [int(math.ceil(rc / w_)) for w_ in widths]
    I, J, D = [], [], []
    for t0 in range(-m[0], m[0] + 1):
        for t1 in range(-m[1], m[1] + 1):
            for t2 in range(-m[2], m[2] + 1):
                shift = t0 * h[0] + t1 * h[1] + t2 * h[2]
                d = R[None, :, :] + shift - R[:, None, :]
                r = np.linalg.norm(d, axis=2)
                ii, jj = np.nonzero((r < rc) & (r > 0.0))
                I.append(ii)
                J.append(jj)
                D.append(d[ii, jj])
    return np.concatenate(I), np.concatenate(J), np.concatenate(D)


def chebyshev_basis(torch, x):
    T = [torch.ones_like(x), x]
    for _ in range(2, K):
        T.append(2.0 * x * T[-1] - T[-2])
    return torch.stack(T[:K], dim=-1)


def legendre(torch, c):
    """P_1 .. P_4 of c, written out."""
    return torch.stack([c, (3 * c ** 2 - 1) / 2, (5 * c ** 3 - 3 * c) / 2,
                        (35 * c ** 4 - 30 * c ** 2 + 3) / 8], dim=-1)[..., :L]


class NEP:
    """NEP-style potential with caller-given weights (see the module text)."""

    def __init__(self, weights, rc=2.1):
        self.w = unpack(weights)
        self.rc = float(rc)

    def _site_energies(self, torch, n, I, J, d):
        p = self.w
        r = torch.sqrt((d * d).sum(dim=1))
        fc = 0.5 * (1.0 + torch.cos(math.pi * r / self.rc))
        x = 2.0 * (r / self.rc - 1.0) ** 2 - 1.0
        fk = 0.5 * (chebyshev_basis(torch, x) + 1.0) * fc[:, None]
        gR = fk @ torch.tensor(p["cR"]).T
        gA = fk @ torch.tensor(p["cA"]).T
        Ii = torch.tensor(I)
        qR = torch.zeros(n, NR, dtype=torch.float64).index_add(0, Ii, gR)
        # angular: every ordered pair (a, b) of entries with the same centre
        order = np.argsort(I, kind="stable")
        A, B = [], []
        start = 0
        counts = np.bincount(I, minlength=n)
        for i in range(n):
            idx = order[start:start + counts[i]]
            start += counts[i]
            aa, bb = np.meshgrid(idx, idx, indexing="ij")
            A.append(aa.ravel())
            B.append(bb.ravel())
        A = torch.tensor(np.concatenate(A))
        B = torch.tensor(np.concatenate(B))
        u = d / r[:, None]
        c = (u[A] * u[B]).sum(dim=1)
        Pl = legendre(torch, c)                                    # (pairs, L)
        term = (gA[A][:, :, None] * gA[B][:, :, None]) * Pl[:, None, :]   # (pairs, NA, L)
        qA = torch.zeros(n, NA, L, dtype=torch.float64).index_add(0, torch.tensor(I)[A], term)
        q = torch.cat([qR, qA.reshape(n, NA * L)], dim=1)
        hid = torch.tanh(q @ torch.tensor(p["W0"]).T - torch.tensor(p["b0"]))
        return hid @ torch.tensor(p["w1"]) - p["b1"], q

    def descriptors(self, R, h):
        import torch
        I, J, d = periodic_pairs(R, h, self.rc)
        _, q = self._site_energies(torch, len(R), I, J, torch.tensor(d))
        return q.detach().numpy()

    def evaluate(self, R, h):
        """Per-atom energies, forces (n, 3), virial (3, 3)."""
        import torch
        n = len(R)
        I, J, d = periodic_pairs(R, h, self.rc)
        dt = torch.tensor(d, requires_grad=True)
        U, _ = self._site_energies(torch, n, I, J, dt)
        (P,) = torch.autograd.grad(U.sum(), dt)
        P = P.numpy()
        F = np.zeros((n, 3))
        np.add.at(F, I, P)
        np.subtract.at(F, J, P)
        V = -(d[:, :, None] * P[:, None, :]).sum(axis=0)
        return U.detach().numpy(), F, V
