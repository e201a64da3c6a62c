"""Shared test cases: the same seeded inputs handed to the oracle and to the
CUDA library through its C ABI."""
import numpy as np

import cfneb_inputs as ci


def perturbed(R, h, seed, amp, shear=0.0):
    rng = np.random.default_rng(seed)
    R = R + rng.normal(0.0, amp, R.shape)
    if shear:
        e = np.eye(3)
        e[0, 1] += shear
        e[2, 0] -= 0.5 * shear
        s = R @ np.linalg.inv(h)
        h = h @ e
        R = s @ h
    return R, h


def lj_structures():
    out = {}
    R, h, _, _ = ci.lj_vacancy_hop()
    out["vacancy31"] = perturbed(R, h, 1, 0.03)
    R, h = ci.fcc(ci.LJ_A, 1, 1, 1)
    out["one_cell"] = perturbed(R, h, 3, 0.04, shear=0.05)
    R, h = ci.fcc(ci.LJ_A, 3, 4, 5)
    out["triclinic240"] = perturbed(R, h, 2, 0.05, shear=0.07)
    R, h = ci.fcc(ci.LJ_A, 9, 9, 9)
    out["fcc2916"] = perturbed(R, h, 4, 0.02, shear=0.01)
    return out


def tersoff_structures():
    out = {}
    Rg, hg, Rd, hd = ci.tersoff_endpoint_cells()
    out["graphite8"] = perturbed(Rg, hg, 7, 0.05, shear=0.03)
    hm = 0.5 * (hg + hd)
    hm[2, 2] = 0.5 * (hg[2, 2] + hd[2, 2]) * 0.72
    sm = 0.5 * (Rg @ np.linalg.inv(hg) + Rd @ np.linalg.inv(hd))
    out["midpath8"] = perturbed(sm @ hm, hm, 8, 0.05, shear=0.03)
    R, h = ci.tile(sm @ hm, hm, (6, 4, 3))
    out["midpath576"] = perturbed(R, h, 9, 0.04, shear=0.01)
    R, h = ci.tile(Rd, hd, (5, 3, 4))
    out["hexdiamond480"] = perturbed(R, h, 10, 0.06)
    return out


def f32_structure(R, h):
    """Positions rounded to FP32 (the mixed path stores coordinates in FP32;
    the oracle is then evaluated at exactly the stored configuration)."""
    return np.asarray(R, dtype=np.float32).astype(np.float64), h


def lj_band_case(n_images=7, strain_seed=None):
    R0, h0, R1, h1 = ci.lj_vacancy_hop()
    if strain_seed is not None:
        h1s = ci.strained_cell(h1, strain_seed, 0.02)
        R1 = ci.affine(R1, h1, h1s)
        h1 = h1s
    return R0, h0, R1, h1


def gpu_band(g, R0, h0, R1, h1, n_images, potential, k, dt, maxstep=0.2, climb=True,
             cell_filter=True, precision=0, noise=None, dt_max=None, adaptive=False, n_min=3,
             n_max=None, variant=0, pressure=0.0, bin_scale=0.0, alpha_ins=1.5, alpha_del=0.5,
             skin=None, cell_factor=0.0):
    opt = g.default_options()
    if skin is not None:
        opt.skin = skin
    opt.k_spring = k
    opt.climb = int(climb)
    opt.precision = precision
    opt.dt = dt
    opt.dt_max = 10 * dt if dt_max is None else dt_max
    opt.maxstep = maxstep
    opt.adaptive = int(adaptive)
    opt.n_min = n_min
    opt.n_max = n_images if n_max is None else n_max
    opt.bin_scale = bin_scale
    opt.alpha_ins = alpha_ins
    opt.alpha_del = alpha_del
    cf = g.CellFilter(int(cell_filter), variant, cell_factor, pressure)
    return g.create_band((R0, h0), (R1, h1), n_images, potential, cf, opt, noise=noise)


def oracle_band(o, pot, R0, h0, R1, h1, n_images, k, dt, maxstep=0.2, climb=True,
                cell_filter=True, noise=None, dt_max=None, adaptive=False, n_min=3, n_max=None,
                variant=0, pressure=0.0, alpha_ins=1.5, alpha_del=0.5, c=None):
    fire = o.Fire(dt=dt, dt_max=10 * dt if dt_max is None else dt_max, maxstep=maxstep)
    return o.make_band(pot, R0, h0, R1, h1, n_images, k=k, climb=climb, c=c,
                       cell_filter=cell_filter, fire=fire, noise=noise, adaptive=adaptive,
                       n_min=n_min, n_max=n_images if n_max is None else n_max,
                       variant=variant, pressure=pressure, alpha_ins=alpha_ins,
                       alpha_del=alpha_del)
