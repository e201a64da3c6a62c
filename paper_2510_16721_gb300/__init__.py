"""Python binding of the CFNEB CUDA library (include/cfneb.h).

Argument marshalling only: every function forwards to the C entry point of
the same name in ``libcfneb.so``, which runs every step of the path in its
own sm_103a kernels.  Importing this package on a machine whose library
cannot be loaded raises; there is no CPU fallback.

Arrays are numpy float64 (host).  ``stream`` may be an integer cudaStream_t
handle, an object with a ``cuda_stream`` attribute (torch.cuda.Stream) or
None for the legacy default stream.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libcfneb.so")

OK = 0
NOT_CONVERGED = 1
ERR_INVALID_ARG = -1
ERR_SHAPE_MISMATCH = -2
ERR_OUT_OF_MEMORY = -3
ERR_HBM_BUDGET = -4
ERR_CUDA = -5
ERR_NONFINITE = -6
ERR_NOT_SPD = -7
ERR_NBR_OVERFLOW = -8
ERR_TIMEOUT = -9
ERR_STATE = -10

LJ = 0
TERSOFF = 1
NEP = 2
NEP_N_WEIGHTS = 261
ROTFREE_B = 0
DEFGRAD_D = 1
CELL_FACTOR_J = -1.0
FP64 = 0
MIXED = 1

# C entry points declared in include/cfneb.h
EXPORTS = [
    "cfneb_default_options", "cfneb_create_band", "cfneb_step", "cfneb_relax",
    "cfneb_insert_image", "cfneb_delete_image", "cfneb_get_path", "cfneb_get_state",
    "cfneb_set_state", "cfneb_get_image_scalars", "cfneb_get_tuning",
    "cfneb_shard_enable", "cfneb_shard_evaluate", "cfneb_shard_get_image", "cfneb_shard_set_ghost",
    "cfneb_shard_project", "cfneb_shard_move",
    "cfneb_destroy_band", "cfneb_evaluate", "cfneb_profile", "cfneb_profile_read",
    "cfneb_kernel_count", "cfneb_kernel_name", "cfneb_launches_per_step",
    "cfneb_status_string", "cfneb_get_work", "cfneb_get_list_stats", "cfneb_lj_evaluate_noalloc",
    "cfneb_band_bytes", "cfneb_batch_create", "cfneb_batch_add", "cfneb_batch_remove",
    "cfneb_batch_step", "cfneb_batch_relax", "cfneb_batch_status", "cfneb_batch_bytes",
    "cfneb_batch_profile", "cfneb_batch_profile_read", "cfneb_batch_destroy",
    "cfneb_autotune", "cfneb_batch_autotune", "cfneb_server_create", "cfneb_server_submit",
    "cfneb_server_run", "cfneb_server_result", "cfneb_server_stats", "cfneb_server_destroy",
]


class CfnebError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        super().__init__("%s: %s (%d)" % (where, status_string(status), status))


class Structure(ctypes.Structure):
    _fields_ = [("n_atoms", ctypes.c_int32), ("types", ctypes.POINTER(ctypes.c_int32)),
                ("positions", ctypes.POINTER(ctypes.c_double)), ("cell", ctypes.c_double * 9)]


class Potential(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("eps", ctypes.c_double), ("sigma", ctypes.c_double),
                ("rc", ctypes.c_double), ("shift_energy", ctypes.c_int32),
                ("tersoff", ctypes.c_double * 11),
                ("nep_weights", ctypes.POINTER(ctypes.c_double)), ("nep_rc", ctypes.c_double)]


class CellFilter(ctypes.Structure):
    _fields_ = [("enabled", ctypes.c_int32), ("variant", ctypes.c_int32),
                ("cell_factor", ctypes.c_double), ("pressure", ctypes.c_double)]


class Options(ctypes.Structure):
    _fields_ = [("k_spring", ctypes.c_double), ("climb", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("dt", ctypes.c_double),
                ("dt_max", ctypes.c_double), ("maxstep", ctypes.c_double),
                ("interior_noise", ctypes.POINTER(ctypes.c_double)),
                ("adaptive", ctypes.c_int32), ("n_min", ctypes.c_int32),
                ("n_max", ctypes.c_int32), ("k_ref", ctypes.c_int32),
                ("cooldown", ctypes.c_int32), ("alpha_ins", ctypes.c_double),
                ("alpha_del", ctypes.c_double), ("bin_scale", ctypes.c_double),
                ("skin", ctypes.c_double)]


_lib = None


def lib():
    """Load libcfneb.so (raises if it is missing: build it with build())."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError("libcfneb.so not built: run paper_2510_16721_gb300.build()")
        L = ctypes.CDLL(LIB_PATH)
        P = ctypes.POINTER
        vp, i32, i64, dbl = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
        dp = P(ctypes.c_double)
        sig = {
            "cfneb_default_options": ([P(Options)], ctypes.c_int),
            "cfneb_create_band": ([P(Structure), P(Structure), i32, P(Potential), P(CellFilter),
                                   P(Options), vp, P(vp)], ctypes.c_int),
            "cfneb_step": ([vp, i32], ctypes.c_int),
            "cfneb_relax": ([vp, dbl, i64, P(i64), P(i32)], ctypes.c_int),
            "cfneb_insert_image": ([vp, i32], ctypes.c_int),
            "cfneb_delete_image": ([vp, i32], ctypes.c_int),
            "cfneb_get_path": ([vp, P(i32), dp, dp, dp, dp], ctypes.c_int),
            "cfneb_get_state": ([vp, dp, dp, dp, dp, dp, P(i32)], ctypes.c_int),
            "cfneb_set_state": ([vp, dp], ctypes.c_int),
            "cfneb_get_image_scalars": ([vp, dp, dp, dp], ctypes.c_int),
            "cfneb_get_tuning": ([vp, dp, P(i32)], ctypes.c_int),
            "cfneb_shard_enable": ([vp], ctypes.c_int),
            "cfneb_shard_evaluate": ([vp, dp], ctypes.c_int),
            "cfneb_shard_get_image": ([vp, i32, dp, dp], ctypes.c_int),
            "cfneb_shard_set_ghost": ([vp, i32, dp, dbl], ctypes.c_int),
            "cfneb_shard_project": ([vp, i32, dp], ctypes.c_int),
            "cfneb_shard_move": ([vp, dp], ctypes.c_int),
            "cfneb_destroy_band": ([vp], ctypes.c_int),
            "cfneb_evaluate": ([P(Structure), i32, P(Potential), i32, vp, dp, dp, dp],
                               ctypes.c_int),
            "cfneb_profile": ([vp, i32], ctypes.c_int),
            "cfneb_profile_read": ([vp, i32, dp, P(i64)], ctypes.c_int),
            "cfneb_kernel_count": ([], ctypes.c_int32),
            "cfneb_kernel_name": ([i32], ctypes.c_char_p),
            "cfneb_launches_per_step": ([vp, P(i32)], ctypes.c_int),
            "cfneb_status_string": ([ctypes.c_int], ctypes.c_char_p),
            "cfneb_get_work": ([vp, dp, dp], ctypes.c_int),
            "cfneb_get_list_stats": ([vp, P(i64), P(i64), dp], ctypes.c_int),
            "cfneb_lj_evaluate_noalloc": ([vp, i32, dp, dbl, dbl, dbl, i32, vp, vp, vp, vp],
                                          ctypes.c_int),
            "cfneb_band_bytes": ([vp, P(ctypes.c_uint64)], ctypes.c_int),
            "cfneb_batch_create": ([i32, ctypes.c_uint64, vp, P(vp)], ctypes.c_int),
            "cfneb_batch_add": ([vp, vp], ctypes.c_int),
            "cfneb_batch_remove": ([vp, vp], ctypes.c_int),
            "cfneb_batch_step": ([vp, i32], ctypes.c_int),
            "cfneb_batch_relax": ([vp, dbl, i64, P(i32)], ctypes.c_int),
            "cfneb_batch_status": ([vp, P(i32), P(i64), P(i32), dp, P(i32)], ctypes.c_int),
            "cfneb_batch_bytes": ([vp, P(ctypes.c_uint64), P(ctypes.c_uint64)], ctypes.c_int),
            "cfneb_batch_profile": ([vp, i32], ctypes.c_int),
            "cfneb_batch_profile_read": ([vp, i32, dp, P(i64)], ctypes.c_int),
            "cfneb_batch_destroy": ([vp], ctypes.c_int),
            "cfneb_autotune": ([vp, i32, dp], ctypes.c_int),
            "cfneb_batch_autotune": ([vp, i32], ctypes.c_int),
            "cfneb_server_create": ([i32, ctypes.c_uint64, vp, P(vp)], ctypes.c_int),
            "cfneb_server_submit": ([vp, P(Structure), P(Structure), i32, P(Potential),
                                     P(CellFilter), P(Options), dbl, i64, dbl, P(i64)],
                                    ctypes.c_int),
            "cfneb_server_run": ([vp, dbl], ctypes.c_int),
            "cfneb_server_result": ([vp, i64, P(i32), dp, P(i64), P(i32), dp, P(i32)],
                                    ctypes.c_int),
            "cfneb_server_stats": ([vp, dp, dp, P(i64), dp], ctypes.c_int),
            "cfneb_server_destroy": ([vp], ctypes.c_int),
        }
        for name, (args, res) in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _lib = L
    return _lib


def build(force=False):
    """Compile the CUDA sources (sm_103a) into libcfneb.so in this package."""
    from . import _build
    return _build.build(force=force)


def status_string(status):
    return lib().cfneb_status_string(int(status)).decode()


def _check(st, where, allow=(OK,)):
    if st not in allow:
        raise CfnebError(st, where)
    return st


def _stream_handle(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(getattr(stream, "cuda_stream"))


def _dptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if a is not None else None


def make_structure(R, h, keep):
    R = np.ascontiguousarray(R, dtype=np.float64).reshape(-1, 3)
    h = np.ascontiguousarray(h, dtype=np.float64).reshape(3, 3)
    keep.append(R)
    s = Structure()
    s.n_atoms = R.shape[0]
    s.types = None
    s.positions = _dptr(R)
    for k in range(9):
        s.cell[k] = h.flat[k]
    return s


def lj_potential(eps=1.0, sigma=1.0, rc=2.5, shift=True):
    p = Potential()
    p.kind, p.eps, p.sigma, p.rc, p.shift_energy = LJ, eps, sigma, rc, int(bool(shift))
    return p


def nep_potential(weights, rc=2.1):
    """NEP-style descriptor + network potential (cfneb.h): weights in the
    order cR, cA, W0, b0, w1, b1 (NEP_N_WEIGHTS doubles), cutoff rc."""
    w = np.ascontiguousarray(weights, dtype=np.float64).ravel()
    if w.size != NEP_N_WEIGHTS:
        raise ValueError("expected %d weights, got %d" % (NEP_N_WEIGHTS, w.size))
    p = Potential()
    p.kind = NEP
    p.nep_weights = _dptr(w)
    p.nep_rc = float(rc)
    p._keep = w  # the array the pointer refers to lives as long as p
    return p


def tersoff_potential(params=None):
    """params: 11 numbers (A, B, lambda1, lambda2, beta, n, c, d, h, R, D) or
    None for Tersoff's 1988 carbon set."""
    p = Potential()
    p.kind = TERSOFF
    if params is not None:
        for k, v in enumerate(params):
            p.tersoff[k] = v
    return p


def default_options():
    o = Options()
    _check(lib().cfneb_default_options(ctypes.byref(o)), "cfneb_default_options")
    return o


class Band:
    """A band owned by the library (wraps cfneb_band*)."""

    def __init__(self, handle, n_atoms, n_max):
        self._h = ctypes.c_void_p(handle)
        self.n_atoms = n_atoms
        self.n_max = n_max

    @property
    def handle(self):
        return self._h

    def step(self, n_steps=1):
        return _check(lib().cfneb_step(self._h, int(n_steps)), "cfneb_step")

    def relax(self, fmax, max_steps):
        done = ctypes.c_int64(0)
        conv = ctypes.c_int32(0)
        st = lib().cfneb_relax(self._h, float(fmax), int(max_steps), ctypes.byref(done),
                               ctypes.byref(conv))
        _check(st, "cfneb_relax", allow=(OK, NOT_CONVERGED))
        return int(done.value), bool(conv.value)

    def insert_image(self, after_index):
        return _check(lib().cfneb_insert_image(self._h, int(after_index)), "cfneb_insert_image")

    def delete_image(self, index):
        return _check(lib().cfneb_delete_image(self._h, int(index)), "cfneb_delete_image")

    @property
    def n_images(self):
        N = ctypes.c_int32(0)
        _check(lib().cfneb_get_path(self._h, ctypes.byref(N), None, None, None, None),
               "cfneb_get_path")
        return int(N.value)

    def get_path(self):
        N = self.n_images
        R = np.zeros((N, self.n_atoms, 3))
        H = np.zeros((N, 3, 3))
        E = np.zeros(N)
        fmax = ctypes.c_double(0.0)
        Nn = ctypes.c_int32(0)
        _check(lib().cfneb_get_path(self._h, ctypes.byref(Nn), _dptr(R), _dptr(H), _dptr(E),
                                    ctypes.byref(fmax)), "cfneb_get_path")
        return dict(positions=R, cells=H, energies=E, fmax=float(fmax.value))

    def get_state(self):
        N = self.n_images
        rows = self.n_atoms + 3
        X = np.zeros((N, rows, 3))
        F = np.zeros((N, rows, 3))
        Fn = np.zeros((N, rows, 3))
        V = np.zeros((N, 3, 3))
        fire = np.zeros(4)
        ci = ctypes.c_int32(-1)
        _check(lib().cfneb_get_state(self._h, _dptr(X), _dptr(F), _dptr(Fn), _dptr(V),
                                     _dptr(fire), ctypes.byref(ci)), "cfneb_get_state")
        return dict(X=X, F=F, Fneb=Fn, virials=V, dt=fire[0], alpha=fire[1], n_pos=int(fire[2]),
                    steps=int(fire[3]), ci=int(ci.value))

    def set_state(self, X):
        """cfneb_set_state: every image's generalised coordinates from X
        (N x (n+3) x 3); FIRE reset, endpoints evaluated again."""
        X = np.ascontiguousarray(X, dtype=np.float64)
        if X.shape != (self.n_images, self.n_atoms + 3, 3):
            raise ValueError("X must have shape (N, n+3, 3)")
        _check(lib().cfneb_set_state(self._h, _dptr(X)), "cfneb_set_state")

    # -- image-range shard (paper_2510_16721_gb300.sharded drives these) --
    def shard_enable(self):
        _check(lib().cfneb_shard_enable(self._h), "cfneb_shard_enable")

    def shard_evaluate(self):
        E = np.zeros(self.n_images)
        _check(lib().cfneb_shard_evaluate(self._h, _dptr(E)), "cfneb_shard_evaluate")
        return E

    def shard_get_image(self, index):
        X = np.zeros((self.n_atoms + 3, 3))
        e = ctypes.c_double(0.0)
        _check(lib().cfneb_shard_get_image(self._h, int(index), _dptr(X), ctypes.byref(e)),
               "cfneb_shard_get_image")
        return X, float(e.value)

    def shard_set_ghost(self, side, X, energy):
        X = np.ascontiguousarray(X, dtype=np.float64)
        _check(lib().cfneb_shard_set_ghost(self._h, int(side), _dptr(X), float(energy)),
               "cfneb_shard_set_ghost")

    def shard_project(self, climbing_index):
        sums = np.zeros(4)
        _check(lib().cfneb_shard_project(self._h, int(climbing_index), _dptr(sums)),
               "cfneb_shard_project")
        return sums

    def shard_move(self, sums):
        sums = np.ascontiguousarray(sums, dtype=np.float64)
        _check(lib().cfneb_shard_move(self._h, _dptr(sums)), "cfneb_shard_move")

    def tuning(self):
        """cfneb_get_tuning: (bin width / list cutoff, force kernel blocks per SM)."""
        sc, mb = ctypes.c_double(0.0), ctypes.c_int32(0)
        _check(lib().cfneb_get_tuning(self._h, ctypes.byref(sc), ctypes.byref(mb)),
               "cfneb_get_tuning")
        return float(sc.value), int(mb.value)

    def image_scalars(self):
        """cfneb_get_image_scalars: step energies (N), the ten dots (N x 10)
        and the f_NEB coefficients (N x 2) of the last step."""
        N = self.n_images
        E = np.zeros(N)
        dots = np.zeros((N, 10))
        coef = np.zeros((N, 2))
        _check(lib().cfneb_get_image_scalars(self._h, _dptr(E), _dptr(dots), _dptr(coef)),
               "cfneb_get_image_scalars")
        return dict(E=E, dots=dots, coef=coef)

    def profile(self, enable=True):
        return _check(lib().cfneb_profile(self._h, int(bool(enable))), "cfneb_profile")

    def profile_read(self):
        out = {}
        for k in range(lib().cfneb_kernel_count()):
            ms = ctypes.c_double(0.0)
            cnt = ctypes.c_int64(0)
            _check(lib().cfneb_profile_read(self._h, k, ctypes.byref(ms), ctypes.byref(cnt)),
                   "cfneb_profile_read")
            out[lib().cfneb_kernel_name(k).decode()] = (float(ms.value), int(cnt.value))
        return out

    def get_work(self):
        p = ctypes.c_double(0.0)
        t = ctypes.c_double(0.0)
        _check(lib().cfneb_get_work(self._h, ctypes.byref(p), ctypes.byref(t)), "cfneb_get_work")
        return float(p.value), float(t.value)

    def list_stats(self):
        """cfneb_get_list_stats: (cell-list builds, evaluations, skin)."""
        nb, ne, sk = ctypes.c_int64(0), ctypes.c_int64(0), ctypes.c_double(0.0)
        _check(lib().cfneb_get_list_stats(self._h, ctypes.byref(nb), ctypes.byref(ne),
                                          ctypes.byref(sk)), "cfneb_get_list_stats")
        return int(nb.value), int(ne.value), float(sk.value)

    def autotune(self, steps=5):
        """cfneb_autotune: returns the chosen bin width / list cutoff."""
        best = ctypes.c_double(0.0)
        _check(lib().cfneb_autotune(self._h, int(steps), ctypes.byref(best)), "cfneb_autotune")
        return float(best.value)

    def bytes(self):
        b = ctypes.c_uint64(0)
        _check(lib().cfneb_band_bytes(self._h, ctypes.byref(b)), "cfneb_band_bytes")
        return int(b.value)

    def launches_per_step(self):
        n = ctypes.c_int32(0)
        _check(lib().cfneb_launches_per_step(self._h, ctypes.byref(n)), "cfneb_launches_per_step")
        return int(n.value)

    def destroy(self):
        if self._h is not None and self._h.value:
            _check(lib().cfneb_destroy_band(self._h), "cfneb_destroy_band")
            self._h = ctypes.c_void_p(0)

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def create_band(initial, final, n_images, potential, cell_filter=None, options=None,
                stream=None, noise=None):
    """cfneb_create_band.  initial/final: (R, h) pairs; noise: interior
    displacements (n_images-2, n, 3) or None."""
    keep = []
    A = make_structure(initial[0], initial[1], keep)
    B = make_structure(final[0], final[1], keep)
    opt = options if options is not None else default_options()
    if noise is not None:
        nz = np.ascontiguousarray(noise, dtype=np.float64)
        keep.append(nz)
        opt.interior_noise = _dptr(nz)
    cf = cell_filter if cell_filter is not None else CellFilter(1, ROTFREE_B, 0.0, 0.0)
    h = ctypes.c_void_p(0)
    st = lib().cfneb_create_band(ctypes.byref(A), ctypes.byref(B), int(n_images),
                                 ctypes.byref(potential), ctypes.byref(cf), ctypes.byref(opt),
                                 _stream_handle(stream), ctypes.byref(h))
    opt.interior_noise = None
    _check(st, "cfneb_create_band")
    n_max = max(int(n_images), int(opt.n_max))
    return Band(h.value, A.n_atoms, n_max)


class Batch:
    """Many bands stepped together (wraps cfneb_batch*); does not own them."""

    def __init__(self, precision=FP64, budget_bytes=0, stream=None):
        h = ctypes.c_void_p(0)
        _check(lib().cfneb_batch_create(int(precision), int(budget_bytes),
                                        _stream_handle(stream), ctypes.byref(h)),
               "cfneb_batch_create")
        self._h = h
        self.members = []

    def add(self, band):
        st = lib().cfneb_batch_add(self._h, band.handle)
        _check(st, "cfneb_batch_add")
        self.members.append(band)
        return st

    def try_add(self, band):
        """Add if the budget allows; returns True on success."""
        st = lib().cfneb_batch_add(self._h, band.handle)
        if st == ERR_HBM_BUDGET:
            return False
        _check(st, "cfneb_batch_add")
        self.members.append(band)
        return True

    def remove(self, band):
        _check(lib().cfneb_batch_remove(self._h, band.handle), "cfneb_batch_remove")
        self.members.remove(band)

    def step(self, n_steps=1):
        return _check(lib().cfneb_batch_step(self._h, int(n_steps)), "cfneb_batch_step")

    def relax(self, fmax, max_steps):
        nc = ctypes.c_int32(0)
        st = lib().cfneb_batch_relax(self._h, float(fmax), int(max_steps), ctypes.byref(nc))
        _check(st, "cfneb_batch_relax", allow=(OK, NOT_CONVERGED))
        return int(nc.value)

    def status(self):
        n = len(self.members)
        steps = (ctypes.c_int64 * max(n, 1))()
        conv = (ctypes.c_int32 * max(n, 1))()
        fm = np.zeros(max(n, 1))
        stt = (ctypes.c_int32 * max(n, 1))()
        cnt = ctypes.c_int32(0)
        _check(lib().cfneb_batch_status(self._h, ctypes.byref(cnt), steps, conv, _dptr(fm), stt),
               "cfneb_batch_status")
        return [dict(steps=int(steps[i]), converged=bool(conv[i]), fmax=float(fm[i]),
                     status=int(stt[i])) for i in range(cnt.value)]

    def autotune(self, steps=5):
        return _check(lib().cfneb_batch_autotune(self._h, int(steps)), "cfneb_batch_autotune")

    def bytes(self):
        u = ctypes.c_uint64(0)
        b = ctypes.c_uint64(0)
        _check(lib().cfneb_batch_bytes(self._h, ctypes.byref(u), ctypes.byref(b)),
               "cfneb_batch_bytes")
        return int(u.value), int(b.value)

    def profile(self, enable=True):
        return _check(lib().cfneb_batch_profile(self._h, int(bool(enable))), "cfneb_batch_profile")

    def profile_read(self):
        out = {}
        for k in range(lib().cfneb_kernel_count()):
            ms = ctypes.c_double(0.0)
            cnt = ctypes.c_int64(0)
            _check(lib().cfneb_batch_profile_read(self._h, k, ctypes.byref(ms),
                                                  ctypes.byref(cnt)), "cfneb_batch_profile_read")
            out[lib().cfneb_kernel_name(k).decode()] = (float(ms.value), int(cnt.value))
        return out

    def destroy(self):
        if self._h is not None and self._h.value:
            _check(lib().cfneb_batch_destroy(self._h), "cfneb_batch_destroy")
            self._h = ctypes.c_void_p(0)
            self.members = []

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


class Server:
    """Continuous-batching request loop (wraps cfneb_server*)."""

    def __init__(self, precision=FP64, budget_bytes=0, stream=None):
        h = ctypes.c_void_p(0)
        _check(lib().cfneb_server_create(int(precision), int(budget_bytes),
                                         _stream_handle(stream), ctypes.byref(h)),
               "cfneb_server_create")
        self._h = h

    def submit(self, initial, final, n_images, potential, cell_filter, options, fmax, max_steps,
               arrival_s):
        keep = []
        A = make_structure(initial[0], initial[1], keep)
        B = make_structure(final[0], final[1], keep)
        rid = ctypes.c_int64(-1)
        _check(lib().cfneb_server_submit(self._h, ctypes.byref(A), ctypes.byref(B),
                                         int(n_images), ctypes.byref(potential),
                                         ctypes.byref(cell_filter), ctypes.byref(options),
                                         float(fmax), int(max_steps), float(arrival_s),
                                         ctypes.byref(rid)), "cfneb_server_submit")
        return int(rid.value)

    def run(self, until_s):
        st = lib().cfneb_server_run(self._h, float(until_s))
        _check(st, "cfneb_server_run", allow=(OK, NOT_CONVERGED))
        return st == OK

    def result(self, rid):
        state, conv, stt = ctypes.c_int32(0), ctypes.c_int32(0), ctypes.c_int32(0)
        lat, bar = ctypes.c_double(0.0), ctypes.c_double(0.0)
        steps = ctypes.c_int64(0)
        _check(lib().cfneb_server_result(self._h, int(rid), ctypes.byref(state),
                                         ctypes.byref(lat), ctypes.byref(steps),
                                         ctypes.byref(conv), ctypes.byref(bar),
                                         ctypes.byref(stt)), "cfneb_server_result")
        return dict(state=int(state.value), latency_s=float(lat.value), steps=int(steps.value),
                    converged=bool(conv.value), barrier=float(bar.value),
                    status=int(stt.value))

    def stats(self):
        p50, p99, thr = ctypes.c_double(0.0), ctypes.c_double(0.0), ctypes.c_double(0.0)
        n = ctypes.c_int64(0)
        _check(lib().cfneb_server_stats(self._h, ctypes.byref(p50), ctypes.byref(p99),
                                        ctypes.byref(n), ctypes.byref(thr)),
               "cfneb_server_stats")
        return dict(p50_s=float(p50.value), p99_s=float(p99.value), retired=int(n.value),
                    atom_steps_per_s=float(thr.value))

    def destroy(self):
        if self._h is not None and self._h.value:
            _check(lib().cfneb_server_destroy(self._h), "cfneb_server_destroy")
            self._h = ctypes.c_void_p(0)

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


NOALLOC_MAX_ATOMS = 32768


def lj_evaluate_noalloc(d_positions, n_atoms, cell, eps, sigma, rc, shift_energy, d_energy,
                        d_forces, d_virial, stream=None):
    """cfneb_lj_evaluate_noalloc: device pointers (ints) in and out, host cell."""
    c = np.ascontiguousarray(cell, dtype=np.float64).reshape(9)
    return lib().cfneb_lj_evaluate_noalloc(d_positions, int(n_atoms), _dptr(c), float(eps),
                                           float(sigma), float(rc), int(shift_energy),
                                           d_energy, d_forces, d_virial,
                                           _stream_handle(stream))


def evaluate(structures, potential, precision=FP64, stream=None):
    """cfneb_evaluate over a list of (R, h): returns (E[count], list of F, V[count,3,3])."""
    keep = []
    arr = (Structure * len(structures))()
    sizes = []
    for k, (R, h) in enumerate(structures):
        arr[k] = make_structure(R, h, keep)
        sizes.append(arr[k].n_atoms)
    E = np.zeros(len(structures))
    F = np.zeros((sum(sizes), 3))
    V = np.zeros((len(structures), 3, 3))
    _check(lib().cfneb_evaluate(arr, len(structures), ctypes.byref(potential), int(precision),
                                _stream_handle(stream), _dptr(E), _dptr(F), _dptr(V)),
           "cfneb_evaluate")
    out, o = [], 0
    for n in sizes:
        out.append(F[o:o + n])
        o += n
    return E, out, V
