"""Python binding of libdmrg, the GB300 two-site DMRG hot path (C-ABI in include/dmrg.h).

Argument marshalling only: every step of the method runs in the CUDA library.  Device
vectors are passed as torch CUDA tensors (float64, contiguous) or raw device pointers.
Importing this package does not need a GPU; creating a context does.  The library must
have been built (``paper_1507_00161_gb300.build.build()``); there is no fallback.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libdmrg.so")

DMRG_OK = 0
DMRG_EINVAL = -1
DMRG_ENOMEM = -2
DMRG_ECUDA = -3
DMRG_ENOCONV = -4
DMRG_ETIMEOUT = -5
FP64 = 0
MIXED_FP32 = 1

EXPORTED = ["dmrg_create", "dmrg_destroy", "dmrg_last_error", "dmrg_build_blocks",
            "dmrg_psi_layout", "dmrg_heff_apply", "dmrg_davidson",
            "dmrg_truncate_renormalize", "dmrg_step", "dmrg_sweep", "dmrg_block_sectors",
            "dmrg_rdm_eigh", "dmrg_set_tuning", "dmrg_get_tuning", "dmrg_partition_terms",
            "dmrg_autotune",
            "dmrg_set_options", "dmrg_set_dbss", "dmrg_set_roots", "dmrg_dot_rdm",
            "dmrg_mutual_information",
            "dmrg_get_counters",
            "dmrg_heff_cost",
            "dmrg_heff_apply_noalloc", "dmrg_mlp_reset", "dmrg_mlp_harvest", "dmrg_mlp_train",
            "dmrg_mlp_params", "dmrg_mlp_loss_grad", "dmrg_mlp_n_params",
            "dmrg_batch_create", "dmrg_batch_destroy", "dmrg_batch_last_error",
            "dmrg_batch_sweep", "dmrg_extrapolate", "dmrg_fiedler_order"]
PRECOND_DIAG = 0
PRECOND_MLP = 1


class DmrgError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"libdmrg status {code}: {msg}")
        self.code = code


class Problem(ctypes.Structure):
    _fields_ = [("n_sites", ctypes.c_int32), ("species", ctypes.c_void_p),
                ("two_m", ctypes.c_void_p), ("eps", ctypes.c_void_p), ("n_v", ctypes.c_int64),
                ("v_idx", ctypes.c_void_p), ("v_val", ctypes.c_void_p),
                ("order", ctypes.c_void_p), ("Np", ctypes.c_int32), ("Nn", ctypes.c_int32),
                ("two_Mz", ctypes.c_int32)]


class Options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int32), ("precond", ctypes.c_int32),
                ("dav_tol", ctypes.c_double), ("dav_max_iter", ctypes.c_int32),
                ("dav_max_sub", ctypes.c_int32), ("stream", ctypes.c_void_p)]


class MpsInit(ctypes.Structure):
    _fields_ = [("n_bonds", ctypes.c_int32), ("bonds", ctypes.c_void_p),
                ("bond_ptr", ctypes.c_void_p), ("sec", ctypes.c_void_p),
                ("u_off", ctypes.c_void_p), ("u", ctypes.c_void_p)]


class DavStats(ctypes.Structure):
    _fields_ = [("n_products", ctypes.c_int32), ("converged", ctypes.c_int32),
                ("residual", ctypes.c_double), ("energy", ctypes.c_double),
                ("heff_flops", ctypes.c_double), ("heff_bytes", ctypes.c_double),
                ("seconds", ctypes.c_double), ("energy1", ctypes.c_double)]


class StepStats(ctypes.Structure):
    _fields_ = [("p", ctypes.c_int32), ("dir", ctypes.c_int32), ("n_products", ctypes.c_int32),
                ("kept", ctypes.c_int32), ("energy", ctypes.c_double),
                ("residual", ctypes.c_double), ("trunc_err", ctypes.c_double),
                ("seconds", ctypes.c_double), ("heff_seconds", ctypes.c_double),
                ("heff_flops", ctypes.c_double), ("heff_bytes", ctypes.c_double),
                ("energy1", ctypes.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class Tuning(ctypes.Structure):
    _fields_ = [("heff_big_edge", ctypes.c_int32), ("svd_cluster", ctypes.c_int32),
                ("heff_graph", ctypes.c_int32)]


class BatchStats(ctypes.Structure):
    _fields_ = [("products", ctypes.c_int64), ("heff_seconds", ctypes.c_double),
                ("launches", ctypes.c_int64)]


class Counters(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_int64), ("heff_products", ctypes.c_int64),
                ("heff_seconds", ctypes.c_double), ("heff_flops", ctypes.c_double),
                ("heff_bytes", ctypes.c_double), ("t_enlarge", ctypes.c_double),
                ("t_super", ctypes.c_double), ("t_davidson", ctypes.c_double),
                ("t_truncate", ctypes.c_double), ("t_project", ctypes.c_double),
                ("t_predict", ctypes.c_double), ("t_sync", ctypes.c_double),
                ("t_enlarge_host", ctypes.c_double), ("t_upload", ctypes.c_double),
                ("upload_bytes", ctypes.c_int64), ("sb_blocks_l", ctypes.c_int64),
                ("sb_blocks_r", ctypes.c_int64), ("sb_terms", ctypes.c_int64),
                ("sb_tiles", ctypes.c_int64), ("t_detail", ctypes.c_double * 24),
                ("pool_mallocs", ctypes.c_int64), ("sb_small_tiles", ctypes.c_int64),
                ("sb_term_hist", ctypes.c_int64 * 8),
                ("sb_kernel_flops", ctypes.c_double)]


_lib = None


def load_library(path: str = LIB_PATH):
    """Load libdmrg.so; raises if it has not been built (no fallback exists)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"libdmrg is not built ({path} missing); run "
                          "paper_1507_00161_gb300.build.build()")
    lib = ctypes.CDLL(path)
    P = ctypes.c_void_p
    i32, i64, dbl = ctypes.c_int32, ctypes.c_int64, ctypes.c_double
    sig = {
        "dmrg_create": [ctypes.POINTER(Problem), ctypes.POINTER(Options), ctypes.POINTER(P)],
        "dmrg_destroy": [P],
        "dmrg_build_blocks": [P, ctypes.POINTER(MpsInit)],
        "dmrg_psi_layout": [P, i32, P, P, P, P, P, P],
        "dmrg_heff_apply": [P, i32, P, P],
        "dmrg_heff_apply_noalloc": [P, i32, P, P],
        "dmrg_davidson": [P, i32, P, P, P, ctypes.POINTER(DavStats)],
        "dmrg_truncate_renormalize": [P, i32, i32, i32, P, P],
        "dmrg_step": [P, i32, i32, i32, ctypes.POINTER(StepStats)],
        "dmrg_sweep": [P, i32, P, P],
        "dmrg_block_sectors": [P, i32, i32, P, P, P],
        "dmrg_heff_cost": [P, i32, P, P, P],
        "dmrg_set_options": [P, ctypes.POINTER(Options)],
        "dmrg_set_dbss": [P, i32, dbl],
        "dmrg_set_roots": [P, i32],
        "dmrg_dot_rdm": [P, i32, P, P],
        "dmrg_mutual_information": [P, i32, P, P, P],
        "dmrg_rdm_eigh": [P, i32, i32, i32, P, P, P, P, P, P],
        "dmrg_set_tuning": [P, ctypes.POINTER(Tuning)],
        "dmrg_partition_terms": [P, i32, P],
        "dmrg_autotune": [P, i32, i32, P, P, P],
        "dmrg_get_tuning": [P, ctypes.POINTER(Tuning)],
        "dmrg_mlp_reset": [P, ctypes.c_uint64],
        "dmrg_mlp_harvest": [P, i32, i32],
        "dmrg_mlp_train": [P, i32, i32, dbl, ctypes.c_uint64, P, P],
        "dmrg_mlp_params": [P, i32, P, i64],
        "dmrg_mlp_loss_grad": [P, i32, P, P, P, i64, P, P],
        "dmrg_get_counters": [P, ctypes.POINTER(Counters)],
        "dmrg_extrapolate": [i32, i32, P, P, P, P],
        "dmrg_fiedler_order": [i32, P, P, P],
    }
    for name, args in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    lib.dmrg_last_error.argtypes = [P]
    lib.dmrg_last_error.restype = ctypes.c_char_p
    lib.dmrg_mlp_n_params.argtypes = []
    lib.dmrg_mlp_n_params.restype = ctypes.c_int64
    lib.dmrg_batch_create.argtypes = [i32, P, ctypes.POINTER(P)]
    lib.dmrg_batch_create.restype = ctypes.c_int
    lib.dmrg_batch_destroy.argtypes = [P]
    lib.dmrg_batch_destroy.restype = ctypes.c_int
    lib.dmrg_batch_last_error.argtypes = [P]
    lib.dmrg_batch_last_error.restype = ctypes.c_char_p
    lib.dmrg_batch_sweep.argtypes = [P, P, P, ctypes.POINTER(BatchStats)]
    lib.dmrg_batch_sweep.restype = ctypes.c_int
    _lib = lib
    return lib


def _ptr(x):
    """Device pointer of a torch tensor, or an int pointer, or None."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    return x.data_ptr()


def _np_ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None and a.size else None


FIT_POWER = 0
FIT_QUADRATIC = 1


def fiedler_order(I):
    """Chain order of the orbitals from a symmetric mutual-information matrix (host code
    in the library): (order, Fiedler vector), order[k] = orbital at chain position k."""
    lib = load_library()
    W = np.ascontiguousarray(I, dtype=np.float64)
    if W.ndim != 2 or W.shape[0] != W.shape[1]:
        raise ValueError("I must be a square matrix")
    n = W.shape[0]
    order = np.zeros(n, dtype=np.int32)
    v = np.zeros(n)
    rc = lib.dmrg_fiedler_order(int(n), _np_ptr(W), _np_ptr(order), _np_ptr(v))
    if rc != DMRG_OK:
        raise DmrgError(rc, "invalid or disconnected mutual-information matrix")
    return [int(x) for x in order], v


def extrapolate(M, E, kind=FIT_POWER):
    """Least-squares fit of energies E at kept-state counts M (host code in the library):
    FIT_POWER -> (E_inf, X1, X2, rms) of E = E_inf + X1 M^X2; FIT_QUADRATIC ->
    (c0, c1, c2, rms) of E = c0 + c1/M + c2/M^2."""
    lib = load_library()
    m = np.ascontiguousarray(M, dtype=np.float64)
    e = np.ascontiguousarray(E, dtype=np.float64)
    if m.shape != e.shape or m.ndim != 1:
        raise ValueError("M and E must be 1-D arrays of equal length")
    coef = np.zeros(3)
    rms = ctypes.c_double()
    rc = lib.dmrg_extrapolate(int(kind), int(m.shape[0]), _np_ptr(m), _np_ptr(e),
                              _np_ptr(coef), ctypes.byref(rms))
    if rc != DMRG_OK:
        why = {DMRG_EINVAL: "invalid points or kind",
               DMRG_ENOCONV: "no power-law minimum inside the exponent range"}
        raise DmrgError(rc, why.get(rc, "fit failed"))
    return float(coef[0]), float(coef[1]), float(coef[2]), rms.value


class DMRG:
    """One problem (Eq. 1 on m-scheme sites, a target sector) on the GPU."""

    def __init__(self, problem, precision=FP64, dav_tol=1e-8, dav_max_iter=100, dav_max_sub=24,
                 stream=None, precond=PRECOND_DIAG):
        self.lib = load_library()
        self._keep = dict(
            species=np.ascontiguousarray(problem.species, dtype=np.int8),
            two_m=np.ascontiguousarray(problem.two_m, dtype=np.int8),
            eps=np.ascontiguousarray(problem.eps, dtype=np.float64),
            v_idx=np.ascontiguousarray(problem.v_idx, dtype=np.int32).reshape(-1),
            v_val=np.ascontiguousarray(problem.v_val, dtype=np.float64),
            order=np.ascontiguousarray(problem.order, dtype=np.int32))
        k = self._keep
        self.n_sites = int(k["species"].shape[0])
        pr = Problem(self.n_sites, k["species"].ctypes.data, k["two_m"].ctypes.data,
                     k["eps"].ctypes.data, int(k["v_val"].shape[0]),
                     k["v_idx"].ctypes.data if k["v_idx"].size else None,
                     k["v_val"].ctypes.data if k["v_val"].size else None,
                     k["order"].ctypes.data, int(problem.Np), int(problem.Nn),
                     int(problem.two_Mz))
        opt = self._options(precision, dav_tol, dav_max_iter, dav_max_sub, stream, precond)
        h = ctypes.c_void_p()
        rc = self.lib.dmrg_create(ctypes.byref(pr), ctypes.byref(opt), ctypes.byref(h))
        self.h = h.value
        if rc != DMRG_OK:
            msg = self.lib.dmrg_last_error(self.h).decode() if self.h else "create failed"
            self.close()
            raise DmrgError(rc, msg)

    @staticmethod
    def _options(precision, dav_tol, dav_max_iter, dav_max_sub, stream, precond=PRECOND_DIAG):
        stream_ptr = None
        if stream is not None:
            stream_ptr = stream if isinstance(stream, int) else stream.cuda_stream
        return Options(int(precision), int(precond), float(dav_tol), int(dav_max_iter),
                       int(dav_max_sub), stream_ptr)

    def set_options(self, precision=FP64, dav_tol=1e-8, dav_max_iter=100, dav_max_sub=24,
                    stream=None, precond=PRECOND_DIAG):
        opt = self._options(precision, dav_tol, dav_max_iter, dav_max_sub, stream, precond)
        self._check(self.lib.dmrg_set_options(self.h, ctypes.byref(opt)))

    def set_roots(self, n_roots):
        """Target the n_roots (1 or 2) lowest states; with 2 the truncation averages
        their density matrices and the second energy is reported as energy1."""
        self._check(self.lib.dmrg_set_roots(self.h, int(n_roots)))

    def dot_rdm(self, p):
        """Two-orbital density matrix (4 x 4) of chain positions p, p+1 from the wave
        function held for p, and (s_p, s_{p+1}, s_{p,p+1}, I_{p,p+1})."""
        rho = np.zeros(16)
        ent = np.zeros(4)
        self._check(self.lib.dmrg_dot_rdm(self.h, int(p), _np_ptr(rho), _np_ptr(ent)))
        return rho.reshape(4, 4), tuple(float(x) for x in ent)

    def mutual_information(self, M):
        """All-pairs orbital mutual information from a left-to-right half sweep at M
        (dmrg_mutual_information): (I (N x N, problem sites), s (N), step records)."""
        N = self.n_sites
        I = np.zeros(N * N)
        s = np.zeros(N)
        arr = (StepStats * (N - 3))()
        self._check(self.lib.dmrg_mutual_information(self.h, int(M), _np_ptr(I), _np_ptr(s), arr))
        return I.reshape(N, N), s, [a.as_dict() for a in arr]

    def partition_terms(self, b):
        """Number of operator products across bond b of the operator partition."""
        n = ctypes.c_int32()
        self._check(self.lib.dmrg_partition_terms(self.h, int(b), ctypes.byref(n)))
        return n.value

    def autotune(self, p, reps=2):
        """Time the product's work split on the superblock at p and keep the fastest
        (dmrg_autotune): (chosen edge, {edge: best ms})."""
        ch = ctypes.c_int32()
        edges = np.zeros(5, dtype=np.int32)
        ms = np.zeros(5)
        self._check(self.lib.dmrg_autotune(self.h, int(p), int(reps), ctypes.byref(ch),
                                           _np_ptr(edges), _np_ptr(ms)))
        return ch.value, {int(e): float(t) for e, t in zip(edges, ms)}

    def tuning(self):
        t = Tuning()
        self._check(self.lib.dmrg_get_tuning(self.h, ctypes.byref(t)))
        return {"heff_big_edge": t.heff_big_edge, "svd_cluster": t.svd_cluster,
                "heff_graph": t.heff_graph}

    def set_tuning(self, heff_big_edge=None, svd_cluster=None, heff_graph=None):
        """Work split and launch mode of the kernels (dmrg_set_tuning); None keeps the
        current value."""
        cur = self.tuning()
        t = Tuning(int(cur["heff_big_edge"] if heff_big_edge is None else heff_big_edge),
                   int(cur["svd_cluster"] if svd_cluster is None else svd_cluster),
                   int(cur["heff_graph"] if heff_graph is None else heff_graph))
        self._check(self.lib.dmrg_set_tuning(self.h, ctypes.byref(t)))

    def rdm_eigh(self, p, direction, cluster=0, vectors=True):
        """Per-sector spectrum (and eigenvectors) of the reduced density matrix of the wave
        function held for p on side `direction`: a list of (qn, w, V) with w descending and
        V (d x d) holding the eigenvectors as columns (None when vectors=False)."""
        n = ctypes.c_int32()
        size = ctypes.c_int64()
        self._check(self.lib.dmrg_rdm_eigh(self.h, int(p), int(direction), int(cluster),
                                           ctypes.byref(n), ctypes.byref(size), None, None,
                                           None, None))
        qn = np.zeros((n.value, 3), dtype=np.int32)
        dims = np.zeros(n.value, dtype=np.int32)
        self._check(self.lib.dmrg_rdm_eigh(self.h, int(p), int(direction), int(cluster), None,
                                           None, _np_ptr(qn), _np_ptr(dims), None, None))
        w = np.zeros(int(dims.sum()))
        vecs = np.zeros(size.value) if vectors else np.zeros(0)
        self._check(self.lib.dmrg_rdm_eigh(self.h, int(p), int(direction), int(cluster), None,
                                           None, _np_ptr(qn), _np_ptr(dims), _np_ptr(w),
                                           _np_ptr(vecs) if vectors else None))
        out, wo, vo = [], 0, 0
        for i in range(n.value):
            d = int(dims[i])
            V = vecs[vo:vo + d * d].reshape(d, d).copy() if vectors else None
            out.append((tuple(int(x) for x in qn[i]), w[wo:wo + d].copy(), V))
            wo += d
            vo += d * d
        return out

    def set_dbss(self, m_min, trunc_target):
        """Dynamic block state selection: M passed to the truncating calls becomes the
        ceiling, m_min the floor, and each truncation keeps the fewest states whose
        discarded weight is at most trunc_target (<= 0: back to a fixed M)."""
        self._check(self.lib.dmrg_set_dbss(self.h, int(m_min), float(trunc_target)))

    def counters(self):
        c = Counters()
        self._check(self.lib.dmrg_get_counters(self.h, ctypes.byref(c)))
        return {f: (list(getattr(c, f)) if f in ("t_detail", "sb_term_hist") else getattr(c, f))
                for f, _ in Counters._fields_}

    def close(self):
        if getattr(self, "h", None):
            self.lib.dmrg_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc, allow=()):
        if rc != DMRG_OK and rc not in allow:
            raise DmrgError(rc, self.lib.dmrg_last_error(self.h).decode())
        return rc

    def build_blocks(self, init):
        bonds, bond_ptr, sec, u_off, u = init.flat() if hasattr(init, "flat") else init
        self._init_keep = [np.ascontiguousarray(a) for a in (bonds, bond_ptr, sec, u_off, u)]
        b, bp, s, uo, uu = self._init_keep
        mi = MpsInit(int(b.shape[0]), _np_ptr(b), _np_ptr(bp), _np_ptr(s), _np_ptr(uo),
                     _np_ptr(uu))
        self._check(self.lib.dmrg_build_blocks(self.h, ctypes.byref(mi)))

    def psi_layout(self, p):
        n = ctypes.c_int64()
        size = ctypes.c_int64()
        self._check(self.lib.dmrg_psi_layout(self.h, p, ctypes.byref(n), ctypes.byref(size),
                                             None, None, None, None))
        nb = n.value
        qn = np.zeros((nb, 3), dtype=np.int32)
        dl = np.zeros(nb, dtype=np.int32)
        dr = np.zeros(nb, dtype=np.int32)
        off = np.zeros(nb, dtype=np.int64)
        self._check(self.lib.dmrg_psi_layout(self.h, p, None, None, _np_ptr(qn), _np_ptr(dl),
                                             _np_ptr(dr), _np_ptr(off)))
        return dict(qn_left=qn, dl=dl, dr=dr, off=off, size=size.value)

    def heff_apply(self, p, x, y):
        self._check(self.lib.dmrg_heff_apply(self.h, p, _ptr(x), _ptr(y)))

    def heff_apply_noalloc(self, p, x, y):
        """H_eff psi through the allocation-free entry point (FP64; the superblock at p
        must have been set up by psi_layout or heff_apply first)."""
        self._check(self.lib.dmrg_heff_apply_noalloc(self.h, p, _ptr(x), _ptr(y)))

    def davidson(self, p, guess=None, out=None, allow_noconv=False):
        e = ctypes.c_double()
        st = DavStats()
        rc = self.lib.dmrg_davidson(self.h, p, _ptr(guess), _ptr(out), ctypes.byref(e),
                                    ctypes.byref(st))
        self._check(rc, allow=(DMRG_ENOCONV,) if allow_noconv else ())
        return e.value, {f: getattr(st, f) for f, _ in DavStats._fields_}

    def truncate_renormalize(self, p, direction, M):
        tr = ctypes.c_double()
        kept = ctypes.c_int32()
        self._check(self.lib.dmrg_truncate_renormalize(self.h, p, direction, M, ctypes.byref(tr),
                                                       ctypes.byref(kept)))
        return tr.value, kept.value

    def step(self, p, direction, M):
        st = StepStats()
        self._check(self.lib.dmrg_step(self.h, p, direction, M, ctypes.byref(st)))
        return st.as_dict()

    def sweep(self, M):
        n = 2 * (self.n_sites - 3)
        arr = (StepStats * n)()
        e = ctypes.c_double()
        self._check(self.lib.dmrg_sweep(self.h, M, arr, ctypes.byref(e)))
        return [a.as_dict() for a in arr], e.value

    def block_sectors(self, side, b):
        n = ctypes.c_int32()
        self._check(self.lib.dmrg_block_sectors(self.h, side, b, ctypes.byref(n), None, None))
        qn = np.zeros((n.value, 3), dtype=np.int32)
        d = np.zeros(n.value, dtype=np.int32)
        self._check(self.lib.dmrg_block_sectors(self.h, side, b, None, _np_ptr(qn), _np_ptr(d)))
        return qn, d

    # ---- learned preconditioner ----
    def mlp_reset(self, seed=1):
        self._check(self.lib.dmrg_mlp_reset(self.h, seed))

    def mlp_harvest(self, enable=True, per_iter=2048):
        self._check(self.lib.dmrg_mlp_harvest(self.h, 1 if enable else 0, per_iter))

    def mlp_train(self, epochs=20, batch=4096, lr=1e-3, seed=1):
        loss = ctypes.c_double()
        ns = ctypes.c_int64()
        self._check(self.lib.dmrg_mlp_train(self.h, epochs, batch, lr, seed, ctypes.byref(loss),
                                            ctypes.byref(ns)))
        return loss.value, ns.value

    def mlp_params(self):
        n = int(self.lib.dmrg_mlp_n_params())
        out = np.zeros(n)
        self._check(self.lib.dmrg_mlp_params(self.h, 0, _np_ptr(out), n))
        return out

    def mlp_set_params(self, theta):
        theta = np.ascontiguousarray(theta, dtype=np.float64)
        self._check(self.lib.dmrg_mlp_params(self.h, 1, _np_ptr(theta), theta.shape[0]))

    def mlp_loss_grad(self, theta, X, T, precision=FP64):
        theta = np.ascontiguousarray(theta, dtype=np.float64)
        X = np.ascontiguousarray(X, dtype=np.float64)
        T = np.ascontiguousarray(T, dtype=np.float64)
        g = np.zeros_like(theta)
        loss = ctypes.c_double()
        self._check(self.lib.dmrg_mlp_loss_grad(self.h, precision, _np_ptr(theta), _np_ptr(X),
                                                _np_ptr(T), X.shape[0], ctypes.byref(loss),
                                                _np_ptr(g)))
        return loss.value, g

    def heff_cost(self, p):
        f = ctypes.c_double()
        b = ctypes.c_double()
        n = ctypes.c_int64()
        self._check(self.lib.dmrg_heff_cost(self.h, p, ctypes.byref(f), ctypes.byref(b),
                                            ctypes.byref(n)))
        return f.value, b.value, n.value


class Batch:
    """Several contexts swept in lockstep with one fused H_eff launch per Davidson
    iteration (dmrg_batch_* in include/dmrg.h).  The contexts must outlive the batch."""

    def __init__(self, contexts):
        self.lib = load_library()
        self.contexts = list(contexts)
        arr = (ctypes.c_void_p * len(self.contexts))(*[d.h for d in self.contexts])
        h = ctypes.c_void_p()
        rc = self.lib.dmrg_batch_create(len(self.contexts), arr, ctypes.byref(h))
        self.h = h.value
        if rc != DMRG_OK:
            msg = self.lib.dmrg_batch_last_error(self.h).decode() if self.h else "create failed"
            self.close()
            raise DmrgError(rc, msg)

    def close(self):
        if getattr(self, "h", None):
            self.lib.dmrg_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def sweep(self, M):
        n = len(self.contexts)
        Ms = np.ascontiguousarray(np.broadcast_to(np.asarray(M, dtype=np.int32), (n,)))
        e = np.zeros(n)
        st = BatchStats()
        rc = self.lib.dmrg_batch_sweep(self.h, _np_ptr(Ms), _np_ptr(e), ctypes.byref(st))
        if rc != DMRG_OK:
            raise DmrgError(rc, self.lib.dmrg_batch_last_error(self.h).decode())
        return e, {f: getattr(st, f) for f, _ in BatchStats._fields_}
