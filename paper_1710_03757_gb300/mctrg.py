"""Thin ctypes binding of the MC-TRG C ABI (include/mctrg.h, include/mctrg_host.h).

Argument marshalling only: every step of the method runs in libmctrg.so.
Names follow the C functions.  Output buffers may be numpy arrays (host) or
torch tensors (host or device); the library detects device pointers itself.
"""
import ctypes
import os

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_lib", "libmctrg.so")

MCTRG_OK, MCTRG_EINVAL, MCTRG_ENOMEM, MCTRG_ENOCONV, MCTRG_EDOMAIN = 0, -1, -2, -3, -4
MCTRG_ECUDA, MCTRG_ESTATE, MCTRG_ETIMEDOUT, MCTRG_EAGAIN, MCTRG_EUNREACHABLE = -5, -6, -7, -8, -9
MCTRG_ENOTFOUND = -10
MCTRG_FP64, MCTRG_TF32, MCTRG_BF16, MCTRG_TF32X3, MCTRG_BF16X3, MCTRG_FP64TC = 0, 1, 2, 3, 4, 5
FLAG_SPLIT_CLUSTER, FLAG_DRAW_TIE, FLAG_TINY_KEPT, FLAG_NOCONV = 1, 2, 4, 16

# every symbol the headers declare (checked by the CPU test suite)
EXPORTS = [
    "mctrg_options_default", "mctrg_create", "mctrg_init_lattice", "mctrg_init_bond_lattice", "mctrg_init_tensor",
    "mctrg_run", "mctrg_footprint", "mctrg_merge_estimates", "mctrg_destroy", "mctrg_strerror",
    "mctrg_server_create", "mctrg_server_submit", "mctrg_server_poll", "mctrg_server_wait",
    "mctrg_server_destroy", "mctrg_plan_level", "mctrg_philox_uniform", "mctrg_kernel_stats",
    "mctrg_reset_kernel_stats", "mctrg_svd_batched", "mctrg_svd_batched_noalloc",
    "mctrg_svd_bidiag_batched", "mctrg_measure_fp64_peak", "mctrg_contract_batched",
    "mctrg_server_footprint", "mctrg_server_memory", "mctrg_batch_run", "mctrg_init_impurity",
    "mctrg_ratio_estimate", "mctrg_hotrg_run", "mctrg_svd_band_batched", "mctrg_band_reduce_batched",
]
(K_FORM_XY, K_GEMM, K_JACOBI, K_SAMPLE, K_TRACE, K_OTHER, K_BIDIAG, K_BISECT, K_VECTORS, K_BAND, K_CHASE,
 K_COUNT) = range(12)
KERNEL_NAMES = ["form_xy", "gemm", "jacobi", "sample_split", "trace", "other", "bidiag", "bisect", "vectors", "band",
                "chase"]
SVD_AUTO, SVD_JACOBI, SVD_BIDIAG, SVD_BAND = 0, 1, 2, 3


class KernelStat(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_int64), ("ms", ctypes.c_double), ("items", ctypes.c_int64),
                ("flops_alg", ctypes.c_double), ("bytes_alg", ctypes.c_double)]


class Options(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int), ("cuda_stream", ctypes.c_void_p), ("precision", ctypes.c_int),
                ("hbm_budget_bytes", ctypes.c_size_t), ("max_sweeps", ctypes.c_int),
                ("max_chunk", ctypes.c_int), ("profile", ctypes.c_int), ("svd", ctypes.c_int),
                ("zero_tol_scale", ctypes.c_double), ("deterministic_levels", ctypes.c_int),
                ("autotune_cache", ctypes.c_char_p)]


class Job(ctypes.Structure):
    _fields_ = [("beta", ctypes.c_double), ("h", ctypes.c_double), ("L", ctypes.c_int), ("chi", ctypes.c_int),
                ("n_samples", ctypes.c_int64), ("seed", ctypes.c_uint64), ("first_traj", ctypes.c_uint64)]


class Estimate(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("ln_mean_Z", ctypes.c_double), ("se_ln_Z", ctypes.c_double),
                ("mean_Z_scaled", ctypes.c_double), ("se_Z_scaled", ctypes.c_double),
                ("ln_scale", ctypes.c_double), ("ess", ctypes.c_double), ("n_negative", ctypes.c_int64),
                ("n_flagged", ctypes.c_int64), ("sum_x", ctypes.c_double), ("m2_x", ctypes.c_double),
                ("status", ctypes.c_int)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


_lib = None


def lib():
    """The loaded library; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libmctrg.so is not built (%s): run "
                               "`python -m paper_1710_03757_gb300.build`" % LIB_PATH)
        L = ctypes.CDLL(LIB_PATH)
        c_int, c_double, vp = ctypes.c_int, ctypes.c_double, ctypes.c_void_p
        i64, u64, u32 = ctypes.c_int64, ctypes.c_uint64, ctypes.c_uint32
        sig = {
            "mctrg_options_default": (c_int, [ctypes.POINTER(Options)]),
            "mctrg_create": (c_int, [ctypes.POINTER(Options), ctypes.POINTER(vp)]),
            "mctrg_init_lattice": (c_int, [vp, c_double, c_double, c_int, c_int]),
            "mctrg_init_bond_lattice": (c_int, [vp, c_double, c_double, c_int, c_int]),
            "mctrg_init_tensor": (c_int, [vp, vp, c_int, c_int, c_int]),
            "mctrg_init_impurity": (c_int, [vp, c_double, c_double, c_int, c_int, c_int]),
            "mctrg_ratio_estimate": (c_int, [ctypes.POINTER(Estimate), ctypes.POINTER(Estimate),
                                             ctypes.POINTER(c_double), ctypes.POINTER(c_double)]),
            "mctrg_run": (c_int, [vp, i64, u64, u64, vp, vp, vp, ctypes.POINTER(Estimate)]),
            "mctrg_hotrg_run": (c_int, [ctypes.POINTER(Options), c_double, c_double, vp, c_int, c_int, c_int, i64,
                                        u64, u64, vp, vp, vp, ctypes.POINTER(Estimate)]),
            "mctrg_footprint": (c_int, [vp, i64, ctypes.POINTER(ctypes.c_size_t)]),
            "mctrg_merge_estimates": (c_int, [ctypes.POINTER(Estimate), c_int, ctypes.POINTER(Estimate)]),
            "mctrg_destroy": (None, [vp]),
            "mctrg_strerror": (ctypes.c_char_p, [c_int]),
            "mctrg_server_create": (c_int, [ctypes.POINTER(Options), ctypes.POINTER(vp)]),
            "mctrg_server_submit": (c_int, [vp, c_double, c_double, c_int, c_int, c_double, i64, u64,
                                            ctypes.POINTER(u64)]),
            "mctrg_server_poll": (c_int, [vp, u64, ctypes.POINTER(Estimate), ctypes.POINTER(c_double)]),
            "mctrg_server_wait": (c_int, [vp, u64, c_double, ctypes.POINTER(Estimate),
                                          ctypes.POINTER(c_double)]),
            "mctrg_server_destroy": (None, [vp]),
            "mctrg_server_footprint": (c_int, [vp, c_int, c_int, i64, ctypes.POINTER(ctypes.c_size_t)]),
            "mctrg_batch_run": (c_int, [ctypes.POINTER(Options), ctypes.POINTER(Job), c_int, ctypes.POINTER(Estimate),
                                        vp, vp, vp]),
            "mctrg_server_memory": (c_int, [vp, ctypes.POINTER(ctypes.c_size_t), ctypes.POINTER(ctypes.c_size_t)]),
            "mctrg_plan_level": (c_int, [c_int, c_int, vp, vp]),
            "mctrg_philox_uniform": (c_double, [u64, u32, u32, u32, u32]),
            "mctrg_kernel_stats": (c_int, [vp, c_int, ctypes.POINTER(KernelStat)]),
            "mctrg_reset_kernel_stats": (c_int, [vp]),
            "mctrg_svd_batched": (c_int, [vp, c_int, i64, vp, vp, c_int, vp]),
            "mctrg_svd_batched_noalloc": (c_int, [vp, c_int, i64, vp, vp, c_int, vp]),
            "mctrg_svd_bidiag_batched": (c_int, [vp, c_int, i64, vp, c_int, vp, vp]),
            "mctrg_svd_band_batched": (c_int, [vp, c_int, i64, vp, c_int, vp, vp]),
            "mctrg_band_reduce_batched": (c_int, [vp, c_int, i64, vp, vp, vp]),
            "mctrg_measure_fp64_peak": (c_int, [c_int, i64, ctypes.POINTER(c_double), ctypes.POINTER(c_double)]),
            "mctrg_contract_batched": (c_int, [vp, vp, c_int, c_int, i64, vp, c_int, vp]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _ptr(x):
    """Raw address of a numpy array or torch tensor (None -> NULL)."""
    if x is None:
        return None
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("output tensors must be contiguous")
        return x.data_ptr()
    if hasattr(x, "ctypes"):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("output arrays must be C-contiguous")
        return x.ctypes.data
    raise TypeError("expected a numpy array or torch tensor")


class MctrgError(RuntimeError):
    def __init__(self, status, what=""):
        self.status = status
        super().__init__("%s: %s (%d)" % (what, mctrg_strerror(status), status))


def _check(status, what):
    if status != MCTRG_OK:
        raise MctrgError(status, what)


def mctrg_strerror(status):
    return lib().mctrg_strerror(int(status)).decode()


def mctrg_options_default():
    o = Options()
    _check(lib().mctrg_options_default(ctypes.byref(o)), "mctrg_options_default")
    return o


def make_options(device=0, stream=None, precision=MCTRG_FP64, hbm_budget_bytes=0, max_sweeps=0,
                 max_chunk=0, profile=0, svd=SVD_AUTO, zero_tol_scale=0.0, deterministic_levels=0,
                 autotune_cache=None):
    o = mctrg_options_default()
    o.deterministic_levels = int(deterministic_levels)
    o.autotune_cache = autotune_cache.encode() if autotune_cache else None
    o.device, o.precision, o.profile, o.svd = int(device), int(precision), int(profile), int(svd)
    o.zero_tol_scale = float(zero_tol_scale)
    o.cuda_stream = stream
    o.hbm_budget_bytes, o.max_sweeps, o.max_chunk = int(hbm_budget_bytes), int(max_sweeps), int(max_chunk)
    return o


def mctrg_create(opts=None):
    opts = opts or mctrg_options_default()
    h = ctypes.c_void_p()
    _check(lib().mctrg_create(ctypes.byref(opts), ctypes.byref(h)), "mctrg_create")
    return h


def mctrg_init_lattice(ctx, beta, h, L, chi):
    return lib().mctrg_init_lattice(ctx, float(beta), float(h), int(L), int(chi))


def mctrg_init_bond_lattice(ctx, beta, h, L, chi):
    """The spins-on-bonds network of the paper's Fig. 1 (L = 8: 128 spins)."""
    return lib().mctrg_init_bond_lattice(ctx, float(beta), float(h), int(L), int(chi))


def mctrg_init_impurity(ctx, beta, h, L, chi, n_imp=1):
    """Site (0,0) (and (1,0) for n_imp = 2) carries its spin: trajectories sample Z <sigma ...>."""
    return lib().mctrg_init_impurity(ctx, float(beta), float(h), int(L), int(chi), int(n_imp))


def mctrg_ratio_estimate(num, den):
    """(status, ratio, standard error) of two estimates' means."""
    r, se = ctypes.c_double(), ctypes.c_double()
    s = lib().mctrg_ratio_estimate(ctypes.byref(num), ctypes.byref(den), ctypes.byref(r), ctypes.byref(se))
    return s, r.value, se.value


def mctrg_init_tensor(ctx, T0, D, L, chi):
    import numpy as np
    T0 = np.ascontiguousarray(T0, dtype=np.float64)
    if T0.size != D ** 4:
        raise ValueError("T0 must hold D^4 values")
    return lib().mctrg_init_tensor(ctx, T0.ctypes.data, int(D), int(L), int(chi))


def mctrg_run(ctx, n_samples, seed, first_traj=0, lnabsZ=None, sign=None, flags=None):
    """Returns (status, Estimate)."""
    est = Estimate()
    s = lib().mctrg_run(ctx, int(n_samples), int(seed), int(first_traj), _ptr(lnabsZ), _ptr(sign),
                        _ptr(flags), ctypes.byref(est))
    return s, est


def mctrg_hotrg_run(opt, L, chi, n_samples, seed, first_traj=0, beta=0.0, h=0.0, T0=None, lnabsZ=None,
                    sign=None, flags=None):
    """Monte Carlo HOTRG trajectories; T0 None for the Ising site tensor at
    (beta, h).  Returns (status, Estimate)."""
    import numpy as np
    est = Estimate()
    if T0 is None:
        tp, D = None, 2
    else:
        T0 = np.ascontiguousarray(T0, dtype=np.float64)
        D = T0.shape[0]
        if T0.size != D ** 4:
            raise ValueError("T0 must hold D^4 values")
        tp = T0.ctypes.data
    s = lib().mctrg_hotrg_run(ctypes.byref(opt), float(beta), float(h), tp, int(D), int(L), int(chi),
                              int(n_samples), int(seed), int(first_traj), _ptr(lnabsZ), _ptr(sign), _ptr(flags),
                              ctypes.byref(est))
    return s, est


def mctrg_footprint(ctx, n_samples):
    b = ctypes.c_size_t()
    _check(lib().mctrg_footprint(ctx, int(n_samples), ctypes.byref(b)), "mctrg_footprint")
    return b.value


def mctrg_merge_estimates(parts):
    arr = (Estimate * len(parts))(*parts)
    out = Estimate()
    _check(lib().mctrg_merge_estimates(arr, len(parts), ctypes.byref(out)), "mctrg_merge_estimates")
    return out


def mctrg_kernel_stats(ctx, kernel):
    st = KernelStat()
    _check(lib().mctrg_kernel_stats(ctx, int(kernel), ctypes.byref(st)), "mctrg_kernel_stats")
    return st


def mctrg_reset_kernel_stats(ctx):
    _check(lib().mctrg_reset_kernel_stats(ctx), "mctrg_reset_kernel_stats")


def mctrg_svd_batched(M, sigma, vt=None, max_sweeps=0, stream=None):
    """M: device tensor (batch, n, n) float64; sigma: (batch, n); vt: (batch, n, n) or None."""
    batch, n = int(M.shape[0]), int(M.shape[-1])
    return lib().mctrg_svd_batched(_ptr(M), n, batch, _ptr(sigma), _ptr(vt), int(max_sweeps), stream)


def mctrg_svd_batched_noalloc(M, sigma, vt=None, max_sweeps=0, stream=None):
    """As mctrg_svd_batched, with the library's fixed working array instead of
    device allocations (for callers that cannot allocate)."""
    batch, n = int(M.shape[0]), int(M.shape[-1])
    return lib().mctrg_svd_batched_noalloc(_ptr(M), n, batch, _ptr(sigma), _ptr(vt), int(max_sweeps), stream)


def mctrg_svd_bidiag_batched(M, sigma, vt=None, stream=None):
    """Bidiagonalization route: M (batch, n, n) float64 device tensor; sigma
    (batch, n); vt (batch, n_vec, n) receives the unit right vectors of the
    n_vec largest singular values (None: values only)."""
    batch, n = int(M.shape[0]), int(M.shape[-1])
    nv = 0 if vt is None else int(vt.shape[1])
    return lib().mctrg_svd_bidiag_batched(_ptr(M), n, batch, _ptr(sigma), nv, _ptr(vt), stream)


def mctrg_svd_band_batched(M, sigma, vt=None, stream=None):
    """Two-stage (band) route: M (batch, n, n) float64 device tensor, n a
    multiple of 8 from 64 to 256; sigma (batch, n); vt (batch, n_vec, n),
    n_vec <= 16, receives the unit right vectors of the n_vec largest singular
    values (None: values only)."""
    batch, n = int(M.shape[0]), int(M.shape[-1])
    nv = 0 if vt is None else int(vt.shape[1])
    return lib().mctrg_svd_band_batched(_ptr(M), n, batch, _ptr(sigma), nv, _ptr(vt), stream)


def mctrg_band_reduce_batched(M, band, bd=None, stream=None):
    """Stage 1 (and 2 when bd is given) of the band route: band (batch, n, 9)
    receives B(i, i+o); bd (batch, 3n) the bidiagonal's d, e."""
    batch, n = int(M.shape[0]), int(M.shape[-1])
    return lib().mctrg_band_reduce_batched(_ptr(M), n, batch, _ptr(band), _ptr(bd), stream)


def mctrg_batch_run(jobs, opts=None, lnabsZ=None, sign=None, flags=None):
    """jobs: sequence of (beta, h, L, chi, n_samples, seed, first_traj).
    Returns (status, [Estimate per job])."""
    arr = (Job * len(jobs))(*[Job(float(b), float(h), int(L), int(c), int(n), int(s), int(f))
                               for b, h, L, c, n, s, f in jobs])
    ests = (Estimate * len(jobs))()
    opts = opts or mctrg_options_default()
    st = lib().mctrg_batch_run(ctypes.byref(opts), arr, len(jobs), ests, _ptr(lnabsZ), _ptr(sign), _ptr(flags))
    return st, list(ests)


def mctrg_contract_batched(X, Yt, M, precision=MCTRG_FP64, stream=None):
    """M[b] = X[b] Yt[b]^T: X, Yt (batch, D*D, K) and M (batch, D*D, D*D) float64 device tensors."""
    batch, n, K = int(X.shape[0]), int(X.shape[1]), int(X.shape[2])
    D = int(round(n ** 0.5))
    if D * D != n:
        raise ValueError("rows must be a perfect square D*D")
    return lib().mctrg_contract_batched(_ptr(X), _ptr(Yt), D, K, batch, _ptr(M), int(precision), stream)


def mctrg_measure_fp64_peak(device=0, steps=1 << 14):
    """(status, TFLOP/s, ms) of the library's DFMA throughput probe."""
    tf, ms = ctypes.c_double(), ctypes.c_double()
    s = lib().mctrg_measure_fp64_peak(int(device), int(steps), ctypes.byref(tf), ctypes.byref(ms))
    return s, tf.value, ms.value


def mctrg_destroy(ctx):
    lib().mctrg_destroy(ctx)


def mctrg_plan_level(L, k):
    """(parity uint8[N_k], parents int64[N_k/2, 4]) of level k, computed by the library."""
    import numpy as np
    N = (L * L) >> k
    par = np.zeros(N, dtype=np.uint8)
    parents = np.zeros((N // 2, 4), dtype=np.int64)
    _check(lib().mctrg_plan_level(int(L), int(k), par.ctypes.data, parents.ctypes.data), "mctrg_plan_level")
    return par, parents


def mctrg_philox_uniform(seed, traj, level, tensor, t):
    return lib().mctrg_philox_uniform(int(seed), int(traj), int(level), int(tensor), int(t))


# ---- serving ----
def mctrg_server_create(opts=None):
    opts = opts or mctrg_options_default()
    h = ctypes.c_void_p()
    _check(lib().mctrg_server_create(ctypes.byref(opts), ctypes.byref(h)), "mctrg_server_create")
    return h


def mctrg_server_submit(srv, beta, h, L, chi, target_se_lnZ, max_samples, seed):
    jid = ctypes.c_uint64()
    s = lib().mctrg_server_submit(srv, float(beta), float(h), int(L), int(chi), float(target_se_lnZ),
                                  int(max_samples), int(seed), ctypes.byref(jid))
    return s, jid.value


def mctrg_server_poll(srv, job_id):
    est, lat = Estimate(), ctypes.c_double()
    s = lib().mctrg_server_poll(srv, int(job_id), ctypes.byref(est), ctypes.byref(lat))
    return s, est, lat.value


def mctrg_server_wait(srv, job_id, timeout_s):
    est, lat = Estimate(), ctypes.c_double()
    s = lib().mctrg_server_wait(srv, int(job_id), float(timeout_s), ctypes.byref(est), ctypes.byref(lat))
    return s, est, lat.value


def mctrg_server_footprint(srv, L, chi, max_samples):
    """(status, bytes) a job would be admitted with."""
    b = ctypes.c_size_t()
    s = lib().mctrg_server_footprint(srv, int(L), int(chi), int(max_samples), ctypes.byref(b))
    return s, b.value


def mctrg_server_memory(srv):
    """(budget, reserved) device bytes of the server."""
    b, r = ctypes.c_size_t(), ctypes.c_size_t()
    _check(lib().mctrg_server_memory(srv, ctypes.byref(b), ctypes.byref(r)), "mctrg_server_memory")
    return b.value, r.value


def mctrg_server_destroy(srv):
    lib().mctrg_server_destroy(srv)
