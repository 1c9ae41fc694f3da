"""Thin ctypes binding of the C ABI declared in include/nsfr.h.

Argument marshalling only: every computation runs in the CUDA library
``libnsfr.so`` built in-tree for sm_103a.  Tensors are passed by
``data_ptr()``, numpy arrays by their buffer address (host pointers, which the
library stages through device memory), streams as the raw cudaStream_t of
``torch.cuda.current_stream()``.  A missing library raises at import: there is
no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libnsfr.so")

NSFR_OK = 0
NSFR_ERR_ARG = -1
STATUS = {0: "NSFR_OK", -1: "NSFR_ERR_ARG", -2: "NSFR_ERR_MESH", -3: "NSFR_ERR_CUDA",
          -4: "NSFR_ERR_NONPHYSICAL", -5: "NSFR_ERR_OOM", -6: "NSFR_ERR_STATE"}
FACE_FLUX = {"ec": 0, "ec_roe": 1, "ec_es": 2}
VOL_FLUX = {"chandrashekar": 0, "ranocha": 1}
PRECISION = {"fp64": 0, "fp32_bulk": 1, "fp32_bulk_ff": 2}
NODES = {"gl": 0, "lgl": 1}
SOURCES = {"none": 0, "manufactured": 1}

# every symbol include/nsfr.h declares
EXPORTS = ["nsfr_setup", "nsfr_setup_uncollocated", "nsfr_residual", "nsfr_residual_raw", "nsfr_rk_step", "nsfr_entropy",
           "nsfr_rk_stage", "nsfr_max_wavespeed", "nsfr_set_source", "nsfr_get_time", "nsfr_vjp", "nsfr_node_coords", "nsfr_get_metrics", "nsfr_set_metrics", "nsfr_quadrature", "nsfr_info", "nsfr_check",
           "nsfr_profile", "nsfr_profile_read", "nsfr_residual_static", "nsfr_math_eval", "nsfr_fma_probe",
           "nsfr_kernel_launches",
           "nsfr_last_error", "nsfr_destroy"]
KERNELS = ["metrics", "face_states", "volume", "max_wavespeed", "diagnostics", "vjp_face", "vjp_volume",
           "vjp_metrics", "face_flux", "source", "rk_update"]


class NSFRError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


def load_library(path=LIB_PATH):
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it with paper_2312_07725_gb300.build.build()")
    lib = ctypes.CDLL(path)
    vp, i, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    lib.nsfr_setup.argtypes = [vp, i, i, i, i, i, d, i, i, d, i, i, ctypes.POINTER(vp)]
    lib.nsfr_setup_uncollocated.argtypes = [vp, i, i, i, i, i, i, d, i, i, d, i, ctypes.POINTER(vp)]
    lib.nsfr_setup_uncollocated.restype = i
    lib.nsfr_setup.restype = i
    for name in ("nsfr_residual", "nsfr_residual_raw"):
        getattr(lib, name).argtypes = [vp, vp, vp, vp]
        getattr(lib, name).restype = i
    lib.nsfr_rk_step.argtypes = [vp, vp, d, d, ctypes.POINTER(d), vp]
    lib.nsfr_rk_step.restype = i
    lib.nsfr_entropy.argtypes = [vp, vp, vp, vp]
    lib.nsfr_entropy.restype = i
    lib.nsfr_vjp.argtypes = [vp, vp, vp, vp, vp, vp]
    lib.nsfr_vjp.restype = i
    lib.nsfr_node_coords.argtypes = [vp, vp, vp]
    lib.nsfr_node_coords.restype = i
    lib.nsfr_get_metrics.argtypes = [vp, vp, vp, vp, vp]
    lib.nsfr_get_metrics.restype = i
    lib.nsfr_set_metrics.argtypes = [vp, vp, vp, vp, vp]
    lib.nsfr_set_metrics.restype = i
    lib.nsfr_quadrature.argtypes = [vp, vp, vp]
    lib.nsfr_quadrature.restype = i
    lib.nsfr_info.argtypes = [vp, ctypes.POINTER(ctypes.c_longlong)]
    lib.nsfr_info.restype = i
    lib.nsfr_check.argtypes = [vp]
    lib.nsfr_check.restype = i
    lib.nsfr_profile.argtypes = [vp, i]
    lib.nsfr_profile.restype = i
    lib.nsfr_profile_read.argtypes = [vp, vp, vp]
    lib.nsfr_profile_read.restype = i
    lib.nsfr_residual_static.argtypes = [vp, vp, vp, vp, i, i, i, i, d, i, d, vp, vp]
    lib.nsfr_residual_static.restype = i
    lib.nsfr_rk_stage.argtypes = [vp, vp, vp, vp, i, d, i, i, vp]
    lib.nsfr_rk_stage.restype = i
    lib.nsfr_max_wavespeed.argtypes = [vp, vp, ctypes.POINTER(d), vp]
    lib.nsfr_max_wavespeed.restype = i
    lib.nsfr_set_source.argtypes = [vp, i, d]
    lib.nsfr_set_source.restype = i
    lib.nsfr_get_time.argtypes = [vp, ctypes.POINTER(d)]
    lib.nsfr_get_time.restype = i
    lib.nsfr_math_eval.argtypes = [i, vp, vp, ctypes.c_longlong, vp]
    lib.nsfr_math_eval.restype = i
    lib.nsfr_fma_probe.argtypes = [i, ctypes.c_longlong, i, vp, ctypes.POINTER(ctypes.c_longlong), vp]
    lib.nsfr_fma_probe.restype = i
    lib.nsfr_kernel_launches.argtypes = [vp]
    lib.nsfr_kernel_launches.restype = ctypes.c_longlong
    lib.nsfr_last_error.argtypes = [vp]
    lib.nsfr_last_error.restype = ctypes.c_char_p
    lib.nsfr_destroy.argtypes = [vp]
    lib.nsfr_destroy.restype = None
    return lib


_LIB = None


def lib():
    global _LIB
    if _LIB is None:
        _LIB = load_library()
    return _LIB


def _ptr(x):
    """Address of a torch tensor (device or host) or a C-contiguous numpy array."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"] or x.dtype != np.float64:
            raise ValueError("numpy buffers must be C-contiguous float64")
        return x.ctypes.data
    if not x.is_contiguous() or str(x.dtype) != "torch.float64":
        raise ValueError("tensors must be contiguous float64")
    return x.data_ptr()


def _stream(stream):
    if stream is not None:
        return stream
    try:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream
    except Exception:  # pragma: no cover
        pass
    return None


def residual_static(u, C, J, Cf, shape, p, c=0.0, face_flux="ec", gamma=1.4, dudt=None, stream=None):
    """du/dt through nsfr_residual_static: no context and no device allocation by the
    library (its working memory is a fixed array inside libnsfr.so).  All buffers
    are caller-owned contiguous float64 CUDA tensors on the current device, sized for
    the mesh (u and dudt N_e*5*n^3, C N_e*9*n^3, J N_e*n^3, Cf N_e*9*n^2 entries);
    anything else raises NSFRError with NSFR_ERR_ARG before the library is called.
    Returns ``dudt``."""
    import torch
    nx, ny, nz = shape
    ne, n = nx * ny * nz, p + 1
    want = {"u": (u, ne * 5 * n ** 3), "C": (C, ne * 9 * n ** 3), "J": (J, ne * n ** 3),
            "Cf": (Cf, ne * 9 * n * n), "dudt": (dudt, ne * 5 * n ** 3)}
    dev = torch.cuda.current_device()
    for name, (x, size) in want.items():
        if not (isinstance(x, torch.Tensor) and x.is_cuda and x.device.index == dev and x.dtype == torch.float64
                and x.is_contiguous() and x.numel() == size):
            raise NSFRError(NSFR_ERR_ARG, f"nsfr_residual_static: {name} must be a contiguous float64 tensor "
                                          f"of {size} entries on cuda:{dev}")
    st = lib().nsfr_residual_static(_ptr(u), _ptr(C), _ptr(J), _ptr(Cf), nx, ny, nz, p, float(c),
                                    FACE_FLUX[face_flux], float(gamma), _ptr(dudt), _stream(stream))
    if st != NSFR_OK:
        raise NSFRError(st, "nsfr_residual_static failed")
    return dudt


def fma_probe(fp32, iters, blocks, sink, stream=None):
    """Launch nsfr_fma_probe (FP64 or FP32 multiply-add chains) on ``stream``; returns the
    number of multiply-adds the launch performs (the caller times it)."""
    n = ctypes.c_longlong(0)
    st = lib().nsfr_fma_probe(int(bool(fp32)), int(iters), int(blocks), _ptr(sink), ctypes.byref(n), _stream(stream))
    if st != NSFR_OK:
        raise NSFRError(st, "nsfr_fma_probe failed")
    return n.value


MATH_FN = {"log": 0, "exp": 1, "rcp": 2, "rcp1": 3, "log_ff": 4, "exp_ff": 5, "join": 6, "logmean1": 7,
           "split": 8, "i2d": 9}


def math_eval(fn, x, y=None, stream=None):
    """y = fn(x) elementwise with the library's device functions (``log``, ``exp``,
    ``rcp``: full-precision reciprocal, ``rcp1``: one Newton step, ``log_ff``,
    ``exp_ff``: the float-float functions of the FP32-bulk kernels, ``join``:
    the integer-pipe join of the float pair packed in each element's 64 bits,
    ``logmean1``: the volume kernels' logarithmic mean of x and 1, ``split``:
    the integer-pipe split of x into two floats, packed as ``join`` takes them,
    ``i2d``: the int in the low 32 bits of x as a double), for checking them;
    x, y contiguous float64 CUDA tensors.  Returns y."""
    import torch
    if y is None:
        y = torch.empty_like(x)
    st = lib().nsfr_math_eval(MATH_FN[fn], _ptr(x), _ptr(y), x.numel(), _stream(stream))
    if st != NSFR_OK:
        raise NSFRError(st, "nsfr_math_eval failed")
    return y


class Solver:
    """One NSFR-EC discretisation (mesh, p, c, fluxes, precision) on the current device."""

    def __init__(self, grid_nodes, shape, p, p_geo=None, c=0.0, face_flux="ec", gamma=1.4,
                 precision="fp64", nodes="gl", nq=None, vol_flux="chandrashekar"):
        """``nodes``: "gl" or "lgl" collocated; with ``nq`` (>= p+1) the uncollocated scheme:
        solution on the LGL nodes, nq GL quadrature points per direction.  ``vol_flux``:
        "chandrashekar" or "ranocha" (Chandrashekar's flux with Ranocha's pressure terms)."""
        self._lib = lib()
        nx, ny, nz = shape
        pg = p if p_geo is None else p_geo
        self.shape, self.p, self.p_geo, self.n = tuple(shape), p, pg, p + 1
        self.nv = self.n ** 3
        self.n_el = nx * ny * nz
        self.c, self.gamma, self.face_flux, self.precision, self.nodes = c, gamma, face_flux, precision, nodes
        self.vol_flux = vol_flux
        self._keep = grid_nodes
        h = ctypes.c_void_p()
        self.nq = nq
        npt = self.n if nq is None else int(nq)
        self.nqv, self.nqf = npt ** 3, npt ** 2  # quadrature points per element / per face
        if nq is None:
            st = self._lib.nsfr_setup(_ptr(grid_nodes), nx, ny, nz, pg, p, float(c), VOL_FLUX[vol_flux],
                                      FACE_FLUX[face_flux],
                                      float(gamma), PRECISION[precision], NODES[nodes], ctypes.byref(h))
        else:
            if precision not in ("fp64", "fp32_bulk"):
                raise ValueError("the uncollocated scheme has the fp64 and fp32_bulk precisions")
            st = self._lib.nsfr_setup_uncollocated(_ptr(grid_nodes), nx, ny, nz, pg, p, int(nq), float(c),
                                                   VOL_FLUX[vol_flux], FACE_FLUX[face_flux], float(gamma),
                                                   PRECISION[precision], ctypes.byref(h))
        if st != NSFR_OK:
            raise NSFRError(st, "nsfr_setup failed")
        self._h = h

    # -- helpers -----------------------------------------------------------
    def _check(self, st, what):
        if st != NSFR_OK:
            msg = self._lib.nsfr_last_error(self._h).decode()
            raise NSFRError(st, f"{what}: {msg}")

    @property
    def state_shape(self):
        return (self.n_el, 5, self.nv)

    def close(self):
        if getattr(self, "_h", None):
            self._lib.nsfr_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- the ABI calls --------------------------------------------------------
    def residual(self, u, dudt, stream=None):
        self._check(self._lib.nsfr_residual(self._h, _ptr(u), _ptr(dudt), _stream(stream)), "nsfr_residual")
        return dudt

    def residual_raw(self, u, R, stream=None):
        self._check(self._lib.nsfr_residual_raw(self._h, _ptr(u), _ptr(R), _stream(stream)), "nsfr_residual_raw")
        return R

    def rk_step(self, u, cfl=0.1, dt=0.0, stream=None):
        used = ctypes.c_double(0.0)
        self._check(self._lib.nsfr_rk_step(self._h, _ptr(u), float(cfl), float(dt), ctypes.byref(used),
                                           _stream(stream)), "nsfr_rk_step")
        return used.value

    def rk_stage(self, u, ustage, acc, stage, dt, elements=None, stream=None):
        """One RK4 stage on caller-owned device arrays (see nsfr_rk_stage); ``elements``
        (begin, end) limits the update to that element range."""
        b, e = (0, self.n_el) if elements is None else elements
        self._check(self._lib.nsfr_rk_stage(self._h, _ptr(u), _ptr(ustage), _ptr(acc), int(stage), float(dt),
                                            int(b), int(e), _stream(stream)), "nsfr_rk_stage")

    def max_wavespeed(self, u, stream=None):
        lam = ctypes.c_double(0.0)
        self._check(self._lib.nsfr_max_wavespeed(self._h, _ptr(u), ctypes.byref(lam), _stream(stream)),
                    "nsfr_max_wavespeed")
        return lam.value

    def set_source(self, kind="manufactured", t=0.0):
        """Volume source ("none" or "manufactured") and the context's time (nsfr_set_source)."""
        self._check(self._lib.nsfr_set_source(self._h, SOURCES[kind], float(t)), "nsfr_set_source")

    @property
    def time(self):
        t = ctypes.c_double(0.0)
        self._check(self._lib.nsfr_get_time(self._h, ctypes.byref(t)), "nsfr_get_time")
        return t.value

    @property
    def dx(self):
        """min_d L_d / (N_d (p+1)), the node spacing of the CFL step (from the control points)."""
        lo = self._keep.reshape(-1, 3).min(axis=0)
        hi = self._keep.reshape(-1, 3).max(axis=0)
        return float(min((hi[d] - lo[d]) / (self.shape[d] * (self.p + 1)) for d in range(3)))

    def entropy(self, u, stream=None):
        out = np.zeros(14)
        self._check(self._lib.nsfr_entropy(self._h, _ptr(u), out.ctypes.data, _stream(stream)), "nsfr_entropy")
        return {"entropy": out[0], "entropy_rate": out[1], "entropy_rate_scale": out[2],
                "Q": out[3:8].copy(), "kinetic_energy": out[8], "sum_R": out[9:14].copy()}

    def vjp(self, u, dudt_bar, u_bar, x_bar=None, stream=None):
        self._check(self._lib.nsfr_vjp(self._h, _ptr(u), _ptr(dudt_bar), _ptr(u_bar), _ptr(x_bar),
                                       _stream(stream)), "nsfr_vjp")

    def node_coords(self, out=None, stream=None):
        if out is None:
            out = np.zeros((self.n_el, 3, self.nv))
        self._check(self._lib.nsfr_node_coords(self._h, _ptr(out), _stream(stream)), "nsfr_node_coords")
        return out

    def metrics(self, stream=None):
        """Metric rows [N_e][9][points], Jacobians [N_e][points] and shared face rows
        [N_e][3][3][face points] at the volume / face quadrature points."""
        C = np.zeros((self.n_el, 9, self.nqv))
        J = np.zeros((self.n_el, self.nqv))
        Cf = np.zeros((self.n_el, 3, 3, self.nqf))
        self._check(self._lib.nsfr_get_metrics(self._h, _ptr(C), _ptr(J), _ptr(Cf), _stream(stream)),
                    "nsfr_get_metrics")
        return C, J, Cf

    def set_metrics(self, C, J, Cf, stream=None):
        """Use caller-supplied metric terms (layouts as ``metrics``)."""
        C, J, Cf = (np.ascontiguousarray(x, dtype=np.float64) if isinstance(x, np.ndarray) else x
                    for x in (C, J, Cf))
        self._check(self._lib.nsfr_set_metrics(self._h, _ptr(C), _ptr(J), _ptr(Cf), _stream(stream)),
                    "nsfr_set_metrics")

    def quadrature(self, out=None, stream=None):
        """W J at the volume quadrature points, [N_e][points]."""
        if out is None:
            out = np.zeros((self.n_el, self.nqv))
        self._check(self._lib.nsfr_quadrature(self._h, _ptr(out), _stream(stream)), "nsfr_quadrature")
        return out

    def check(self):
        self._check(self._lib.nsfr_check(self._h), "nsfr_check")

    def profile(self, on=True):
        self._check(self._lib.nsfr_profile(self._h, 1 if on else 0), "nsfr_profile")

    def profile_read(self):
        ms = np.zeros(len(KERNELS))
        cnt = np.zeros(len(KERNELS), dtype=np.int64)
        self._check(self._lib.nsfr_profile_read(self._h, ms.ctypes.data, cnt.ctypes.data), "nsfr_profile_read")
        return {k: (float(ms[i]), int(cnt[i])) for i, k in enumerate(KERNELS) if cnt[i]}

    def kernel_launches(self):
        return int(self._lib.nsfr_kernel_launches(self._h))
