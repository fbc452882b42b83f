"""ctypes binding of libnlfdtd.so (include/nlfdtd.h): argument marshalling only.

Every computation happens in the CUDA library.  Importing this module does not
need a GPU; the first call that needs the library raises if it has not been
built (``paper_2005_06997_gb300.build.build()``) or if no CUDA device is present.
There is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from . import build as _build

NLF_OK = 0
ERRORS = {-1: "NLF_E_ARG", -2: "NLF_E_CFL", -3: "NLF_E_GEOMETRY", -4: "NLF_E_OOM", -5: "NLF_E_CUDA",
          -6: "NLF_E_UNSTABLE", -7: "NLF_E_TIMEOUT", -8: "NLF_E_STATE", -9: "NLF_E_UNSUPPORTED"}
BC = {"pec": 0, "cpml": 1}
SHAPE = {"sphere": 1, "box": 2, "cube_tips": 3}
WAVE = {"gaussian": 1, "raised_cos": 2}
FIELD = {"Ex": 0, "Ey": 1, "Ez": 2, "Hx": 3, "Hy": 4, "Hz": 5, "Px": 6, "Py": 7, "Pz": 8, "density": 9}
MAX_POLES = 4


class nlf_grid(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int), ("dx", C.c_double),
                ("courant", C.c_double), ("pml_cells", C.c_int), ("boundary", C.c_int * 3),
                ("eps_background", C.c_double)]


class nlf_material(C.Structure):
    _fields_ = [("eps_inf", C.c_double), ("wp", C.c_double), ("gamma", C.c_double), ("beta", C.c_double),
                ("diff", C.c_double), ("n_poles", C.c_int), ("A", C.c_double * MAX_POLES),
                ("Omega", C.c_double * MAX_POLES), ("Gamma", C.c_double * MAX_POLES),
                ("phi", C.c_double * MAX_POLES)]


class nlf_shape(C.Structure):
    _fields_ = [("kind", C.c_int), ("material", C.c_int), ("center", C.c_int * 3), ("radius", C.c_int),
                ("half", C.c_int * 3), ("side", C.c_int), ("tip_base", C.c_int), ("tip_height", C.c_int),
                ("tip_radius", C.c_int), ("tip_center", C.c_int), ("tip_cut", C.c_int)]


class nlf_source(C.Structure):
    _fields_ = [("axis_prop", C.c_int), ("axis_pol", C.c_int), ("tf_lo", C.c_int * 3), ("tf_hi", C.c_int * 3),
                ("waveform", C.c_int), ("w0", C.c_double), ("tau", C.c_double), ("t0", C.c_double),
                ("amplitude", C.c_double)]


class nlf_plane_monitor(C.Structure):
    _fields_ = [("axis", C.c_int), ("index", C.c_int), ("nf", C.c_int), ("omega", C.POINTER(C.c_double)),
                ("decimate_k", C.c_int)]


NLF_MAP_DENSITY = 9


class nlf_monitors(C.Structure):
    _fields_ = [("nf", C.c_int), ("omega", C.POINTER(C.c_double)), ("abs_lo", C.c_int * 3),
                ("abs_hi", C.c_int * 3), ("sca_lo", C.c_int * 3), ("sca_hi", C.c_int * 3),
                ("decimate_k", C.c_int), ("block_b", C.c_int)]


class nlf_info(C.Structure):
    _fields_ = [("cells", C.c_longlong), ("metal_sites", C.c_longlong), ("pole_sites", C.c_longlong),
                ("bbox_cells", C.c_longlong), ("pml_slab_cells", C.c_longlong), ("dft_records", C.c_longlong),
                ("step_bytes", C.c_double), ("step_kernel_bytes", C.c_double), ("metal_kernel_bytes", C.c_double),
                ("material_sites", C.c_longlong), ("dt", C.c_double), ("gnor", C.c_int), ("n_poles", C.c_int),
                ("h2d_bytes", C.c_longlong), ("d2h_bytes", C.c_longlong)]


_P = C.c_void_p
# name -> (restype, argtypes): the entry points declared in include/nlfdtd.h
SIGNATURES = {
    "nlf_create": (C.c_int, [C.POINTER(nlf_grid), C.POINTER(_P)]),
    "nlf_set_materials": (C.c_int, [_P, C.POINTER(nlf_material), C.c_int]),
    "nlf_set_shapes": (C.c_int, [_P, C.POINTER(nlf_shape), C.c_int]),
    "nlf_set_material_map": (C.c_int, [_P, C.c_void_p, C.c_int]),
    "nlf_set_source": (C.c_int, [_P, C.POINTER(nlf_source)]),
    "nlf_set_monitors": (C.c_int, [_P, C.POINTER(nlf_monitors)]),
    "nlf_set_plane_monitor": (C.c_int, [_P, C.POINTER(nlf_plane_monitor)]),
    "nlf_get_plane_map": (C.c_int, [_P, C.c_int, C.POINTER(C.c_double)]),
    "nlf_state_bytes": (C.c_size_t, [_P]),
    "nlf_bind_state": (C.c_int, [_P, C.c_void_p, C.c_size_t]),
    "nlf_run": (C.c_int, [_P, C.c_longlong, C.c_void_p]),
    "nlf_reset": (C.c_int, [_P, C.c_void_p]),
    "nlf_sync": (C.c_int, [_P, C.c_int]),
    "nlf_get_field": (C.c_int, [_P, C.c_int, C.c_void_p, C.c_int]),
    "nlf_set_field": (C.c_int, [_P, C.c_int, C.c_void_p, C.c_int]),
    "nlf_get_voxels": (C.c_int, [_P, C.c_void_p]),
    "nlf_get_spectra": (C.c_int, [_P, C.c_void_p, C.c_void_p, C.c_void_p]),
    "nlf_get_dft": (C.c_int, [_P, C.c_void_p]),
    "nlf_num_records": (C.c_longlong, [_P]),
    "nlf_get_flux_weights": (C.c_int, [_P, C.c_void_p, C.POINTER(C.c_longlong)]),
    "nlf_save_state": (C.c_int, [_P, C.c_void_p]),
    "nlf_load_state": (C.c_int, [_P, C.c_void_p]),
    "nlf_batch_run": (C.c_int, [C.POINTER(_P), C.c_int, C.POINTER(C.c_longlong), C.c_void_p,
                                C.POINTER(C.c_int)]),
    "nlf_flux_spectra_static": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_longlong, C.c_longlong, C.c_int,
                                          C.c_double, C.c_void_p, C.c_void_p]),
    "nlf_time_index": (C.c_longlong, [_P]),
    "nlf_time_kernels": (C.c_int, [_P, C.c_longlong, C.c_void_p, C.POINTER(C.c_double)]),
    "nlf_get_info": (C.c_int, [_P, C.POINTER(nlf_info)]),
    "nlf_kernel_launches": (C.c_longlong, [_P]),
    "nlf_last_error": (C.c_char_p, [_P]),
    "nlf_destroy": (None, [_P]),
}

_lock = threading.Lock()
_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libnlfdtd.so (building it in-tree first if asked).  Raises if missing."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB
        if not os.path.exists(path):
            if not build_if_missing:
                raise RuntimeError("libnlfdtd.so is not built (run paper_2005_06997_gb300.build.build())")
            _build.build()
        L = C.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
        return L


def require_gpu():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("no CUDA device: the nonlocal FDTD library runs on the GPU only")


class NLFError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s (%d): %s" % (ERRORS.get(code, "?"), code, msg))
        self.code = code


def _check(ctx, rc):
    if rc != NLF_OK:
        msg = load().nlf_last_error(ctx).decode() if ctx else ""
        raise NLFError(rc, msg)


# ----------------------------------------------------------- problem dicts

def make_grid(prob) -> nlf_grid:
    g = nlf_grid()
    g.nx, g.ny, g.nz = prob["shape"]
    g.dx = prob["dx"]
    g.courant = prob["courant"]
    g.pml_cells = prob.get("pml", 0)
    for a, b in enumerate(prob.get("bc", ("pec",) * 3)):
        g.boundary[a] = BC[b]
    g.eps_background = prob.get("eps_b", 1.0)
    return g


def make_materials(prob):
    mats = prob.get("materials", [])
    arr = (nlf_material * max(1, len(mats)))()
    for q, m in enumerate(mats):
        o = arr[q]
        o.eps_inf = m.get("eps_inf", 1.0)
        o.wp, o.gamma = m.get("wp", 0.0), m.get("gamma", 0.0)
        o.beta, o.diff = m.get("beta", 0.0), m.get("diff", 0.0)
        poles = m.get("poles", [])
        o.n_poles = len(poles)
        for p, (A, Om, Ga, ph) in enumerate(poles):
            o.A[p], o.Omega[p], o.Gamma[p], o.phi[p] = A, Om, Ga, ph
    return arr, len(mats)


def make_shapes(prob):
    shapes = prob.get("shapes", [])
    arr = (nlf_shape * max(1, len(shapes)))()
    for q, s in enumerate(shapes):
        o = arr[q]
        o.kind = SHAPE[s["kind"]]
        o.material = s["material"]
        for a in range(3):
            o.center[a] = s["c"][a]
            o.half[a] = s.get("half", (0, 0, 0))[a]
        o.radius = s.get("radius", 0)
        o.side = s.get("side", 0)
        o.tip_base, o.tip_height = s.get("tip_base", 0), s.get("tip_height", 0)
        o.tip_radius, o.tip_center, o.tip_cut = s.get("tip_radius", 0), s.get("tip_center", 0), s.get("tip_cut", 0)
    return arr, len(shapes)


def make_source(s) -> nlf_source:
    o = nlf_source()
    o.axis_prop, o.axis_pol = 2, 0
    for a in range(3):
        o.tf_lo[a], o.tf_hi[a] = s["tf_lo"][a], s["tf_hi"][a]
    o.waveform = WAVE[s.get("waveform", "gaussian")]
    o.w0, o.tau, o.t0, o.amplitude = s["w0"], s.get("tau", 0.0), s.get("t0", 0.0), s.get("amp", 1.0)
    return o


def make_monitors(m, block_b=32):
    omega = np.ascontiguousarray(m["omega"], dtype=np.float64)
    o = nlf_monitors()
    o.nf = len(omega)
    o.omega = omega.ctypes.data_as(C.POINTER(C.c_double))
    for a in range(3):
        o.abs_lo[a], o.abs_hi[a] = m["abs_lo"][a], m["abs_hi"][a]
        o.sca_lo[a], o.sca_hi[a] = m["sca_lo"][a], m["sca_hi"][a]
    o.decimate_k = m.get("K", 16)
    o.block_b = block_b
    return o, omega


# ------------------------------------------------------------------ Solver

class Solver:
    """One configured context (nlf_create + nlf_set_*) for a problem dict."""

    def __init__(self, prob: dict, material_map=None, block_b: int = 32):
        require_gpu()
        L = load()
        self.L = L
        self.prob = prob
        h = C.c_void_p()
        g = make_grid(prob)
        rc = L.nlf_create(C.byref(g), C.byref(h))
        if rc != NLF_OK:
            raise NLFError(rc, "nlf_create")
        self.h = h
        mats, nm = make_materials(prob)
        _check(h, L.nlf_set_materials(h, mats, nm))
        if material_map is not None and hasattr(material_map, "data_ptr"):
            # a device-resident map (a torch uint8 tensor on the GPU)
            self._map = material_map
            _check(h, L.nlf_set_material_map(h, C.c_void_p(material_map.data_ptr()), 1))
        elif material_map is not None:
            self._map = np.ascontiguousarray(material_map, dtype=np.uint8)
            _check(h, L.nlf_set_material_map(h, self._map.ctypes.data, 0))
        else:
            shp, ns = make_shapes(prob)
            _check(h, L.nlf_set_shapes(h, shp, ns))
        if prob.get("source") is not None:
            src = make_source(prob["source"])
            _check(h, L.nlf_set_source(h, C.byref(src)))
        if prob.get("monitors") is not None:
            mon, self._omega = make_monitors(prob["monitors"], block_b)
            _check(h, L.nlf_set_monitors(h, C.byref(mon)))
        self.shape3 = tuple(reversed(prob["shape"]))
        self.nf = len(prob["monitors"]["omega"]) if prob.get("monitors") is not None else 0
        pm = prob.get("plane_map")
        if pm is not None:
            # {"axis", "index", "omega", "K"}: single-frequency maps on one plane
            self._pl_omega = np.ascontiguousarray(pm["omega"], dtype=np.float64)
            m = nlf_plane_monitor(int(pm["axis"]), int(pm["index"]), len(self._pl_omega),
                                  self._pl_omega.ctypes.data_as(C.POINTER(C.c_double)), int(pm["K"]))
            _check(h, L.nlf_set_plane_monitor(h, C.byref(m)))
            nz, ny, nx = self.shape3
            a = int(pm["axis"])
            self._pl_ext = (nz, ny) if a == 0 else ((nz, nx) if a == 1 else (ny, nx))

    def close(self):
        if getattr(self, "h", None):
            self.L.nlf_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def plane_map(self, which) -> np.ndarray:
        """Complex [nf][n1][n2] plane map: "Ex", "Ey", "Ez" or "density"."""
        code = {"Ex": 0, "Ey": 1, "Ez": 2, "density": NLF_MAP_DENSITY}[which]
        n1, n2 = self._pl_ext
        out = np.zeros((len(self._pl_omega), n1, n2, 2))
        _check(self.h, self.L.nlf_get_plane_map(self.h, code, out.ctypes.data_as(C.POINTER(C.c_double))))
        return out[..., 0] + 1j * out[..., 1]

    def state_bytes(self) -> int:
        return int(self.L.nlf_state_bytes(self.h))

    def bind_state(self, ptr: int, nbytes: int):
        _check(self.h, self.L.nlf_bind_state(self.h, C.c_void_p(ptr), nbytes))

    def run(self, steps: int, stream=None):
        s = C.c_void_p(int(stream) if stream is not None else 0)
        _check(self.h, self.L.nlf_run(self.h, int(steps), s))

    def time_kernels(self, steps: int, stream=None) -> dict:
        """Advance `steps` steps (replayed as one CUDA graph) with CUDA events
        around each kernel; summed device ms per kernel class."""
        s = C.c_void_p(int(stream) if stream is not None else 0)
        ms = (C.c_double * 3)()
        _check(self.h, self.L.nlf_time_kernels(self.h, int(steps), s, ms))
        return {"step_ms": ms[0], "metal_ms": ms[1], "dft_ms": ms[2]}

    def reset(self, stream=None):
        s = C.c_void_p(int(stream) if stream is not None else 0)
        _check(self.h, self.L.nlf_reset(self.h, s))

    def sync(self, timeout_ms: int = -1):
        _check(self.h, self.L.nlf_sync(self.h, timeout_ms))

    def field(self, name: str) -> np.ndarray:
        out = np.empty(self.shape3, dtype=np.float32)
        _check(self.h, self.L.nlf_get_field(self.h, FIELD[name], out.ctypes.data, 0))
        return out

    def set_field(self, name: str, values):
        """Set E^n or H^{n-1/2} ("Ex".."Hz", SI) from a [nz][ny][nx] array."""
        a = np.ascontiguousarray(values, dtype=np.float32)
        assert a.shape == self.shape3
        _check(self.h, self.L.nlf_set_field(self.h, FIELD[name], a.ctypes.data, 0))

    def field_to_device(self, name: str, dst_ptr: int):
        _check(self.h, self.L.nlf_get_field(self.h, FIELD[name], C.c_void_p(dst_ptr), 1))

    def voxels(self) -> np.ndarray:
        out = np.empty((3,) + self.shape3, dtype=np.uint8)
        _check(self.h, self.L.nlf_get_voxels(self.h, out.ctypes.data))
        return out

    def spectra(self):
        nf = self.nf
        ext, ab, sc = np.empty(nf), np.empty(nf), np.empty(nf)
        _check(self.h, self.L.nlf_get_spectra(self.h, ext.ctypes.data, ab.ctypes.data, sc.ctypes.data))
        return {"ext": ext, "abs": ab, "sca": sc}

    def flux_weights(self):
        """Signed face weights of the flux records and the absorption-box record count."""
        nr = int(self.L.nlf_num_records(self.h))
        coef = np.empty(nr)
        n_abs = C.c_longlong()
        _check(self.h, self.L.nlf_get_flux_weights(self.h, coef.ctypes.data, C.byref(n_abs)))
        return coef, int(n_abs.value)

    def dft(self):
        nr = int(self.L.nlf_num_records(self.h))
        buf = np.empty((2, nr + 1, self.nf, 2))
        _check(self.h, self.L.nlf_get_dft(self.h, buf.ctypes.data))
        return buf[0], buf[1]

    def save_state(self) -> np.ndarray:
        buf = np.empty(self.state_bytes(), dtype=np.uint8)
        _check(self.h, self.L.nlf_save_state(self.h, buf.ctypes.data))
        return buf

    def load_state(self, buf: np.ndarray):
        buf = np.ascontiguousarray(buf, dtype=np.uint8)
        _check(self.h, self.L.nlf_load_state(self.h, buf.ctypes.data))

    @property
    def n(self) -> int:
        return int(self.L.nlf_time_index(self.h))

    def info(self) -> dict:
        i = nlf_info()
        _check(self.h, self.L.nlf_get_info(self.h, C.byref(i)))
        return {k: getattr(i, k) for k, _ in nlf_info._fields_}

    @property
    def launches(self) -> int:
        return int(self.L.nlf_kernel_launches(self.h))


def batch_run(solvers, steps, stream=None):
    """nlf_batch_run over several Solver objects; returns per-context status codes."""
    L = load()
    n = len(solvers)
    hs = (C.c_void_p * n)(*[s.h.value for s in solvers])
    st = (C.c_longlong * n)(*[int(x) for x in steps])
    status = (C.c_int * n)()
    s = C.c_void_p(int(stream) if stream is not None else 0)
    L.nlf_batch_run(hs, n, st, s, status)
    return list(status)
