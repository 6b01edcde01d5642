"""Thin ctypes binding of the lsb C ABI (include/lsb.h).

Argument marshalling only: every step of the method runs in the CUDA library
``_lib/liblsb.so``.  Importing this module does not need a GPU; creating a
Grid does, and fails loudly when the library or the device is missing (there
is no CPU fallback).  PyTorch is used only to hold the initial level set in
device memory and to hand over CUDA streams.
"""
import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.environ.get("LSB_LIBRARY") or os.path.join(HERE, "_lib", "liblsb.so")

D2Q9, D3Q19, D3Q27 = 0, 1, 2
BGK, CUMULANT = 0, 1
PERIODIC, WALL, SLIP = 0, 1, 2
FP32, FP16S = 0, 1
SENSOR_BAND, SENSOR_SIGNED = 0, 1
FIELD = dict(rho=0, u=1, phi=2, phase=3, f=4, tag=5, blocks=6, cutmask=7, kappa=8, uext=9, adj_f=10, adj_uext=11)
NPARAM_ADJ = 5  # sigma, rho[0], rho[1], nu[0], nu[1]
STATUS = {0: "LSB_OK", 1: "LSB_EINVAL", 2: "LSB_ENOMEM", 3: "LSB_ECUDA", 4: "LSB_EUNSTABLE",
          5: "LSB_ETIMEOUT", 6: "LSB_ESTATE"}


class GridDesc(ctypes.Structure):
    _fields_ = [("lattice", ctypes.c_int), ("base", ctypes.c_int * 3), ("n_levels", ctypes.c_int),
                ("block", ctypes.c_int * 3), ("bc", ctypes.c_int * 3), ("wall_u", (ctypes.c_double * 3) * 6),
                ("storage", ctypes.c_int), ("fp16_scale", ctypes.c_double), ("collision", ctypes.c_int * 2)]


class Params(ctypes.Structure):
    _fields_ = [("rho", ctypes.c_double * 2), ("nu", ctypes.c_double * 2), ("body_force", ctypes.c_double * 3),
                ("gravity", ctypes.c_double * 3), ("sigma", ctypes.c_double), ("x_ref", ctypes.c_double * 3),
                ("p_gas0", ctypes.c_double),
                ("n_ext", ctypes.c_int), ("dtau_ext", ctypes.c_double), ("reinit_every", ctypes.c_int),
                ("n_reinit", ctypes.c_int), ("dtau_reinit", ctypes.c_double), ("refine_dist", ctypes.c_double * 4),
                ("sensor", ctypes.c_int), ("regrid_every", ctypes.c_int), ("ls_active", ctypes.c_int)]


class LsbError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


_lib = None


def load():
    """Load liblsb.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} missing: build it with paper_2601_05936_gb300.build.build()")
    lib = ctypes.CDLL(LIB_PATH)
    vp = ctypes.c_void_p
    lib.lsb_create_grid.argtypes = [ctypes.c_int, ctypes.POINTER(GridDesc), ctypes.POINTER(Params),
                                    ctypes.POINTER(ctypes.c_void_p), vp, ctypes.POINTER(vp)]
    lib.lsb_set_params.argtypes = [vp, ctypes.c_int, ctypes.POINTER(Params)]
    lib.lsb_step.argtypes = [vp, ctypes.c_int]
    lib.lsb_use_graphs.argtypes = [vp, ctypes.c_int]
    lib.lsb_refine.argtypes = [vp]
    lib.lsb_get_fields.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, vp, ctypes.c_size_t, ctypes.c_int]
    lib.lsb_get_fields_noalloc.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, vp, ctypes.c_size_t,
                                           ctypes.c_int]
    lib.lsb_field_bytes.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int]
    lib.lsb_field_bytes.restype = ctypes.c_size_t
    lib.lsb_observables.argtypes = [vp, ctypes.POINTER(ctypes.c_double), ctypes.c_size_t]
    lib.lsb_cell_updates.argtypes = [vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
    lib.lsb_backward.argtypes = [vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double), vp]
    lib.lsb_record.argtypes = [vp, ctypes.c_int]
    lib.lsb_set_driver.argtypes = [vp, ctypes.c_int]
    lib.lsb_set_wait_limit.argtypes = [vp, ctypes.c_longlong]
    lib.lsb_set_objective.argtypes = [vp, ctypes.c_double]
    lib.lsb_work_counts.argtypes = [vp, ctypes.c_int, ctypes.POINTER(ctypes.c_longlong), ctypes.c_int]
    lib.lsb_autotune.argtypes = [ctypes.c_int, ctypes.POINTER(GridDesc), ctypes.POINTER(Params),
                                 ctypes.POINTER(ctypes.c_void_p), vp, ctypes.POINTER(ctypes.c_int), ctypes.c_int,
                                 ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)]
    lib.lsb_sync.argtypes = [vp]
    lib.lsb_kernel_launches.argtypes = [vp]
    lib.lsb_kernel_launches.restype = ctypes.c_uint64
    lib.lsb_last_error.argtypes = [vp]
    lib.lsb_last_error.restype = ctypes.c_char_p
    lib.lsb_destroy.argtypes = [vp]
    lib.lsb_destroy.restype = None
    lib.lsb_lattice_table.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_float),
                                      ctypes.POINTER(ctypes.c_int)]
    lib.lsb_profile.argtypes = [vp, ctypes.c_int]
    lib.lsb_profile_read.argtypes = [vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                                     ctypes.POINTER(ctypes.c_uint64), ctypes.c_int]
    lib.lsb_kernel_name.argtypes = [ctypes.c_int]
    lib.lsb_kernel_name.restype = ctypes.c_char_p
    lib.lsb_kernel_count.argtypes = []
    lib.lsb_kernel_count.restype = ctypes.c_int
    for name in ("lsb_use_graphs", "lsb_get_fields_noalloc", "lsb_profile", "lsb_profile_read", "lsb_create_grid", "lsb_set_params", "lsb_step", "lsb_refine", "lsb_get_fields",
                 "lsb_observables", "lsb_cell_updates", "lsb_backward", "lsb_record", "lsb_autotune", "lsb_set_driver", "lsb_sync",
                 "lsb_set_wait_limit", "lsb_work_counts", "lsb_set_objective"):
        getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib


def lattice_table(lattice):
    """(c (Q,3) int, w (Q,) float32, opp (Q,) int) compiled into the library."""
    lib = load()
    c = (ctypes.c_int * 81)()
    w = (ctypes.c_float * 27)()
    o = (ctypes.c_int * 27)()
    Q = lib.lsb_lattice_table(lattice, c, w, o)
    return (np.ctypeslib.as_array(c)[:3 * Q].reshape(Q, 3).copy(), np.ctypeslib.as_array(w)[:Q].copy(),
            np.ctypeslib.as_array(o)[:Q].copy())


def _desc(case):
    D = 2 if case["lattice"] == "D2Q9" else 3
    d = GridDesc()
    d.lattice = {"D2Q9": D2Q9, "D3Q19": D3Q19, "D3Q27": D3Q27}[case["lattice"]]
    for k, op in enumerate(case.get("collision", ("bgk", "bgk"))):
        d.collision[k] = {"bgk": BGK, "cumulant": CUMULANT}[op]
    for a in range(3):
        d.base[a] = int(case["base"][a]) if a < D else 1
        d.block[a] = int(case["block"][a]) if a < D else 1
        slip = bool((case.get("slip") or (False,) * D)[a]) if a < D else False
        d.bc[a] = (PERIODIC if case["periodic"][a] else (SLIP if slip else WALL)) if a < D else PERIODIC
    d.n_levels = int(case.get("n_levels", 1))
    wu = np.zeros((6, 3))
    if case.get("wall_u") is not None:
        w = np.asarray(case["wall_u"], float).reshape(2 * D, D)
        wu[:2 * D, :D] = w
    for f in range(6):
        for a in range(3):
            d.wall_u[f][a] = wu[f, a]
    d.storage = FP16S if case.get("storage", "fp32") == "fp16s" else FP32
    d.fp16_scale = float(case.get("fp16_scale", 1024.0))
    return d, D


def _params(case, D):
    p = Params()
    for k in range(2):
        p.rho[k] = float(case["rho_phys"][k])
        p.nu[k] = float(case["nu"][k])
    for name in ("body_force", "gravity", "x_ref"):
        v = case.get(name)
        v = np.zeros(D) if v is None else np.asarray(v, float)
        for a in range(3):
            getattr(p, name)[a] = float(v[a]) if a < D else 0.0
    p.sigma = float(case.get("sigma", 0.0))
    p.p_gas0 = float(case.get("p_gas0", 0.0))
    p.n_ext = int(case.get("n_ext", 8))
    p.dtau_ext = float(case.get("dtau_ext", 0.5))
    p.reinit_every = int(case.get("reinit_every", 1))
    p.n_reinit = int(case.get("n_reinit", 1))
    p.dtau_reinit = float(case.get("dtau_reinit", 0.3))
    rd = case.get("refine_dist")
    L = int(case.get("n_levels", 1))
    rd = [8.0] * max(L - 1, 0) if rd is None else list(rd)
    for l in range(4):
        p.refine_dist[l] = float(rd[l]) if l < len(rd) else 0.0
    p.sensor = SENSOR_SIGNED if case.get("sensor", "band") == "signed" else SENSOR_BAND
    p.regrid_every = int(case.get("regrid_every", 0))
    p.ls_active = 1 if case.get("ls_active", True) else 0
    return p


def _marshal(cases, device):
    """ctypes arrays of descriptors and parameters, and the device copies of phi0."""
    import torch

    if not torch.cuda.is_available():
        raise RuntimeError("lsb needs a CUDA device; there is no CPU fallback")
    n = len(cases)
    descs = (GridDesc * n)()
    params = (Params * n)()
    D = None
    phis = []
    for c, case in enumerate(cases):
        d, D = _desc(case)
        descs[c] = d
        params[c] = _params(case, D)
        phis.append(torch.as_tensor(np.ascontiguousarray(np.asarray(case["phi0"], np.float32).reshape(-1)),
                                    device=f"cuda:{device}"))
    ptrs = (ctypes.c_void_p * n)(*[t.data_ptr() for t in phis])
    return descs, params, ptrs, phis, D


def autotune(cases, candidates=None, steps=10, stream=None, device=0):
    """Time each block shape on these cases (lsb_autotune).  candidates: list of
    (bx, by, bz) or None for the built-in list.  Returns (best shape, {shape: ms per
    coarse step or nan})."""
    lib = load()
    if isinstance(cases, dict):
        cases = [cases]
    descs, params, ptrs, phis, D = _marshal(cases, device)
    if candidates is None:
        cand = None
        nc = 6
        shapes = None
    else:
        shapes = [tuple(int(v) for v in (list(c) + [1, 1])[:3]) for c in candidates]
        nc = len(shapes)
        cand = (ctypes.c_int * (3 * nc))(*[v for sh in shapes for v in sh])
    best = (ctypes.c_int * 3)()
    ms = (ctypes.c_double * nc)()
    sp = ctypes.c_void_p(stream.cuda_stream if stream is not None else 0)
    st = lib.lsb_autotune(len(cases), descs, params, ptrs, sp, cand, nc, int(steps), best, ms)
    if st != 0:
        raise LsbError(st, lib.lsb_last_error(None).decode())
    if shapes is None:
        shapes = [None] * nc
    res = {(sh if sh is not None else k): ms[k] for k, sh in enumerate(shapes)}
    return tuple(best), res


class Grid:
    """One handle of the library: an ensemble of one or more cases.

    ``cases``: list of dicts with the keys of the oracle's case description
    (lattice, base, n_levels, block, periodic, wall_u, rho_phys, nu, body_force,
    gravity, sigma, x_ref, level-set and sensor parameters, phi0 [finest level,
    x fastest]) plus storage ('fp32' | 'fp16s') and fp16_scale.
    """

    def __init__(self, cases, stream=None, device=0):
        self.lib = load()
        if isinstance(cases, dict):
            cases = [cases]
        self.cases = cases
        n = len(cases)
        descs, params, ptrs, self._phi, self.D = _marshal(cases, device)
        self.stream = stream
        sp = ctypes.c_void_p(stream.cuda_stream if stream is not None else 0)
        h = ctypes.c_void_p()
        st = self.lib.lsb_create_grid(n, descs, params, ptrs, sp, ctypes.byref(h))
        if st != 0:
            raise LsbError(st, self.lib.lsb_last_error(None).decode())
        self.h = h
        self.Q = 9 if self.D == 2 else 19

    def _check(self, st):
        if st != 0:
            raise LsbError(st, self.lib.lsb_last_error(self.h).decode())

    def step(self, n=1):
        self._check(self.lib.lsb_step(self.h, int(n)))

    def use_graphs(self, enable=True):
        """Replay coarse steps from CUDA graphs, two per replay and one for an odd remainder
        (needs a non-default stream); results are identical to eager stepping."""
        self._check(self.lib.lsb_use_graphs(self.h, 1 if enable else 0))

    def set_driver(self, mode):
        """0: one launch per level-set pass; 1: one persistent cooperative launch per finest step."""
        self._check(self.lib.lsb_set_driver(self.h, int(mode)))

    def set_objective(self, eps=1.5):
        """Gas indicator of volume, centroid and velocity: 0 sharp, > 0 smoothed H_eps (width eps)."""
        self._check(self.lib.lsb_set_objective(self.h, float(eps)))

    def set_wait_limit(self, spins):
        """Iteration limit of the bounded device-side waits (~64 ns each; 0 gives up at once)."""
        self._check(self.lib.lsb_set_wait_limit(self.h, int(spins)))

    def refine(self):
        self._check(self.lib.lsb_refine(self.h))

    def sync(self):
        self._check(self.lib.lsb_sync(self.h))

    def set_params(self, case, case_idx=-1):
        self._check(self.lib.lsb_set_params(self.h, case_idx, ctypes.byref(_params(case, self.D))))

    def level_dims(self, case_idx=0, level=None):
        c = self.cases[case_idx]
        L = int(c.get("n_levels", 1))
        level = L - 1 if level is None else level
        return tuple(int(b) * 2 ** level for b in c["base"])

    def get(self, field, case_idx=0, level=None):
        """Dense numpy copy of one field: shape (nz,) ny, nx with components first."""
        c = self.cases[case_idx]
        L = int(c.get("n_levels", 1))
        level = L - 1 if level is None else level
        code = FIELD[field]
        nbytes = self.lib.lsb_field_bytes(self.h, case_idx, code, level)
        if nbytes == 0:
            raise LsbError(1, f"field {field} not available on level {level}")
        dt = {"phase": np.uint8, "tag": np.uint8, "blocks": np.int8, "cutmask": np.uint32}.get(field, np.float32)
        out = np.empty(nbytes // np.dtype(dt).itemsize, dtype=dt)
        self._check(self.lib.lsb_get_fields(self.h, case_idx, code, level, out.ctypes.data, nbytes, 1))
        if field == "blocks":
            return out
        dims = self.level_dims(case_idx, level)[::-1]
        ncomp = out.size // int(np.prod(dims))
        return out.reshape((ncomp,) + dims) if ncomp > 1 else out.reshape(dims)

    def get_device(self, field, dst_ptr, nbytes, case_idx=0, level=None):
        """Copy a field into caller device memory (dst_ptr, nbytes)."""
        c = self.cases[case_idx]
        level = int(c.get("n_levels", 1)) - 1 if level is None else level
        self._check(self.lib.lsb_get_fields(self.h, case_idx, FIELD[field], level, ctypes.c_void_p(dst_ptr),
                                            int(nbytes), 0))

    def observables(self):
        """Per case: dict(mass (2,), volume, leaf_cells, centroid (D,), velocity (D,)), float64."""
        D = self.D
        stride = 4 + 2 * D
        buf = (ctypes.c_double * (stride * len(self.cases)))()
        self._check(self.lib.lsb_observables(self.h, buf, len(buf)))
        a = np.ctypeslib.as_array(buf).reshape(len(self.cases), stride).copy()
        return [dict(mass=r[0:2], volume=r[2], leaf_cells=r[3], centroid=r[4:4 + D], velocity=r[4 + D:4 + 2 * D])
                for r in a]

    def cell_updates(self, total=False):
        """Leaf cell updates per coarse step now, or (total=True) done since creation."""
        v = ctypes.c_double()
        t = ctypes.c_double()
        self._check(self.lib.lsb_cell_updates(self.h, ctypes.byref(v), ctypes.byref(t)))
        return t.value if total else v.value

    def profile(self, mode):
        """0 off, 1 time collide-and-stream launches, 2 time every launch."""
        self._check(self.lib.lsb_profile(self.h, int(mode)))

    def profile_read(self):
        """{kernel name: (ms, launches, algorithmic bytes)} since the last profile/read."""
        n = self.lib.lsb_kernel_count()
        ms = (ctypes.c_double * n)()
        by = (ctypes.c_double * n)()
        la = (ctypes.c_uint64 * n)()
        self._check(self.lib.lsb_profile_read(self.h, ms, by, la, n))
        return {self.lib.lsb_kernel_name(k).decode(): (ms[k], int(la[k]), by[k]) for k in range(n) if la[k]}

    def work_counts(self, level):
        """Work-list sizes of global level ``level`` after the last step (lsb_work_counts)."""
        names = ("leaf", "band", "iface", "links", "flipped", "ghost", "restrict")
        out = (ctypes.c_longlong * len(names))()
        self._check(self.lib.lsb_work_counts(self.h, int(level), out, len(names)))
        return dict(zip(names, (int(v) for v in out)))

    def kernel_launches(self):
        return int(self.lib.lsb_kernel_launches(self.h))

    def record(self, checkpoint_every=100):
        """Start recording the following steps for backward (FP32; frozen level set on any number of
        levels, or a moving level set on one level)."""
        self._check(self.lib.lsb_record(self.h, int(checkpoint_every)))

    def backward(self, dJ_dobs, want_phi=False):
        """Reverse sweep over the recorded steps for J = sum of dJ_dobs . observables
        (dJ_dobs: n_cases x (4 + 2 D), observables order).  Returns dJ/dp, shape
        (n_cases, 5): sigma, rho[0], rho[1], nu[0], nu[1]; with ``want_phi`` also
        the list of dJ/dphi arrays (finest level of each case, shape (nz,) ny, nx)."""
        import torch
        w = np.ascontiguousarray(np.asarray(dJ_dobs, dtype=np.float64).reshape(-1))
        nc = len(self.cases)
        if w.size != nc * (4 + 2 * self.D):
            raise ValueError("dJ_dobs needs n_cases x (4 + 2 D) values")
        out = np.zeros(nc * NPARAM_ADJ, dtype=np.float64)
        dims = [self.level_dims(k)[::-1] for k in range(nc)]
        dphi = None
        if want_phi:
            dphi = torch.zeros(sum(int(np.prod(d)) for d in dims), dtype=torch.float32,
                               device=torch.cuda.current_device())
        self._check(self.lib.lsb_backward(self.h, w.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                          out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                          ctypes.c_void_p(dphi.data_ptr()) if want_phi else None))
        dp = out.reshape(nc, NPARAM_ADJ)
        if not want_phi:
            return dp
        h = dphi.cpu().numpy()
        res, o = [], 0
        for d in dims:
            m = int(np.prod(d))
            res.append(h[o:o + m].reshape(d))
            o += m
        return dp, res

    def close(self):
        if getattr(self, "h", None):
            self.lib.lsb_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
