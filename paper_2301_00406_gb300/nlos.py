"""Thin ctypes binding of the C ABI in include/nlos.h (libnlos.so).

Argument marshalling only: every operation runs in the library's CUDA
kernels.  Device buffers are passed as raw pointers (``tensor.data_ptr()``)
and streams as ``cudaStream_t`` handles (``torch.cuda.current_stream().cuda_stream``).
If the library has not been built, ``load()`` raises: there is no fallback.
"""

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libnlos.so")

NLOS_OK = 0
STATUS_NAMES = {0: "NLOS_OK", -1: "NLOS_ERR_INVALID_ARG", -2: "NLOS_ERR_OOM", -3: "NLOS_ERR_CUDA",
                -4: "NLOS_ERR_BUSY", -5: "NLOS_ERR_NOT_READY", -6: "NLOS_ERR_TIMEOUT",
                -7: "NLOS_ERR_DIVERGED"}
globals().update({name: code for code, name in STATUS_NAMES.items()})
RADIOMETRY = {"compensated": 0, "raw": 1}
# curvature weights phi(kappa) (NLOS_PHI_*): a + b kappa^2, a + b |kappa|, sqrt(a + b kappa^2)
LATERAL_FFT, LATERAL_GEMM_BF16X3, LATERAL_GEMM_BF16 = 0, 1, 2
PHI_TSC, PHI_TAC, PHI_TRV = 0, 1, 2
INIT_ZERO, INIT_BACKPROJECT = 0, 1
PHI = {"tsc": 0, "tac": 1, "trv": 2}


class Geometry(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nt", ctypes.c_int32),
                ("bin_width_s", ctypes.c_double), ("wall_width_m", ctypes.c_double),
                ("radiometry", ctypes.c_int32), ("mask", ctypes.POINTER(ctypes.c_uint8))]


class Params(ctypes.Structure):
    _fields_ = [("model", ctypes.c_int32), ("phi", ctypes.c_int32),
                ("a", ctypes.c_double), ("b", ctypes.c_double), ("mu", ctypes.c_double),
                ("a_u", ctypes.c_double), ("b_u", ctypes.c_double), ("a_tau", ctypes.c_double),
                ("b_tau", ctypes.c_double), ("lambda_", ctypes.c_double),
                ("mu1", ctypes.c_double), ("mu2", ctypes.c_double), ("mu3", ctypes.c_double),
                ("iters", ctypes.c_int32), ("eps_stop", ctypes.c_double), ("L0", ctypes.c_double),
                ("eta", ctypes.c_double), ("max_backtracks", ctypes.c_int32),
                ("eps_normal", ctypes.c_double), ("restart", ctypes.c_int32),
                ("warm_start_iters", ctypes.c_int32), ("init", ctypes.c_int32)]


class Stats(ctypes.Structure):
    _fields_ = [("iters_done", ctypes.c_int32), ("backtracks", ctypes.c_int32),
                ("restarts", ctypes.c_int32), ("status", ctypes.c_int32),
                ("L", ctypes.c_double), ("energy", ctypes.c_double), ("rel_change", ctypes.c_double),
                ("data_fit", ctypes.c_double), ("primal_res", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class NlosError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


_lib = None

# name -> (restype, argtypes)
_P = ctypes.c_void_p
_SIGS = {
    "nlos_last_error": (ctypes.c_int32, [ctypes.c_char_p, ctypes.c_size_t]),
    "nlos_version": (ctypes.c_int32, []),
    "nlos_params_default": (ctypes.c_int32, [ctypes.c_int32, ctypes.POINTER(Params)]),
    "nlos_plan_create": (ctypes.c_int32, [ctypes.POINTER(Geometry), _P, ctypes.POINTER(_P)]),
    "nlos_plan_destroy": (ctypes.c_int32, [_P]),
    "nlos_plan_norm2": (ctypes.c_int32, [_P, ctypes.c_int32, _P, ctypes.POINTER(ctypes.c_double)]),
    "nlos_geometry_tables": (ctypes.c_int32, [ctypes.POINTER(Geometry), _P, _P, _P, _P, _P,
                                              ctypes.POINTER(ctypes.c_int32)]),
    "nlos_forward": (ctypes.c_int32, [_P, _P, _P, ctypes.c_int32, _P]),
    "nlos_adjoint": (ctypes.c_int32, [_P, _P, _P, ctypes.c_int32, _P]),
    "nlos_solve": (ctypes.c_int32, [_P, _P, _P, ctypes.c_double, ctypes.c_double, _P]),
    "nlos_curvature_weight": (ctypes.c_int32, [_P, _P, _P, ctypes.c_double, ctypes.c_double,
                                               ctypes.c_int32, ctypes.c_double, _P]),
    "nlos_reconstruct": (ctypes.c_int32, [_P, ctypes.POINTER(Params), _P, _P, _P,
                                          ctypes.POINTER(Stats), _P]),
    "nlos_forward_directional": (ctypes.c_int32, [_P, _P, _P, _P, ctypes.c_int32, _P]),
    "nlos_adjoint_directional": (ctypes.c_int32, [_P, _P, _P, _P, ctypes.c_int32, _P]),
    "nlos_reconstruct_host": (ctypes.c_int32, [_P, ctypes.POINTER(Params), _P, _P, _P, ctypes.POINTER(Stats), _P]),
    "nlos_reconstruct_prepare": (ctypes.c_int32, [_P, ctypes.POINTER(Params), _P, _P, _P,
                                                  ctypes.POINTER(ctypes.c_int32), _P]),
    "nlos_solve_static": (ctypes.c_int32, [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, _P, _P,
                                           ctypes.c_double, ctypes.c_double, _P]),
    "nlos_reconstruct_batch": (ctypes.c_int32, [_P, ctypes.POINTER(Params), _P, _P, _P, ctypes.c_int32,
                                                ctypes.POINTER(Stats), _P]),
    "nlos_server_create": (ctypes.c_int32, [ctypes.c_size_t, ctypes.c_int32, ctypes.POINTER(_P)]),
    "nlos_submit": (ctypes.c_int32, [_P, ctypes.POINTER(Geometry), ctypes.POINTER(Params), _P, _P,
                                     ctypes.POINTER(ctypes.c_uint64)]),
    "nlos_poll": (ctypes.c_int32, [_P, ctypes.c_uint64, ctypes.POINTER(Stats)]),
    "nlos_wait": (ctypes.c_int32, [_P, ctypes.c_uint64, ctypes.c_double, ctypes.POINTER(Stats)]),
    "nlos_job_times": (ctypes.c_int32, [_P, ctypes.c_uint64, ctypes.POINTER(ctypes.c_double),
                                        ctypes.POINTER(ctypes.c_double)]),
    "nlos_server_info": (ctypes.c_int32, [_P, _P]),
    "nlos_server_prepare": (ctypes.c_int32, [_P, ctypes.POINTER(Geometry), ctypes.POINTER(Params), ctypes.c_int32,
                                             ctypes.c_double, ctypes.POINTER(ctypes.c_int32)]),
    "nlos_server_destroy": (ctypes.c_int32, [_P, ctypes.c_int32, ctypes.c_double]),
    "nlos_midpoint_confocal": (ctypes.c_int32, [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_double,
                                                ctypes.c_double, ctypes.c_double, ctypes.c_double, _P, _P, _P]),
    "nlos_selftest_wait_timeout": (ctypes.c_int32, [ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p]),
    "nlos_timing_enable": (ctypes.c_int32, [_P, ctypes.c_int32]),
    "nlos_plan_set_lateral": (ctypes.c_int32, [_P, ctypes.c_int32, _P]),
    "nlos_timing_read": (ctypes.c_int32, [_P, _P, _P, ctypes.c_int32]),
}

TIMING_CATEGORIES = ["k_conv", "k_tfwd", "k_tinv", "k_tadj", "k_sxy", "k_sfwd", "k_sinv", "k_pre", "k_post",
                     "small", "k_kspec"]


def exported_symbols():
    """Names of the entry points the binding expects (those declared in include/nlos.h)."""
    return list(_SIGS)


def load(path=LIB_PATH):
    """Load libnlos.so and declare the signatures; raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it first (python -c 'import __graft_entry__ as g; g.build()')")
    lib = ctypes.CDLL(path)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def last_error():
    buf = ctypes.create_string_buffer(1024)
    load().nlos_last_error(buf, len(buf))
    return buf.value.decode(errors="replace")


def check(status):
    if status != NLOS_OK:
        raise NlosError(status, last_error())
    return status


def _geometry(nx, ny, nt, bin_width_s, wall_width_m, radiometry, mask):
    g = Geometry(nx, ny, nt, bin_width_s, wall_width_m, RADIOMETRY[radiometry], None)
    keep = None
    if mask is not None:
        keep = np.ascontiguousarray(np.asarray(mask, dtype=np.uint8).reshape(nx * ny))
        g.mask = keep.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))
    return g, keep


def geometry_tables(nx, ny, nt, bin_width_s, wall_width_m=1.0, radiometry="compensated", mask=None):
    """Host-side R_z / R_t^{-1} tables and the sampled-column list (no GPU needed)."""
    g, _keep = _geometry(nx, ny, nt, bin_width_s, wall_width_m, radiometry, mask)
    rz_i0 = np.zeros(nt, np.int32)
    rt_k0 = np.zeros(nt, np.int32)
    rz_w = np.zeros(3 * nt, np.float32)
    rt_w = np.zeros(3 * nt, np.float32)
    cols = np.zeros(nx * ny, np.int32)
    n = ctypes.c_int32()
    check(load().nlos_geometry_tables(ctypes.byref(g), rz_i0.ctypes.data, rz_w.ctypes.data, rt_k0.ctypes.data,
                                      rt_w.ctypes.data, cols.ctypes.data, ctypes.byref(n)))
    return {"rz_i0": rz_i0, "rz_w": rz_w.reshape(nt, 3), "rt_k0": rt_k0, "rt_w": rt_w.reshape(nt, 3),
            "cols": cols[: n.value]}


def params_default(model):
    p = Params()
    check(load().nlos_params_default(model, ctypes.byref(p)))
    return p


class Plan:
    """Owns an nlos_plan.  ``mask`` is an (nx, ny) uint8 array (nonzero = sampled) or None."""

    def __init__(self, nx, ny, nt, bin_width_s, wall_width_m=1.0, radiometry="compensated", mask=None, stream=0):
        lib = load()
        self.shape = (nx, ny, nt)
        g, self._mask = _geometry(nx, ny, nt, bin_width_s, wall_width_m, radiometry, mask)
        h = _P()
        check(lib.nlos_plan_create(ctypes.byref(g), stream, ctypes.byref(h)))
        self.handle = h

    def close(self):
        if getattr(self, "handle", None):
            load().nlos_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def norm2(self, masked=True, stream=0):
        out = ctypes.c_double()
        check(load().nlos_plan_norm2(self.handle, int(masked), stream, ctypes.byref(out)))
        return out.value

    def set_lateral(self, mode, stream=0):
        """Lateral stage: 0 FFT kernels, 1 split-BF16 tensor-core DFT products, 2 single-BF16 ones."""
        check(load().nlos_plan_set_lateral(self.handle, int(mode), stream))

    def timing_enable(self, enable=True):
        check(load().nlos_timing_enable(self.handle, int(enable)))

    def timing_read(self):
        n = len(TIMING_CATEGORIES)
        ms = np.zeros(n, np.float64)
        cnt = np.zeros(n, np.int32)
        check(load().nlos_timing_read(self.handle, ms.ctypes.data, cnt.ctypes.data, n))
        return {k: (float(ms[i]), int(cnt[i])) for i, k in enumerate(TIMING_CATEGORIES)}

    # raw-pointer entry points (same names as the C ABI)
    def forward(self, u_ptr, tau_ptr, apply_mask, stream=0):
        check(load().nlos_forward(self.handle, u_ptr, tau_ptr, int(apply_mask), stream))

    def adjoint(self, tau_ptr, u_ptr, apply_mask, stream=0):
        check(load().nlos_adjoint(self.handle, tau_ptr, u_ptr, int(apply_mask), stream))

    def solve(self, rhs_ptr, x_ptr, c0, c1, stream=0):
        check(load().nlos_solve(self.handle, rhs_ptr, x_ptr, c0, c1, stream))

    def curvature_weight(self, u_ptr, phi_ptr, a, b, phi_kind=0, eps=1e-6, stream=0):
        check(load().nlos_curvature_weight(self.handle, u_ptr, phi_ptr, a, b, phi_kind, eps, stream))

    def reconstruct_prepare(self, params, tau0_ptr, u_ptr, tau_out_ptr=0, stream=0):
        """Capture the graph reconstruct() would launch for these arguments; True when one is cached."""
        g = ctypes.c_int32(0)
        check(load().nlos_reconstruct_prepare(self.handle, ctypes.byref(params), tau0_ptr, u_ptr,
                                              tau_out_ptr or None, ctypes.byref(g), stream))
        return bool(g.value)

    def reconstruct_host(self, params, tau0_ptr, u_ptr, tau_out_ptr=0, stream=0):
        """nlos_reconstruct_host on host pointers (e.g. numpy arrays' or pinned tensors' data pointers)."""
        st = Stats()
        check(load().nlos_reconstruct_host(self.handle, ctypes.byref(params), tau0_ptr, u_ptr, tau_out_ptr or None,
                                           ctypes.byref(st), stream))
        return st.as_dict()

    def reconstruct(self, params, tau0_ptr, u_ptr, tau_out_ptr=0, stream=0):
        st = Stats()
        status = load().nlos_reconstruct(self.handle, ctypes.byref(params), tau0_ptr, u_ptr, tau_out_ptr or None,
                                         ctypes.byref(st), stream)
        check(status)
        return st.as_dict()


def reconstruct_batch(plans, params, tau0_ptrs, u_ptrs, tau_out_ptrs=None, stream=0):
    """nlos_reconstruct_batch over lists of plans / params / device pointers; returns per-scene stats."""
    n = len(plans)
    hs = (_P * n)(*[p.handle for p in plans])
    ps = (Params * n)(*params)
    t0 = (_P * n)(*tau0_ptrs)
    uo = (_P * n)(*u_ptrs)
    to = (_P * n)(*tau_out_ptrs) if tau_out_ptrs is not None else None
    st = (Stats * n)()
    check(load().nlos_reconstruct_batch(hs, ps, t0, uo, to, n, st, stream))
    return [s.as_dict() for s in st]


class Server:
    """nlos_server: asynchronous, continuously batched reconstructions from host buffers."""

    INFO = ["queued", "running", "completed", "failed", "peak_running", "bytes_in_use", "bytes_peak", "budget"]

    def __init__(self, hbm_budget_bytes, max_slots):
        h = _P()
        check(load().nlos_server_create(int(hbm_budget_bytes), int(max_slots), ctypes.byref(h)))
        self.handle = h
        self._keep = {}

    def submit(self, nx, ny, nt, bin_width_s, params, tau0, u_out, wall_width_m=1.0, radiometry="compensated",
               mask=None):
        """tau0: float32 C-contiguous numpy array (copied at submit); u_out: float32 numpy array written when done."""
        g, keep = _geometry(nx, ny, nt, bin_width_s, wall_width_m, radiometry, mask)
        tau0 = np.ascontiguousarray(tau0, dtype=np.float32)
        assert u_out.dtype == np.float32 and u_out.flags["C_CONTIGUOUS"] and u_out.size == tau0.size
        jid = ctypes.c_uint64()
        check(load().nlos_submit(self.handle, ctypes.byref(g), ctypes.byref(params), tau0.ctypes.data,
                                 u_out.ctypes.data, ctypes.byref(jid)))
        self._keep[jid.value] = u_out   # the caller's buffer must outlive the job
        return jid.value

    def prepare(self, nx, ny, nt, bin_width_s, params, contexts=1, timeout_s=600.0, wall_width_m=1.0,
                radiometry="compensated", mask=None):
        """nlos_server_prepare: build the geometry's plan and `contexts` idle job contexts with the
        graph of `params` captured; returns how many contexts are ready."""
        g, keep = _geometry(nx, ny, nt, bin_width_s, wall_width_m, radiometry, mask)
        ready = ctypes.c_int32()
        check(load().nlos_server_prepare(self.handle, ctypes.byref(g), ctypes.byref(params), int(contexts),
                                         float(timeout_s), ctypes.byref(ready)))
        return ready.value

    def poll(self, job_id):
        st = Stats()
        s = load().nlos_poll(self.handle, job_id, ctypes.byref(st))
        if s == -5:
            return None
        check(s)
        return st.as_dict()

    def wait(self, job_id, timeout_s=60.0):
        st = Stats()
        s = load().nlos_wait(self.handle, job_id, timeout_s, ctypes.byref(st))
        if s == -5:
            return None
        check(s)
        self._keep.pop(job_id, None)
        return st.as_dict()

    def job_times(self, job_id):
        q, t = ctypes.c_double(), ctypes.c_double()
        check(load().nlos_job_times(self.handle, job_id, ctypes.byref(q), ctypes.byref(t)))
        return q.value, t.value

    def info(self):
        out = np.zeros(8, np.int64)
        check(load().nlos_server_info(self.handle, out.ctypes.data))
        return dict(zip(self.INFO, out.tolist()))

    def close(self, cancel_pending=False, timeout_s=120.0):
        if getattr(self, "handle", None):
            s = load().nlos_server_destroy(self.handle, int(cancel_pending), timeout_s)
            self.handle = None
            check(s)

    def __del__(self):
        try:
            self.close(cancel_pending=True, timeout_s=10.0)
        except Exception:
            pass


# ---------------------------------------------------------------------------
# torch conveniences: allocate outputs with torch and pass pointers/streams
# ---------------------------------------------------------------------------

def _stream():
    import torch
    return torch.cuda.current_stream().cuda_stream


def midpoint_confocal(nx, ny, nt, bin_width_s, wall_width_m, laser_xy, tau_nc_ptr, tau_c_ptr, stream=0):
    """nlos_midpoint_confocal: confocal transients at the midpoints of the detector grid and the laser point
    from non-confocal ones (device pointers, [nx][ny][nt] float32); the result is a confocal scan of wall
    width wall_width_m / 2 centred at laser_xy / 2."""
    check(load().nlos_midpoint_confocal(int(nx), int(ny), int(nt), float(bin_width_s), float(wall_width_m),
                                        float(laser_xy[0]), float(laser_xy[1]), tau_nc_ptr, tau_c_ptr, stream))


def midpoint_confocal_t(tau_nc, bin_width_s, wall_width_m, laser_xy):
    """Torch convenience: tau_nc a [nx][ny][nt] float32 CUDA tensor; returns the converted tensor."""
    import torch
    out = torch.empty_like(tau_nc)
    nx, ny, nt = tau_nc.shape
    midpoint_confocal(nx, ny, nt, bin_width_s, wall_width_m, laser_xy, tau_nc.data_ptr(), out.data_ptr(), _stream())
    return out


def forward_t(plan, u, apply_mask=False):
    import torch
    tau = torch.empty_like(u)
    plan.forward(u.data_ptr(), tau.data_ptr(), apply_mask, _stream())
    return tau


def adjoint_t(plan, tau, apply_mask=False):
    import torch
    u = torch.empty_like(tau)
    plan.adjoint(tau.data_ptr(), u.data_ptr(), apply_mask, _stream())
    return u


def forward_directional_t(plan, u, normals, apply_mask=False):
    """nlos_forward_directional on tensors; normals: [3, nx, ny, nt] float32 on the device."""
    import torch
    tau = torch.empty_like(u)
    check(load().nlos_forward_directional(plan.handle, u.data_ptr(), normals.data_ptr(), tau.data_ptr(),
                                          int(bool(apply_mask)), _stream()))
    return tau


def adjoint_directional_t(plan, tau, normals, apply_mask=False):
    """nlos_adjoint_directional on tensors."""
    import torch
    u = torch.empty_like(tau)
    check(load().nlos_adjoint_directional(plan.handle, tau.data_ptr(), normals.data_ptr(), u.data_ptr(),
                                          int(bool(apply_mask)), _stream()))
    return u


def solve_t(plan, rhs, c0, c1):
    import torch
    x = torch.empty_like(rhs)
    plan.solve(rhs.data_ptr(), x.data_ptr(), c0, c1, _stream())
    return x


def curvature_weight_t(plan, u, a, b, phi="tsc", eps=1e-6):
    import torch
    ph = torch.empty_like(u)
    plan.curvature_weight(u.data_ptr(), ph.data_ptr(), a, b, PHI[phi], eps, _stream())
    return ph


def reconstruct_t(plan, params, tau0, want_tau=False):
    import torch
    u = torch.empty_like(tau0)
    tau = torch.empty_like(tau0) if want_tau else None
    stats = plan.reconstruct(params, tau0.data_ptr(), u.data_ptr(), tau.data_ptr() if tau is not None else 0,
                             _stream())
    return (u, tau, stats) if want_tau else (u, stats)


def selftest_wait_timeout(wait_ms, status_t):
    """Queue the bounded-wait self-test on torch's current stream; the kernel
    writes its status (NLOS_ERR_TIMEOUT when the wait gave up) to the int32
    CUDA tensor ``status_t``."""
    check(load().nlos_selftest_wait_timeout(int(wait_ms), ctypes.c_void_p(status_t.data_ptr()), _stream()))
