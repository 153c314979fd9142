"""Thin ctypes binding of libbte (include/bte.h).

Argument marshalling only: every step of the collision operator, projection
and time stepping runs in libbte's CUDA kernels. Tensors are torch CUDA
tensors (float64, contiguous); pointers and the current CUDA stream are handed
to the C ABI unchanged. There is no CPU fallback: if libbte.so is missing or no
GPU is visible, the calls raise.
"""
import ctypes
import os

from . import build as _build

FP64_PLAIN = 0
FP32 = 1
LEARNED = 2
BC_DIFFUSE = 0
BC_SPECULAR = 1
BC_NOFLUX = 2
FLAG_RAW = 1
FLAG_NO_FALLBACK = 2

STATUS = {0: "BTE_OK", -1: "BTE_EINVAL", -2: "BTE_ENOMEM", -3: "BTE_ECUDA", -4: "BTE_ETIMEOUT",
          -5: "BTE_ENONFINITE", -6: "BTE_ESTATE"}

# Every symbol include/bte.h declares (checked by the ABI tests).
EXPORTS = ["bte_create", "bte_destroy", "bte_last_error", "bte_init_weights", "bte_init_weights_ex", "bte_collide",
           "bte_collide_ex", "bte_project", "bte_step", "bte_step_ex", "bte_sync_status", "bte_moments",
           "bte_version", "bte_profile_enable", "bte_profile_read", "bte_launch_count", "bte_batch_count", "bte_graph_count",
           "bte_set_option", "bte_get_option", "bte_collide_noalloc", "bte_tc_gemm", "bte_mlp_init", "bte_mlp_info",
           "bte_mlp_set_scales", "bte_mlp_fit_scales", "bte_mlp_get_params", "bte_mlp_set_params", "bte_mlp_train",
           "bte_mlp_grads", "bte_mlp_infer", "bte_learned_stats", "bte_learned_sample",
           "bte_learned_indicator", "bte_autotune", "bte_tune_save",
           "bte_tune_load", "bte_state_save", "bte_state_load", "bte_alu_peak", "bte_transfer"]


class Grid(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int), ("L", ctypes.c_double), ("lambda_", ctypes.c_double)]


class GridEx(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int), ("L", ctypes.c_double), ("lambda_", ctypes.c_double),
                ("beta", ctypes.c_double)]


class Instance(ctypes.Structure):
    _fields_ = [("table", ctypes.c_int32), ("pad_", ctypes.c_int32), ("offset", ctypes.c_int64)]


class Transport(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("x0", ctypes.c_double), ("x1", ctypes.c_double),
                ("bc_left", ctypes.c_int), ("bc_right", ctypes.c_int),
                ("Tw_left", ctypes.c_double), ("Tw_right", ctypes.c_double)]


class TransportEx(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("dx", ctypes.c_void_p), ("x0", ctypes.c_double), ("x1", ctypes.c_double),
                ("bc_left", ctypes.c_int), ("bc_right", ctypes.c_int),
                ("Tw_left", ctypes.c_double), ("Tw_right", ctypes.c_double)]


class BteError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s: %s" % (STATUS.get(code, str(code)), msg))
        self.code = code


_lib = None


def library_path():
    return _build.LIB


def load(path=None):
    """Load libbte.so (built in-tree by __graft_entry__.build())."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or _build.LIB
    if not os.path.exists(path):
        raise RuntimeError("libbte.so is not built (%s): run __graft_entry__.build()" % path)
    L = ctypes.CDLL(path)
    c_int, c_i64, c_u, vp, c_d = ctypes.c_int, ctypes.c_int64, ctypes.c_uint, ctypes.c_void_p, ctypes.c_double
    sig = {
        "bte_create": (c_int, [ctypes.POINTER(vp), c_int]),
        "bte_destroy": (None, [vp]),
        "bte_last_error": (ctypes.c_char_p, [vp]),
        "bte_init_weights": (c_int, [vp, ctypes.POINTER(Grid), c_int, ctypes.POINTER(c_int)]),
        "bte_init_weights_ex": (c_int, [vp, ctypes.POINTER(GridEx), c_int, ctypes.POINTER(c_int)]),
        "bte_collide": (c_int, [vp, vp, vp, ctypes.POINTER(Instance), c_i64, c_int, vp]),
        "bte_collide_ex": (c_int, [vp, vp, vp, ctypes.POINTER(Instance), c_i64, c_int, c_u, vp]),
        "bte_project": (c_int, [vp, vp, ctypes.POINTER(Instance), c_i64, vp]),
        "bte_step": (c_int, [vp, vp, ctypes.POINTER(Instance), c_i64, c_d, c_d,
                             ctypes.POINTER(Transport), c_int, vp]),
        "bte_step_ex": (c_int, [vp, vp, ctypes.POINTER(Instance), c_i64, c_d, c_d,
                                ctypes.POINTER(TransportEx), c_int, vp]),
        "bte_sync_status": (c_int, [vp, vp]),
        "bte_transfer": (c_int, [vp, vp, vp, ctypes.c_size_t, c_int, vp]),
        "bte_moments": (c_int, [vp, vp, vp, ctypes.POINTER(Instance), c_i64, vp]),
        "bte_version": (ctypes.c_char_p, []),
        "bte_profile_enable": (c_int, [vp, c_int]),
        "bte_profile_read": (c_int, [vp, ctypes.c_char_p, ctypes.POINTER(c_i64),
                                     ctypes.POINTER(c_d), vp]),
        "bte_launch_count": (c_int, [vp, ctypes.POINTER(c_i64)]),
        "bte_batch_count": (c_int, [vp, ctypes.POINTER(c_i64)]),
        "bte_graph_count": (c_int, [vp, ctypes.POINTER(c_i64)]),
        "bte_set_option": (c_int, [vp, ctypes.c_char_p, c_int]),
        "bte_get_option": (c_int, [vp, ctypes.c_char_p, ctypes.POINTER(c_int)]),
        "bte_collide_noalloc": (c_int, [vp, vp, vp, c_i64, vp]),
        "bte_tc_gemm": (c_int, [vp, vp, vp, vp, c_int, c_int, c_int, vp, c_int, vp, vp, c_int, vp]),
        "bte_mlp_init": (c_int, [vp, c_int, c_int, ctypes.c_uint64]),
        "bte_mlp_info": (c_int, [vp, ctypes.POINTER(c_i64), ctypes.POINTER(c_int), ctypes.POINTER(c_int),
                                 ctypes.POINTER(c_d), ctypes.POINTER(c_d)]),
        "bte_mlp_set_scales": (c_int, [vp, c_d, c_d]),
        "bte_mlp_fit_scales": (c_int, [vp, vp, vp, c_i64, c_d, ctypes.POINTER(c_d), vp]),
        "bte_mlp_get_params": (c_int, [vp, vp, c_i64]),
        "bte_mlp_set_params": (c_int, [vp, vp, c_i64]),
        "bte_mlp_train": (c_int, [vp, vp, vp, c_i64, c_int, c_int, c_d, c_d, ctypes.c_uint64,
                                  ctypes.POINTER(c_d), vp]),
        "bte_mlp_grads": (c_int, [vp, vp, vp, c_i64, ctypes.POINTER(c_d), vp, vp]),
        "bte_mlp_infer": (c_int, [vp, vp, vp, c_i64, vp]),
        "bte_learned_stats": (c_int, [vp, ctypes.POINTER(c_i64), ctypes.POINTER(c_i64), ctypes.POINTER(c_d),
                                      c_int]),
        "bte_learned_sample": (c_int, [vp, ctypes.POINTER(c_int), c_int, ctypes.POINTER(c_int)]),
        "bte_learned_indicator": (c_int, [vp, vp, vp, c_i64, vp, vp]),
        "bte_autotune": (c_int, [vp, vp, ctypes.POINTER(Instance), c_i64, c_int, ctypes.POINTER(c_int),
                                 ctypes.POINTER(c_d), vp]),
        "bte_tune_save": (c_int, [vp, ctypes.c_char_p]),
        "bte_tune_load": (c_int, [vp, ctypes.c_char_p, ctypes.POINTER(c_int)]),
        "bte_state_save": (c_int, [vp, ctypes.c_char_p, vp, c_i64, c_d, c_i64, vp]),
        "bte_alu_peak": (c_int, [vp, c_int, ctypes.POINTER(c_d), ctypes.POINTER(c_d), vp]),
        "bte_state_load": (c_int, [vp, ctypes.c_char_p, vp, c_i64, ctypes.POINTER(c_d), ctypes.POINTER(c_i64), vp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def _stream(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def _check_f64(t, name):
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
        raise TypeError("%s must be a contiguous float64 CUDA tensor" % name)


class Context:
    """One libbte context on one CUDA device (owns weight tables and scratch)."""

    def __init__(self, device=0):
        self._lib = load()
        h = ctypes.c_void_p()
        rc = self._lib.bte_create(ctypes.byref(h), int(device))
        if rc != 0:
            raise BteError(rc, "bte_create(device=%d) failed" % device)
        self._h = h
        self.device = int(device)
        self.grids = []

    def close(self):
        if getattr(self, "_h", None):
            self._lib.bte_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _rc(self, rc, what):
        if rc != 0:
            msg = self._lib.bte_last_error(self._h)
            raise BteError(rc, "%s: %s" % (what, msg.decode() if msg else ""))

    def init_weights(self, grids):
        """grids: list of (N, L, lambda) or (N, L, lambda, beta) (beta = 1: elastic).
        Returns the table ids."""
        full = [tuple(g) + (1.0,) if len(g) == 3 else tuple(g) for g in grids]
        arr = (GridEx * len(full))(*[GridEx(int(N), float(L), float(lam), float(beta))
                                      for (N, L, lam, beta) in full])
        ids = (ctypes.c_int * len(full))()
        self._rc(self._lib.bte_init_weights_ex(self._h, arr, len(full), ids), "bte_init_weights")
        self.grids += [g[:3] for g in full]
        return list(ids)

    def _inst(self, inst, f):
        if inst is None:
            N = self.grids[0][0]
            M = N ** 3
            if f.numel() % M:
                raise ValueError("f size is not a multiple of N^3 of table 0")
            return None, f.numel() // M
        arr = (Instance * len(inst))(*[Instance(int(t), 0, int(o)) for (t, o) in inst])
        return arr, len(inst)

    def collide(self, f, Q=None, inst=None, mode=FP32, raw=False, fallback=True, stream=None):
        _check_f64(f, "f")
        if Q is None:
            import torch
            Q = torch.empty_like(f)
        _check_f64(Q, "Q")
        arr, n = self._inst(inst, f)
        flags = (FLAG_RAW if raw else 0) | (0 if fallback else FLAG_NO_FALLBACK)
        self._rc(self._lib.bte_collide_ex(self._h, _ptr(f), _ptr(Q), arr, n, int(mode), flags,
                                          _stream(stream)), "bte_collide")
        return Q

    def learned_stats(self, reset=False):
        a, b, d = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_double()
        self._rc(self._lib.bte_learned_stats(self._h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(d),
                                             int(bool(reset))), "bte_learned_stats")
        return dict(cells=a.value, fallbacks=b.value, max_indicator=d.value)

    def learned_sample(self):
        """The indicator's sampled pencils (k1 N + k2), in drawing order."""
        S = ctypes.c_int()
        buf = (ctypes.c_int * 1024)()
        self._rc(self._lib.bte_learned_sample(self._h, buf, 1024, ctypes.byref(S)), "bte_learned_sample")
        return list(buf[:S.value])

    def learned_indicator(self, f, Q, stream=None):
        """Indicator of the learned mode for caller-given (f, Q) pairs (uniform cells of table 0)."""
        import torch
        _check_f64(f, "f")
        _check_f64(Q, "Q")
        _, n = self._inst(None, f)
        out = torch.empty(n, dtype=torch.float64, device=f.device)
        self._rc(self._lib.bte_learned_indicator(self._h, _ptr(f), _ptr(Q), n, _ptr(out), _stream(stream)),
                 "bte_learned_indicator")
        return out

    def project(self, Q, inst=None, stream=None):
        _check_f64(Q, "Q")
        arr, n = self._inst(inst, Q)
        self._rc(self._lib.bte_project(self._h, _ptr(Q), arr, n, _stream(stream)), "bte_project")
        return Q

    def moments(self, f, inst=None, stream=None):
        import torch
        _check_f64(f, "f")
        arr, n = self._inst(inst, f)
        out = torch.zeros((n, 5), dtype=torch.float64, device=f.device)
        self._rc(self._lib.bte_moments(self._h, _ptr(f), _ptr(out), arr, n, _stream(stream)),
                 "bte_moments")
        return out

    def step(self, f, dt, eps=1.0, transport=None, inst=None, mode=FP32, stream=None):
        """One RK2 (homogeneous) or Strang (transport dict given) step, in place.
        transport keys: nx, x0, x1, bc_left, bc_right, Tw_left, Tw_right, and dx
        (a sequence of nx cell widths, for cells of unequal width)."""
        _check_f64(f, "f")
        arr, n = self._inst(inst, f)
        tr = None
        keep = None
        if transport is not None:
            t = transport
            dxp = None
            if t.get("dx") is not None:
                keep = (ctypes.c_double * len(t["dx"]))(*[float(x) for x in t["dx"]])
                dxp = ctypes.cast(keep, ctypes.c_void_p)
            tr = TransportEx(int(t.get("nx", n)), dxp, float(t.get("x0", 0.0)), float(t.get("x1", 1.0)),
                             int(t.get("bc_left", BC_DIFFUSE)), int(t.get("bc_right", BC_SPECULAR)),
                             float(t.get("Tw_left", 1.0)), float(t.get("Tw_right", 1.0)))
            tr = ctypes.byref(tr)
        self._rc(self._lib.bte_step_ex(self._h, _ptr(f), arr, n, float(dt), float(eps), tr, int(mode),
                                       _stream(stream)), "bte_step")
        del keep
        return f

    def profile_enable(self, on=True):
        self._rc(self._lib.bte_profile_enable(self._h, int(bool(on))), "bte_profile_enable")

    def profile_read(self, kernel="conv32", stream=None):
        """(launches, total_ms) of profiled launches since the last read."""
        n = ctypes.c_int64()
        ms = ctypes.c_double()
        self._rc(self._lib.bte_profile_read(self._h, kernel.encode(), ctypes.byref(n),
                                            ctypes.byref(ms), _stream(stream)), "bte_profile_read")
        return n.value, ms.value

    def launch_count(self):
        n = ctypes.c_int64()
        self._rc(self._lib.bte_launch_count(self._h, ctypes.byref(n)), "bte_launch_count")
        return n.value

    def batch_count(self):
        n = ctypes.c_int64()
        self._rc(self._lib.bte_batch_count(self._h, ctypes.byref(n)), "bte_batch_count")
        return n.value

    def graph_count(self):
        n = ctypes.c_int64()
        self._rc(self._lib.bte_graph_count(self._h, ctypes.byref(n)), "bte_graph_count")
        return n.value

    def set_option(self, name, value):
        self._rc(self._lib.bte_set_option(self._h, name.encode(), int(value)), "bte_set_option")

    def get_option(self, name):
        v = ctypes.c_int()
        self._rc(self._lib.bte_get_option(self._h, name.encode(), ctypes.byref(v)), "bte_get_option")
        return v.value

    def tc_gemm(self, A, B, bias=None, gelu=False, out_f32=True, out_bf16=False, out_bf16_t=False,
                stream=None):
        """D = A B^T (+ bias) on the tensor cores; A [M, K], B [N, K] bf16 CUDA tensors.
        Returns (D fp32 or None, D bf16 or None, D^T bf16 or None)."""
        import torch
        M, K = A.shape
        N = B.shape[0]
        D = torch.empty((M, N), dtype=torch.float32, device=A.device) if out_f32 else None
        Db = torch.empty((M, N), dtype=torch.bfloat16, device=A.device) if out_bf16 else None
        Dt = torch.zeros((N, M), dtype=torch.bfloat16, device=A.device) if out_bf16_t else None
        vp = ctypes.c_void_p
        self._rc(self._lib.bte_tc_gemm(self._h, vp(A.data_ptr()), vp(B.data_ptr()),
                                       vp(D.data_ptr()) if D is not None else None, M, N, K,
                                       vp(bias.data_ptr()) if bias is not None else None, int(gelu),
                                       vp(Db.data_ptr()) if Db is not None else None,
                                       vp(Dt.data_ptr()) if Dt is not None else None, M,
                                       _stream(stream)), "bte_tc_gemm")
        return D, Db, Dt

    # ---- learned surrogate ----
    def mlp_init(self, table=0, width=1024, seed=0):
        self._rc(self._lib.bte_mlp_init(self._h, int(table), int(width), int(seed)), "bte_mlp_init")

    def mlp_info(self):
        n, w, d = ctypes.c_int64(), ctypes.c_int(), ctypes.c_int()
        si, so = ctypes.c_double(), ctypes.c_double()
        self._rc(self._lib.bte_mlp_info(self._h, ctypes.byref(n), ctypes.byref(w), ctypes.byref(d),
                                        ctypes.byref(si), ctypes.byref(so)), "bte_mlp_info")
        return dict(nparams=n.value, width=w.value, ndim=d.value, s_in=si.value, s_out=so.value)

    def mlp_set_scales(self, s_in, s_out):
        self._rc(self._lib.bte_mlp_set_scales(self._h, float(s_in), float(s_out)), "bte_mlp_set_scales")

    def mlp_fit_scales(self, f, Q, s_in=10.0, stream=None):
        """Set s_in and the s_out that makes the targets s_out Q / rho^2 of (f, Q) unit-RMS."""
        _check_f64(f, "f")
        _check_f64(Q, "Q")
        n = f.numel() // self.mlp_info()["ndim"]
        so = ctypes.c_double()
        self._rc(self._lib.bte_mlp_fit_scales(self._h, _ptr(f), _ptr(Q), n, float(s_in), ctypes.byref(so),
                                              _stream(stream)), "bte_mlp_fit_scales")
        return so.value

    def mlp_get_params(self):
        import numpy as np
        n = self.mlp_info()["nparams"]
        out = np.empty(n, dtype=np.float32)
        self._rc(self._lib.bte_mlp_get_params(self._h, out.ctypes.data_as(ctypes.c_void_p), n),
                 "bte_mlp_get_params")
        return out

    def mlp_set_params(self, p):
        import numpy as np
        p = np.ascontiguousarray(p, dtype=np.float32)
        self._rc(self._lib.bte_mlp_set_params(self._h, p.ctypes.data_as(ctypes.c_void_p), p.size),
                 "bte_mlp_set_params")

    def mlp_train(self, f, Q, epochs=1, batch=1024, lr=1e-3, weight_decay=0.0, seed=0, stream=None):
        _check_f64(f, "f")
        _check_f64(Q, "Q")
        n = f.numel() // self.mlp_info()["ndim"]
        loss = ctypes.c_double()
        self._rc(self._lib.bte_mlp_train(self._h, _ptr(f), _ptr(Q), n, int(epochs), int(batch), float(lr),
                                         float(weight_decay), int(seed), ctypes.byref(loss),
                                         _stream(stream)), "bte_mlp_train")
        return loss.value

    def mlp_grads(self, f, Q, stream=None):
        import numpy as np
        _check_f64(f, "f")
        _check_f64(Q, "Q")
        info = self.mlp_info()
        n = f.numel() // info["ndim"]
        g = np.empty(info["nparams"], dtype=np.float32)
        loss = ctypes.c_double()
        self._rc(self._lib.bte_mlp_grads(self._h, _ptr(f), _ptr(Q), n, ctypes.byref(loss),
                                         g.ctypes.data_as(ctypes.c_void_p), _stream(stream)),
                 "bte_mlp_grads")
        return loss.value, g

    def mlp_infer(self, f, Q=None, stream=None):
        import torch
        _check_f64(f, "f")
        if Q is None:
            Q = torch.empty_like(f)
        n = f.numel() // self.mlp_info()["ndim"]
        self._rc(self._lib.bte_mlp_infer(self._h, _ptr(f), _ptr(Q), n, _stream(stream)), "bte_mlp_infer")
        return Q

    def autotune(self, f, inst=None, reps=3, stream=None):
        """Time the candidate FP32 configurations on f (batch shape of inst) and keep
        the fastest for batches of this shape. Returns the chosen configuration."""
        _check_f64(f, "f")
        arr, n = self._inst(inst, f)
        cfg = (ctypes.c_int * 6)()
        ms = ctypes.c_double()
        self._rc(self._lib.bte_autotune(self._h, _ptr(f), arr, n, int(reps), cfg, ctypes.byref(ms),
                                        _stream(stream)), "bte_autotune")
        return dict(conv_impl=cfg[0], conv_warps=cfg[1], conv_stages=cfg[2], conv_merge=cfg[3],
                    dft_split=cfg[4], conv_split=cfg[5], ms=ms.value)

    def tune_save(self, path):
        self._rc(self._lib.bte_tune_save(self._h, str(path).encode()), "bte_tune_save")

    def tune_load(self, path):
        n = ctypes.c_int()
        self._rc(self._lib.bte_tune_load(self._h, str(path).encode(), ctypes.byref(n)), "bte_tune_load")
        return n.value

    def save_state(self, path, f, t=0.0, step=0, stream=None):
        """Checkpoint f (device, FP64), the time and the step counter to path."""
        _check_f64(f, "f")
        self._rc(self._lib.bte_state_save(self._h, str(path).encode(), _ptr(f), f.numel(), float(t), int(step),
                                          _stream(stream)), "bte_state_save")

    def load_state(self, path, f, stream=None):
        """Read a checkpoint into f (device, FP64, same size); returns (t, step)."""
        _check_f64(f, "f")
        t, step = ctypes.c_double(), ctypes.c_int64()
        self._rc(self._lib.bte_state_load(self._h, str(path).encode(), _ptr(f), f.numel(), ctypes.byref(t),
                                          ctypes.byref(step), _stream(stream)), "bte_state_load")
        return t.value, step.value

    def alu_peak(self, kind=0, stream=None):
        """Measured FMA rate of this GPU in TFLOP/s: kind 0 FP32, 1 packed FP32x2, 2 FP64."""
        tf, ms = ctypes.c_double(), ctypes.c_double()
        self._rc(self._lib.bte_alu_peak(self._h, int(kind), ctypes.byref(tf), ctypes.byref(ms), _stream(stream)),
                 "bte_alu_peak")
        return tf.value

    def transfer(self, dst, src, stream=None):
        """Copy tensor src into tensor dst (same size) between host and device
        memory through bte_transfer; the host tensor should be pinned."""
        if dst.numel() * dst.element_size() != src.numel() * src.element_size():
            raise ValueError("transfer: dst and src differ in size")
        if dst.is_cuda == src.is_cuda:
            raise ValueError("transfer: one tensor on the host, one on the device")
        kind = 0 if dst.is_cuda else 1
        self._rc(self._lib.bte_transfer(self._h, _ptr(dst), _ptr(src), dst.numel() * dst.element_size(), kind,
                                        _stream(stream)), "bte_transfer")
        return dst

    def sync_status(self, stream=None):
        rc = self._lib.bte_sync_status(self._h, _stream(stream))
        self._rc(rc, "device status")
