"""Python binding of the C ABI in ``include/rljsde.h`` (argument marshalling only).

Every step of the reconstruction runs in the CUDA library ``librljsde.so``;
this module converts numpy masks and torch CUDA tensors into the pointers and
sizes the ABI takes.  It raises if the library has not been built: there is
no fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "librljsde.so")

STATUS = {0: "OK", 1: "INVALID_ARG", 2: "BAD_SHAPE", 3: "BAD_MASK", 4: "OUT_OF_MEMORY", 5: "CUDA",
          6: "TIMEOUT", 7: "NONFINITE_INPUT", 8: "UNSUPPORTED"}


class RljsdeError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        super().__init__("%s: %s (%s)" % (what, _lib().rljsde_status_string(status).decode(),
                                          STATUS.get(status, status)))


class Params(ctypes.Structure):
    """``rljsde_params``: B, W, nu_max, gamma_odc, rho_decay, q_mode, q_table,
    precision, path, layout, pairs, c_supply (see the header for meanings and
    defaults)."""
    _fields_ = [("block", ctypes.c_int), ("window", ctypes.c_int), ("nu_max", ctypes.c_int),
                ("gamma_odc", ctypes.c_double), ("rho_decay", ctypes.c_double),
                ("q_mode", ctypes.c_int), ("q_table", ctypes.POINTER(ctypes.c_double)),
                ("precision", ctypes.c_int), ("path", ctypes.c_int), ("layout", ctypes.c_int),
                ("pairs", ctypes.c_int), ("c_supply", ctypes.c_int)]


LAYOUT_THREE_QUARTER = 0   # mask code = opaque sub-pixel 2 * dy + dx
LAYOUT_APERTURE = 1        # mask code = bit set of transparent sub-pixels


class PlanInfo(ctypes.Structure):
    _fields_ = [("n_images", ctypes.c_int), ("n_blocks", ctypes.c_int), ("n_tables", ctypes.c_int),
                ("n_interior_tables", ctypes.c_int), ("n_work_entries", ctypes.c_int),
                ("warps_per_cta", ctypes.c_int), ("ctas_per_sm", ctypes.c_int), ("grid", ctypes.c_int),
                ("device_table_bytes", ctypes.c_int64), ("paper_B_bytes", ctypes.c_int64),
                ("paper_C_bytes", ctypes.c_int64), ("paper_D_bytes", ctypes.c_int64),
                ("path", ctypes.c_int), ("n_apertures", ctypes.c_int), ("n_stored_c_tables", ctypes.c_int),
                ("n_stored_c_blocks", ctypes.c_int), ("device_c_bytes", ctypes.c_int64),
                ("n_launches", ctypes.c_int)]


class Image(ctypes.Structure):
    _fields_ = [("lr", ctypes.c_void_p), ("hr", ctypes.c_void_p), ("lr_pitch", ctypes.c_int64),
                ("hr_pitch", ctypes.c_int64)]


EXPORTS = ["rljsde_default_params", "rljsde_plan_create", "rljsde_plan_create_batch",
           "rljsde_reconstruct", "rljsde_reconstruct_trace", "rljsde_set_images",
           "rljsde_reconstruct_batch", "rljsde_set_launch", "rljsde_plan_info", "rljsde_check",
           "rljsde_plan_destroy", "rljsde_status_string", "rljsde_autotune", "rljsde_graph_capture",
           "rljsde_graph_launch", "rljsde_net_create", "rljsde_net_destroy", "rljsde_net_num_params",
           "rljsde_net_get_params", "rljsde_net_set_params", "rljsde_net_patches", "rljsde_net_gradient",
           "rljsde_net_train_step", "rljsde_net_logits", "rljsde_propose_workspace", "rljsde_propose",
           "rljsde_reconstruct_learned", "rljsde_propose_noalloc", "rljsde_fp32_peak",
           "rljsde_l2_read_peak"]

SHORTLIST_BYTES = 136

_LIB = None


def _lib():
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError("librljsde.so is not built (run __graft_entry__.build() or "
                              "python -m paper_2205_02646_gb300.build); there is no CPU fallback")
        lib = ctypes.CDLL(LIB_PATH)
        vp, i, sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_size_t
        lib.rljsde_default_params.argtypes = [ctypes.POINTER(Params)]
        lib.rljsde_plan_create.argtypes = [ctypes.POINTER(vp), vp, i, i, ctypes.POINTER(Params)]
        lib.rljsde_plan_create_batch.argtypes = [ctypes.POINTER(vp), i, ctypes.POINTER(vp),
                                                 ctypes.POINTER(i), ctypes.POINTER(i), ctypes.POINTER(Params)]
        lib.rljsde_reconstruct.argtypes = [vp, vp, sz, vp, sz, vp]
        lib.rljsde_reconstruct_trace.argtypes = [vp, vp, sz, vp, sz, vp, vp, vp]
        lib.rljsde_set_images.argtypes = [vp, ctypes.POINTER(Image)]
        lib.rljsde_reconstruct_batch.argtypes = [vp, vp]
        lib.rljsde_set_launch.argtypes = [vp, i, i]
        lib.rljsde_plan_info.argtypes = [vp, ctypes.POINTER(PlanInfo)]
        lib.rljsde_check.argtypes = [vp, vp]
        lib.rljsde_plan_destroy.argtypes = [vp]
        lib.rljsde_plan_destroy.restype = None
        lib.rljsde_autotune.argtypes = [vp, vp, sz, vp, sz, i, vp, ctypes.POINTER(i), ctypes.POINTER(i),
                                        ctypes.POINTER(ctypes.c_float)]
        lib.rljsde_graph_capture.argtypes = [vp, vp]
        lib.rljsde_graph_launch.argtypes = [vp, vp]
        f, u64, i32p = ctypes.c_float, ctypes.c_uint64, ctypes.c_void_p
        lib.rljsde_net_create.argtypes = [ctypes.POINTER(vp), u64]
        lib.rljsde_net_destroy.argtypes = [vp]
        lib.rljsde_net_destroy.restype = None
        lib.rljsde_net_num_params.argtypes = []
        lib.rljsde_net_get_params.argtypes = [vp, vp]
        lib.rljsde_net_set_params.argtypes = [vp, vp]
        lib.rljsde_net_patches.argtypes = [vp, sz, vp, i, i, i32p, i, vp, vp]
        lib.rljsde_net_gradient.argtypes = [vp, vp, i32p, i, i, i, vp, vp, vp, f, f, f, vp, ctypes.POINTER(f), vp]
        lib.rljsde_net_train_step.argtypes = [vp, vp, i32p, i, i, i, vp, vp, vp, f, f, f, f, ctypes.POINTER(f), vp]
        lib.rljsde_net_logits.argtypes = [vp, vp, i32p, i, i, i, vp, vp]
        lib.rljsde_propose_workspace.argtypes = [vp]
        lib.rljsde_propose_workspace.restype = ctypes.c_size_t
        lib.rljsde_propose.argtypes = [vp, vp, vp, sz, vp, vp, sz, vp]
        lib.rljsde_reconstruct_learned.argtypes = [vp, vp, sz, vp, sz, vp, f, i, vp, vp, vp, vp]
        lib.rljsde_propose_noalloc.argtypes = [vp, vp, vp, sz, vp, vp]
        lib.rljsde_fp32_peak.argtypes = [i, vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(f)]
        lib.rljsde_l2_read_peak.argtypes = [i, vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(f)]
        lib.rljsde_status_string.argtypes = [i]
        lib.rljsde_status_string.restype = ctypes.c_char_p
        _LIB = lib
    return _LIB


def load():
    """Load the shared library (raises ImportError if it is not built)."""
    return _lib()


def _ok(st, what):
    if st != 0:
        raise RljsdeError(st, what)


def default_params(**kw) -> Params:
    p = Params()
    _ok(_lib().rljsde_default_params(ctypes.byref(p)), "rljsde_default_params")
    q_table = kw.pop("q_table", None)
    for k, v in kw.items():
        setattr(p, k, v)
    if q_table is not None:
        arr = np.ascontiguousarray(q_table, dtype=np.float64).ravel()
        p._q_keep = arr
        p.q_table = arr.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        p.q_mode = 2
    return p


def _stream_ptr(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if hasattr(stream, "cuda_stream"):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


def _check_tensor(t, shape, name):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float32:
        raise TypeError("%s must be a float32 CUDA tensor" % name)
    if t.dim() != 2 or tuple(t.shape) != tuple(shape) or t.stride(1) != 1:
        raise ValueError("%s must be %s with unit column stride, got %s" % (name, shape, tuple(t.shape)))


class Plan:
    """Owns an ``rljsde_plan_t`` (tables and work list in device memory)."""

    def __init__(self, masks, params: Params | None = None):
        lib = _lib()
        self.params = params if params is not None else default_params()
        single = isinstance(masks, np.ndarray)
        ms = [np.ascontiguousarray(masks if single else m, dtype=np.uint8)
              for m in ([masks] if single else masks)]
        self.shapes = [m.shape for m in ms]
        self.single = single
        h = ctypes.c_void_p()
        if single:
            st = lib.rljsde_plan_create(ctypes.byref(h), ms[0].ctypes.data, ms[0].shape[0], ms[0].shape[1],
                                        ctypes.byref(self.params))
        else:
            n = len(ms)
            ptrs = (ctypes.c_void_p * n)(*[m.ctypes.data for m in ms])
            hs = (ctypes.c_int * n)(*[m.shape[0] for m in ms])
            ws = (ctypes.c_int * n)(*[m.shape[1] for m in ms])
            st = lib.rljsde_plan_create_batch(ctypes.byref(h), n, ptrs, hs, ws, ctypes.byref(self.params))
        _ok(st, "rljsde_plan_create")
        self._h = h
        self._images = None

    @property
    def handle(self):
        return self._h

    def info(self) -> dict:
        out = PlanInfo()
        _ok(_lib().rljsde_plan_info(self._h, ctypes.byref(out)), "rljsde_plan_info")
        return {f: getattr(out, f) for f, _ in PlanInfo._fields_}

    def set_launch(self, warps_per_cta=0, ctas_per_sm=0):
        _ok(_lib().rljsde_set_launch(self._h, warps_per_cta, ctas_per_sm), "rljsde_set_launch")

    def reconstruct(self, lr, hr, stream=None):
        lr_h, lr_w = self.shapes[0]
        _check_tensor(lr, (lr_h, lr_w), "lr")
        _check_tensor(hr, (2 * lr_h, 2 * lr_w), "hr")
        _ok(_lib().rljsde_reconstruct(self._h, lr.data_ptr(), lr.stride(0), hr.data_ptr(), hr.stride(0),
                                      _stream_ptr(stream)), "rljsde_reconstruct")

    def reconstruct_trace(self, lr, hr, sel, dc, stream=None):
        import torch
        lr_h, lr_w = self.shapes[0]
        _check_tensor(lr, (lr_h, lr_w), "lr")
        _check_tensor(hr, (2 * lr_h, 2 * lr_w), "hr")
        nb = (lr_h // 2) * (lr_w // 2)
        nu = self.params.nu_max
        if sel.dtype != torch.int16 or sel.numel() != nb * nu or not sel.is_cuda:
            raise ValueError("sel must be a CUDA int16 tensor of n_blocks * nu_max entries")
        if dc.dtype != torch.float32 or dc.numel() != nb * nu * 2 or not dc.is_cuda:
            raise ValueError("dc must be a CUDA float32 tensor of n_blocks * nu_max * 2 entries")
        _ok(_lib().rljsde_reconstruct_trace(self._h, lr.data_ptr(), lr.stride(0), hr.data_ptr(), hr.stride(0),
                                            sel.data_ptr(), dc.data_ptr(), _stream_ptr(stream)),
            "rljsde_reconstruct_trace")

    def set_images(self, lrs, hrs):
        n = len(self.shapes)
        if len(lrs) != n or len(hrs) != n:
            raise ValueError("need one lr and one hr tensor per image")
        arr = (Image * n)()
        for i, ((lr_h, lr_w), lr, hr) in enumerate(zip(self.shapes, lrs, hrs)):
            _check_tensor(lr, (lr_h, lr_w), "lr[%d]" % i)
            _check_tensor(hr, (2 * lr_h, 2 * lr_w), "hr[%d]" % i)
            arr[i] = Image(lr.data_ptr(), hr.data_ptr(), lr.stride(0), hr.stride(0))
        _ok(_lib().rljsde_set_images(self._h, arr), "rljsde_set_images")
        self._images = (list(lrs), list(hrs))       # keep the buffers alive

    def reconstruct_batch(self, stream=None):
        _ok(_lib().rljsde_reconstruct_batch(self._h, _stream_ptr(stream)), "rljsde_reconstruct_batch")

    def autotune(self, lr=None, hr=None, reps=3, stream=None) -> dict:
        """Time every launch shape on this plan's work and keep the fastest."""
        w, c, ms = ctypes.c_int(), ctypes.c_int(), ctypes.c_float()
        if lr is None:
            st = _lib().rljsde_autotune(self._h, None, 0, None, 0, reps, _stream_ptr(stream),
                                        ctypes.byref(w), ctypes.byref(c), ctypes.byref(ms))
        else:
            lr_h, lr_w = self.shapes[0]
            _check_tensor(lr, (lr_h, lr_w), "lr")
            _check_tensor(hr, (2 * lr_h, 2 * lr_w), "hr")
            st = _lib().rljsde_autotune(self._h, lr.data_ptr(), lr.stride(0), hr.data_ptr(), hr.stride(0), reps,
                                        _stream_ptr(stream), ctypes.byref(w), ctypes.byref(c), ctypes.byref(ms))
        _ok(st, "rljsde_autotune")
        return dict(warps_per_cta=w.value, ctas_per_sm=c.value, ms=ms.value)

    def graph_capture(self, stream):
        """Capture one batch launch on ``stream`` (a non-default torch stream)."""
        _ok(_lib().rljsde_graph_capture(self._h, _stream_ptr(stream)), "rljsde_graph_capture")

    def graph_launch(self, stream=None):
        _ok(_lib().rljsde_graph_launch(self._h, _stream_ptr(stream)), "rljsde_graph_launch")

    def propose(self, net, lr, shortlists=None, workspace=None, stream=None):
        """Run the proposal network over the image; returns the shortlist
        buffer (uint8 CUDA tensor, 136 bytes per block)."""
        import torch
        lr_h, lr_w = self.shapes[0]
        _check_tensor(lr, (lr_h, lr_w), "lr")
        nb = (lr_h // 2) * (lr_w // 2)
        if shortlists is None:
            shortlists = torch.empty(nb * SHORTLIST_BYTES, dtype=torch.uint8, device=lr.device)
        need = _lib().rljsde_propose_workspace(self._h)
        if workspace is None or workspace.numel() < need:
            workspace = torch.empty(need, dtype=torch.uint8, device=lr.device)
        _ok(_lib().rljsde_propose(self._h, net.handle, lr.data_ptr(), lr.stride(0), shortlists.data_ptr(),
                                  workspace.data_ptr(), workspace.numel(), _stream_ptr(stream)), "rljsde_propose")
        self._ws = workspace
        return shortlists

    def reconstruct_learned(self, lr, hr, shortlists, max_missing=1.0, use_nu_hat=False, sel=None, dc=None,
                            counter=None, stream=None):
        lr_h, lr_w = self.shapes[0]
        _check_tensor(lr, (lr_h, lr_w), "lr")
        _check_tensor(hr, (2 * lr_h, 2 * lr_w), "hr")
        _ok(_lib().rljsde_reconstruct_learned(
            self._h, lr.data_ptr(), lr.stride(0), hr.data_ptr(), hr.stride(0), shortlists.data_ptr(),
            float(max_missing), int(bool(use_nu_hat)), None if sel is None else sel.data_ptr(),
            None if dc is None else dc.data_ptr(), None if counter is None else counter.data_ptr(),
            _stream_ptr(stream)), "rljsde_reconstruct_learned")

    def check(self, stream=None):
        _ok(_lib().rljsde_check(self._h, _stream_ptr(stream)), "rljsde_check")

    def close(self):
        if getattr(self, "_h", None):
            _lib().rljsde_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def fp32_peak(reps=5, stream=None) -> dict:
    """FP32 FMA throughput of the current device (``rljsde_fp32_peak``)."""
    tf, ms = ctypes.c_double(), ctypes.c_float()
    _ok(_lib().rljsde_fp32_peak(int(reps), _stream_ptr(stream), ctypes.byref(tf), ctypes.byref(ms)),
        "rljsde_fp32_peak")
    return dict(tflops=tf.value, ms=ms.value)


def l2_read_peak(reps=5, stream=None) -> dict:
    """L2 read bandwidth of the current device (``rljsde_l2_read_peak``)."""
    gbs, ms = ctypes.c_double(), ctypes.c_float()
    _ok(_lib().rljsde_l2_read_peak(int(reps), _stream_ptr(stream), ctypes.byref(gbs), ctypes.byref(ms)),
        "rljsde_l2_read_peak")
    return dict(gbs=gbs.value, ms=ms.value)


def shortlist_view(buf, n_blocks):
    """Host view of a shortlist buffer: (idx (n, 64) uint16, missing (n,), nu_frac (n,))."""
    raw = buf.cpu().numpy() if hasattr(buf, "cpu") else np.asarray(buf)
    rec = np.dtype([("idx", "<u2", (64,)), ("missing", "<f4"), ("nu_frac", "<f4")])
    arr = raw[: n_blocks * SHORTLIST_BYTES].view(rec)
    return arr["idx"], arr["missing"], arr["nu_frac"]


def shortlist_from_indices(idx, missing=None, nu_frac=None):
    """Pack (n, 64) candidate indices into a shortlist buffer (uint8 numpy)."""
    idx = np.asarray(idx, dtype=np.uint16)
    n = idx.shape[0]
    rec = np.dtype([("idx", "<u2", (64,)), ("missing", "<f4"), ("nu_frac", "<f4")])
    arr = np.zeros(n, rec)
    arr["idx"] = idx
    arr["missing"] = 0.0 if missing is None else missing
    arr["nu_frac"] = 1.0 if nu_frac is None else nu_frac
    return arr.view(np.uint8)


class Net:
    """The proposal network (``rljsde_net_t``): seeded init, training steps
    and parameter access; all arithmetic in the CUDA library."""

    def __init__(self, seed: int = 0):
        h = ctypes.c_void_p()
        _ok(_lib().rljsde_net_create(ctypes.byref(h), ctypes.c_uint64(seed)), "rljsde_net_create")
        self._h = h

    @property
    def handle(self):
        return self._h

    @staticmethod
    def num_params() -> int:
        return _lib().rljsde_net_num_params()

    def get_params(self) -> np.ndarray:
        out = np.zeros(self.num_params(), np.float32)
        _ok(_lib().rljsde_net_get_params(self._h, out.ctypes.data), "rljsde_net_get_params")
        return out

    def set_params(self, arr):
        arr = np.ascontiguousarray(arr, dtype=np.float32)
        assert arr.size == self.num_params()
        _ok(_lib().rljsde_net_set_params(self._h, arr.ctypes.data), "rljsde_net_set_params")

    @staticmethod
    def patches(lr, mask_dev, blocks_dev, stream=None):
        """x (n, 5, 16, 16) for blocks (CUDA int32 (n, 2)) of lr with mask (CUDA uint8)."""
        import torch
        n = blocks_dev.shape[0]
        x = torch.empty((n, 5, 16, 16), dtype=torch.float32, device=lr.device)
        _ok(_lib().rljsde_net_patches(lr.data_ptr(), lr.stride(0), mask_dev.data_ptr(), lr.shape[0], lr.shape[1],
                                      blocks_dev.data_ptr(), n, x.data_ptr(), _stream_ptr(stream)),
            "rljsde_net_patches")
        return x

    def gradient(self, x, blocks, lr_shape, targets, nu_t, mass=None, pos_weight=8.0, nu_weight=0.1,
                 gate_weight=1.0, stream=None):
        import torch
        g = torch.empty(self.num_params(), dtype=torch.float32, device=x.device)
        loss = ctypes.c_float()
        _ok(_lib().rljsde_net_gradient(self._h, x.data_ptr(), blocks.data_ptr(), x.shape[0], lr_shape[0],
                                       lr_shape[1], targets.data_ptr(), nu_t.data_ptr(),
                                       None if mass is None else mass.data_ptr(), pos_weight, nu_weight, gate_weight,
                                       g.data_ptr(), ctypes.byref(loss), _stream_ptr(stream)), "rljsde_net_gradient")
        return g, loss.value

    def train_step(self, x, blocks, lr_shape, targets, nu_t, mass=None, lr=1e-3, pos_weight=8.0, nu_weight=0.1,
                   gate_weight=1.0, stream=None):
        loss = ctypes.c_float()
        _ok(_lib().rljsde_net_train_step(self._h, x.data_ptr(), blocks.data_ptr(), x.shape[0], lr_shape[0],
                                         lr_shape[1], targets.data_ptr(), nu_t.data_ptr(),
                                         None if mass is None else mass.data_ptr(), pos_weight, nu_weight,
                                         gate_weight, lr, ctypes.byref(loss), _stream_ptr(stream)),
            "rljsde_net_train_step")
        return loss.value

    def logits(self, x, blocks, lr_shape, stream=None):
        import torch
        z = torch.empty((x.shape[0], 1026), dtype=torch.float32, device=x.device)
        _ok(_lib().rljsde_net_logits(self._h, x.data_ptr(), blocks.data_ptr(), x.shape[0], lr_shape[0],
                                     lr_shape[1], z.data_ptr(), _stream_ptr(stream)), "rljsde_net_logits")
        return z

    def close(self):
        if getattr(self, "_h", None):
            _lib().rljsde_net_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
