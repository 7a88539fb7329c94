"""GB300 (sm_103a) BAD / HashSIFT binary descriptors and Hamming matching.

Python binding of ``libbindesc.so`` (declared in ``include/bindesc.h``).  The
``bd_*`` functions here carry the C names and only marshal arguments; every
step of the computation runs in the library's CUDA kernels.  PyTorch serves
for device memory and streams: tensors are passed by ``data_ptr()`` and work
is enqueued on ``torch.cuda.current_stream()`` unless a context says otherwise.

There is no CPU fallback: if the library is missing or the device is not an
sm_103 GPU, the calls raise.
"""
from __future__ import annotations

import ctypes
import os
import threading
import atexit
import weakref

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libbindesc.so")

BD_OK = 0
BD_ERR_INVALID = 1
BD_ERR_CUDA = 2
BD_ERR_NOMEM = 3
BD_ERR_TIMEOUT = 4
BD_ERR_DEVICE_CHECK = 5
BD_ERR_UNSUPPORTED = 6
BD_FLAG_INVALID_KEYPOINT = 0x1
BD_FLAG_TIMEOUT = 0x2
BD_HS_FP32 = 0
BD_HS_BF16_RESCUE = 1
BD_HS_VARIANT_TRILINEAR = 1
BD_HS_VARIANT_CLIP = 2
BD_HS_VARIANT_ROOT = 4
BD_PROBE_GATHER = 0
BD_PROBE_POPC = 1
BD_PROBE_FFMA = 2
BD_PROBE_MUFU = 3
BD_PROBE_L1_SECTORS = 4

_STATUS_NAMES = {0: "BD_OK", 1: "BD_ERR_INVALID", 2: "BD_ERR_CUDA", 3: "BD_ERR_NOMEM",
                 4: "BD_ERR_TIMEOUT", 5: "BD_ERR_DEVICE_CHECK", 6: "BD_ERR_UNSUPPORTED"}

# (name, restype, argtypes) of every exported call; include/bindesc.h is the reference.
_P = ctypes.c_void_p
_I = ctypes.c_int
_F = ctypes.c_float
_SZ = ctypes.c_size_t
_SIGS = [
    ("bd_create", _I, [_I, _P, ctypes.POINTER(_P)]),
    ("bd_destroy", None, [_P]),
    ("bd_set_stream", _I, [_P, _P]),
    ("bd_last_error", ctypes.c_char_p, [_P]),
    ("bd_sync_status", _I, [_P, ctypes.POINTER(ctypes.c_uint32)]),
    ("bd_rescued_count", _I, [_P, ctypes.POINTER(ctypes.c_uint64), _I]),
    ("bd_kernel_launches", ctypes.c_uint64, []),
    ("bd_trace_enable", _I, [_P, _I]),
    ("bd_trace_reset", _I, [_P]),
    ("bd_trace_read", _I, [_P, _I, ctypes.POINTER(_F), ctypes.POINTER(ctypes.c_char_p)]),
    ("bd_reserve", _I, [_P, _SZ]),
    ("bd_scratch_bytes_bad", _SZ, [_I, _I]),
    ("bd_scratch_bytes_hashsift", _SZ, [_I]),
    ("bd_scratch_bytes_match", _SZ, [_I, _I, _I]),
    ("bd_bad_params_create", _I, [_P, _I, _P, _P, _P, ctypes.c_int32, _I, _P, _I, ctypes.POINTER(_P)]),
    ("bd_bad_params_destroy", None, [_P]),
    ("bd_bad_params_table", _I, [_P, _P, _P]),
    ("bd_hs_params_create", _I, [_P, _I, _P, _P, _F, _I, _F, ctypes.POINTER(_P)]),
    ("bd_hs_params_destroy", None, [_P]),
    ("bd_integral", _I, [_P, _P, _I, _I, _I, _P, _I]),
    ("bd_bad_describe", _I, [_P, _P, _P, _I, _I, _I, _P, _I, _P]),
    ("bd_hashsift_warp", _I, [_P, _P, _P, _I, _I, _I, _P, _I, _P]),
    ("bd_hashsift_hist", _I, [_P, _P, _I, _P]),
    ("bd_hashsift_project", _I, [_P, _P, _P, _I, _P]),
    ("bd_hashsift_describe", _I, [_P, _P, _P, _I, _I, _I, _P, _I, _P, _P]),
    ("bd_match", _I, [_P, _P, _I, _P, _I, _I, _I, _I, _P]),
    ("bd_match_tc", _I, [_P, _P, _I, _P, _I, _I, _I, _I, _P]),
    ("bd_batch_create", _I, [_P, _P, _P, _I, _P, _P, _P, _P, ctypes.POINTER(_P)]),
    ("bd_batch_destroy", None, [_P]),
    ("bd_batch_set_config", _I, [_P, _P]),
    ("bd_batch_get_config", _I, [_P, _P]),
    ("bd_describe_batch", _I, [_P, _P, _P, _P, _P, _P, _I]),
    ("bd_batch_autotune", _I, [_P, _P, _P, _P, _P, _P, _I, _P, ctypes.POINTER(_F)]),
    ("bd_train_create", _I, [_P, _P, _I, _I, _F, _F, _F, ctypes.POINTER(_P)]),
    ("bd_train_destroy", None, [_P]),
    ("bd_train_forward", _I, [_P, _P, _P, _P, _P, _P, _P, _P, _P]),
    ("bd_train_backward", _I, [_P, _P, _P, _P, _P, _P, _P, _P, _P]),
    ("bd_bad_describe_noalloc", _I, [_P, _P, _I, _I, _I, _P, _I, _P, _P]),
    ("bd_match_batch", _I, [_P, _P, _I]),
    ("bd_hs_params_set_variant", _I, [_P, _I]),
    ("bd_match_mnn", _I, [_P, _P, _I, _P, _I, _I, _I, _I, _I, _P, _P]),
    ("bd_select_feature", _I, [_P, _P, _I, _P, _P, _I, _P, _P, _I, _P, _P, _P]),
    ("bd_probe", _I, [_P, _I, _P, ctypes.c_size_t, ctypes.c_size_t, _I, _P,
                      ctypes.POINTER(ctypes.c_uint64)]),
    ("bd_batch_set_timeline", _I, [_P, _I]),
    ("bd_batch_set_wait_limit", _I, [_P, ctypes.c_uint64]),
    ("bd_batch_set_matches", _I, [_P, _P, _I]),
    ("bd_batch_get_timeline", _I, [_P, _P, _I, ctypes.POINTER(_I)]),
]

_lock = threading.Lock()
_lib = None


class BindescError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def lib() -> ctypes.CDLL:
    """The loaded library; raises if it has not been built (no fallback)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise ImportError(
                    f"{LIB_PATH} is missing: build it with `python -c 'import __graft_entry__ as g; "
                    "g.build()'` (or paper_2108_08380_gb300/build.py); there is no CPU fallback")
            L = ctypes.CDLL(LIB_PATH)
            for name, res, args in _SIGS:
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
        return _lib


def kernel_launches() -> int:
    """Kernels launched by the library in this process so far."""
    return int(lib().bd_kernel_launches())


def exported_names():
    return [s[0] for s in _SIGS]


# --------------------------------------------------------------------------
# raw C calls under their C names (pointers and sizes only)
# --------------------------------------------------------------------------

def _fwd(name):
    def call(*args):
        return getattr(lib(), name)(*args)
    call.__name__ = name
    call.__doc__ = f"Direct call of {name} (see include/bindesc.h)."
    return call


for _name, _r, _a in _SIGS:
    globals()[_name] = _fwd(_name)


# --------------------------------------------------------------------------
# torch conveniences
# --------------------------------------------------------------------------

def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(None)


def _np_ptr(a):
    return ctypes.c_void_p(a.ctypes.data)


_live_contexts = weakref.WeakSet()
_exit_hook = []


def _close_live_contexts():
    """At interpreter exit, closes every context still open (and the plans
    and parameter sets made from it) while the CUDA runtime is still up."""
    for c in list(_live_contexts):
        try:
            c.close()
        except Exception:
            pass


class Context:
    """Owns a bd_ctx on one CUDA device; calls enqueue on the current torch stream.
    Contexts still open at interpreter exit are closed by an exit handler
    registered after CUDA is initialised (exit handlers run last-in, first-out,
    so it runs before the runtime's own)."""

    def __init__(self, device: int = 0, stream=None):
        import torch
        self._torch = torch
        self.device = int(device)
        h = ctypes.c_void_p()
        s = stream if stream is not None else torch.cuda.current_stream(self.device).cuda_stream
        st = lib().bd_create(self.device, ctypes.c_void_p(s), ctypes.byref(h))
        if st != BD_OK:
            raise BindescError(st, "bd_create failed (an sm_103 GPU is required)")
        self.handle = h
        self._explicit_stream = stream is not None
        self._children = weakref.WeakSet()
        _live_contexts.add(self)
        if not _exit_hook:
            atexit.register(_close_live_contexts)
            _exit_hook.append(True)

    def _adopt(self, child):
        self._children.add(child)
        return child

    def close(self):
        """Destroys the context after every parameter set, batch plan and
        training plan created from it that is still alive."""
        if getattr(self, "handle", None):
            for child in list(self._children):
                child.close()
            lib().bd_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st, what):
        if st != BD_OK:
            msg = lib().bd_last_error(self.handle)
            raise BindescError(st, f"{what}: {msg.decode() if msg else ''}")

    def _stream(self):
        if not self._explicit_stream:
            s = self._torch.cuda.current_stream(self.device).cuda_stream
            lib().bd_set_stream(self.handle, ctypes.c_void_p(s))

    # ---- status ---------------------------------------------------------
    def sync_status(self) -> int:
        f = ctypes.c_uint32(0)
        st = lib().bd_sync_status(self.handle, ctypes.byref(f))
        if st not in (BD_OK, BD_ERR_DEVICE_CHECK, BD_ERR_TIMEOUT):
            self._check(st, "bd_sync_status")
        return int(f.value)

    def rescued_count(self, reset: bool = False) -> int:
        c = ctypes.c_uint64(0)
        self._check(lib().bd_rescued_count(self.handle, ctypes.byref(c), int(reset)), "bd_rescued_count")
        return int(c.value)

    def trace(self, on: bool = True):
        self._check(lib().bd_trace_enable(self.handle, int(on)), "bd_trace_enable")

    def trace_reset(self):
        self._check(lib().bd_trace_reset(self.handle), "bd_trace_reset")

    def trace_read(self, max_marks: int = 256):
        """[(kernel name, ms)] of the traced kernels since the last reset ('begin' gaps dropped)."""
        ms = (ctypes.c_float * max_marks)()
        lab = (ctypes.c_char_p * max_marks)()
        n = lib().bd_trace_read(self.handle, max_marks, ms, lab)
        if n < 0:
            raise BindescError(BD_ERR_CUDA, "bd_trace_read failed")
        return [(lab[i].decode(), float(ms[i])) for i in range(n) if lab[i] != b"begin"]

    def trace_read_raw(self, max_marks: int = 256):
        """[(name, ms)] including the 'begin' gaps that separate calls."""
        ms = (ctypes.c_float * max_marks)()
        lab = (ctypes.c_char_p * max_marks)()
        n = lib().bd_trace_read(self.handle, max_marks, ms, lab)
        if n < 0:
            raise BindescError(BD_ERR_CUDA, "bd_trace_read failed")
        return [(lab[i].decode(), float(ms[i])) for i in range(n)]

    def reserve(self, nbytes: int):
        self._check(lib().bd_reserve(self.handle, int(nbytes)), "bd_reserve")

    # ---- parameters -----------------------------------------------------
    def bad_params(self, p) -> "BadParamsHandle":
        return BadParamsHandle(self, p)

    def hs_params(self, p, precision: int = BD_HS_BF16_RESCUE, band: float = -1.0) -> "HsParamsHandle":
        return HsParamsHandle(self, p, precision, band)

    def batch(self, bad, hs, images, kp_offsets) -> "Batch":
        """Plan for a list of uint8 device images (bad / hs params handles or None)."""
        return Batch(self, bad, hs, [(int(t.shape[1]), int(t.shape[0])) for t in images],
                     [int(t.stride(0)) for t in images], kp_offsets)

    # ---- work -----------------------------------------------------------
    def integral(self, img, out=None):
        torch = self._torch
        h, w = img.shape
        if out is None:
            out = torch.empty((h + 1, w + 1), dtype=torch.int32, device=img.device)
        self._stream()
        self._check(lib().bd_integral(self.handle, _ptr(img), w, h, img.stride(0), _ptr(out),
                                      out.stride(0)), "bd_integral")
        return out

    def bad_describe(self, params, img, kps, out=None):
        torch = self._torch
        h, w = img.shape
        n = kps.shape[0]
        if out is None:
            out = torch.empty((n, params.nbits // 32), dtype=torch.int32, device=img.device)
        self._stream()
        self._check(lib().bd_bad_describe(self.handle, params.handle, _ptr(img), w, h, img.stride(0),
                                          _ptr(kps), n, _ptr(out)), "bd_bad_describe")
        return out

    def hashsift_warp(self, params, img, kps, out=None):
        torch = self._torch
        h, w = img.shape
        n = kps.shape[0]
        if out is None:
            out = torch.empty((n, 32, 32), dtype=torch.float32, device=img.device)
        self._stream()
        self._check(lib().bd_hashsift_warp(self.handle, params.handle, _ptr(img), w, h, img.stride(0),
                                           _ptr(kps), n, _ptr(out)), "bd_hashsift_warp")
        return out

    def hashsift_hist(self, patches, out=None):
        torch = self._torch
        n = patches.shape[0]
        if out is None:
            out = torch.empty((n, 128), dtype=torch.float32, device=patches.device)
        self._stream()
        self._check(lib().bd_hashsift_hist(self.handle, _ptr(patches), n, _ptr(out)), "bd_hashsift_hist")
        return out

    def hashsift_project(self, params, hist, out=None):
        torch = self._torch
        n = hist.shape[0]
        if out is None:
            out = torch.empty((n, params.nbits // 32), dtype=torch.int32, device=hist.device)
        self._stream()
        self._check(lib().bd_hashsift_project(self.handle, params.handle, _ptr(hist), n, _ptr(out)),
                    "bd_hashsift_project")
        return out

    def hashsift_describe(self, params, img, kps, out=None, hist_out=None):
        torch = self._torch
        h, w = img.shape
        n = kps.shape[0]
        if out is None:
            out = torch.empty((n, params.nbits // 32), dtype=torch.int32, device=img.device)
        self._stream()
        self._check(lib().bd_hashsift_describe(self.handle, params.handle, _ptr(img), w, h,
                                               img.stride(0), _ptr(kps), n, _ptr(out),
                                               _ptr(hist_out)), "bd_hashsift_describe")
        return out

    def match(self, q, t, nbits: int, ratio_num: int = 4, ratio_den: int = 5, out=None,
              tensor_cores: bool = False):
        """Returns an int32 [nq, 3] tensor viewing bd_match_result records:
        column 0 = idx, column 1 = d1 | d2 << 16, column 2 = accept.
        tensor_cores selects bd_match_tc (same results)."""
        torch = self._torch
        nq, nt = q.shape[0], t.shape[0]
        if out is None:
            out = torch.empty((nq, 3), dtype=torch.int32, device=q.device)
        self._stream()
        fn = lib().bd_match_tc if tensor_cores else lib().bd_match
        self._check(fn(self.handle, _ptr(q), nq, _ptr(t), nt, nbits, ratio_num, ratio_den, _ptr(out)),
                    "bd_match_tc" if tensor_cores else "bd_match")
        return out


    def match_batch(self, jobs, ratio_num: int = 4, ratio_den: int = 5, outs=None):
        """bd_match_batch: jobs = [(q, t, nbits), ...] (at most 8); returns the
        records tensors, one per job, as match() returns them."""
        torch = self._torch
        n = len(jobs)
        arr = (MatchJob * max(n, 1))()
        res = []
        for k, (q, t, nbits) in enumerate(jobs):
            out = outs[k] if outs is not None else torch.empty((q.shape[0], 3), dtype=torch.int32,
                                                              device=q.device)
            res.append(out)
            arr[k] = MatchJob(q.data_ptr(), t.data_ptr(), out.data_ptr(), q.shape[0], t.shape[0],
                              nbits, ratio_num, ratio_den)
        self._stream()
        self._check(lib().bd_match_batch(self.handle, ctypes.cast(arr, ctypes.c_void_p), n),
                    "bd_match_batch")
        return res

    def match_mnn(self, q, t, nbits: int, ratio_num: int = 4, ratio_den: int = 5,
                  tensor_cores: bool = False, out=None, mnn=None):
        """Mutual nearest neighbours: (records as match() returns them,
        int32 [nq] partner index or -1)."""
        torch = self._torch
        nq, nt = q.shape[0], t.shape[0]
        if out is None:
            out = torch.empty((nq, 3), dtype=torch.int32, device=q.device)
        if mnn is None:
            mnn = torch.empty(nq, dtype=torch.int32, device=q.device)
        self._stream()
        self._check(lib().bd_match_mnn(self.handle, _ptr(q), nq, _ptr(t), nt, nbits, ratio_num,
                                       ratio_den, int(bool(tensor_cores)), _ptr(out), _ptr(mnn)),
                    "bd_match_mnn")
        return out, mnn

    def select_feature(self, patches, sim_ap, sim_an, tau: int, centres, sides):
        """bd_select_feature: patches uint8 [3, n, 32, 32] (device), sim_ap / sim_an
        int32 [n] (device), centres int32 [J, 4] and sides int32 [J] (host numpy).
        Returns (theta_q int32 [J], loss int64 [J], best int32 [1]) device tensors."""
        import numpy as np
        torch = self._torch
        n = patches.shape[1] if patches.dim() == 4 else patches.shape[0] // 3
        c = np.ascontiguousarray(centres, dtype=np.int32).reshape(-1, 4)
        s = np.ascontiguousarray(sides, dtype=np.int32).reshape(-1)
        J = c.shape[0]
        tq = torch.empty(J, dtype=torch.int32, device=patches.device)
        loss = torch.empty(J, dtype=torch.int64, device=patches.device)
        best = torch.empty(1, dtype=torch.int32, device=patches.device)
        self._stream()
        self._check(lib().bd_select_feature(self.handle, _ptr(patches), n, _ptr(sim_ap), _ptr(sim_an),
                                            int(tau), _np_ptr(c), _np_ptr(s), J, _ptr(tq),
                                            _ptr(loss), _ptr(best)), "bd_select_feature")
        return tq, loss, best

    def probe(self, kind: int, reps: int, table=None, window_words: int = 0, sink=None) -> int:
        """Enqueues one bd_probe kernel on the current stream; returns the
        loads / instructions it performs (time it with events around the call)."""
        torch = self._torch
        if sink is None:
            sink = torch.zeros(1, dtype=torch.int32, device="cuda")
        units = ctypes.c_uint64(0)
        tw = table.numel() if table is not None else 0
        self._stream()
        self._check(lib().bd_probe(self.handle, kind, _ptr(table), tw, window_words, reps,
                                   _ptr(sink), ctypes.byref(units)), "bd_probe")
        return int(units.value)


class MatchJob(ctypes.Structure):
    """bd_match_job."""
    _fields_ = [("q", ctypes.c_void_p), ("t", ctypes.c_void_p), ("out", ctypes.c_void_p),
                ("nq", ctypes.c_int), ("nt", ctypes.c_int), ("nbits", ctypes.c_int),
                ("ratio_num", ctypes.c_int), ("ratio_den", ctypes.c_int)]


class BatchConfig(ctypes.Structure):
    _fields_ = [("bad_kp_per_item", ctypes.c_int), ("ctas_per_sm", ctypes.c_int),
                ("hs_first", ctypes.c_int), ("hs_kp_per_item", ctypes.c_int),
                ("proj_fused", ctypes.c_int), ("bad_shared", ctypes.c_int),
                ("proj_half", ctypes.c_int)]

    def as_dict(self):
        return {"bad_kp_per_item": self.bad_kp_per_item, "ctas_per_sm": self.ctas_per_sm,
                "hs_first": self.hs_first, "hs_kp_per_item": self.hs_kp_per_item,
                "proj_fused": self.proj_fused, "bad_shared": self.bad_shared,
                "proj_half": self.proj_half}


class BatchEvent(ctypes.Structure):
    """bd_batch_event: one work item of the persistent kernel."""
    _fields_ = [("kind", ctypes.c_int32), ("index", ctypes.c_int32), ("sm", ctypes.c_int32),
                ("cta", ctypes.c_int32), ("t_claim", ctypes.c_uint64),
                ("t_ready", ctypes.c_uint64), ("t_end", ctypes.c_uint64)]


# work item kinds of the batched kernel's queue (bd_batch_event.kind)
BD_ITEM_II_TILE, BD_ITEM_HASHSIFT, BD_ITEM_BAD, BD_ITEM_PROJ, BD_ITEM_MATCH = 0, 1, 3, 4, 5
BD_ITEM_MATCH = 5
# descriptor of a batch matching (bd_batch_match.desc)
BD_DESC_BAD, BD_DESC_HASHSIFT = 0, 1


class BatchMatch(ctypes.Structure):
    """bd_batch_match: one matching done by the batched launch."""
    _fields_ = [("desc", ctypes.c_int), ("query_image", ctypes.c_int),
                ("train_image", ctypes.c_int), ("ratio_num", ctypes.c_int),
                ("ratio_den", ctypes.c_int), ("out", ctypes.c_void_p)]
BATCH_EVENT_DTYPE = [("kind", "<i4"), ("index", "<i4"), ("sm", "<i4"), ("cta", "<i4"),
                     ("t_claim", "<u8"), ("t_ready", "<u8"), ("t_end", "<u8")]


class Batch:
    """A bd_batch plan: many images described by one persistent launch."""

    def __init__(self, ctx: Context, bad, hs, sizes, pitches, kp_offsets):
        import numpy as np
        self.ctx = ctx
        self.bad, self.hs = bad, hs
        self.n_img = len(sizes)
        w = np.ascontiguousarray([s[0] for s in sizes], dtype=np.int32)
        h = np.ascontiguousarray([s[1] for s in sizes], dtype=np.int32)
        p = np.ascontiguousarray(pitches, dtype=np.int32)
        o = np.ascontiguousarray(kp_offsets, dtype=np.int32)
        self._keep = (w, h, p, o)
        self.n_kp = int(o[-1])
        hd = ctypes.c_void_p()
        st = lib().bd_batch_create(ctx.handle, bad.handle if bad else None, hs.handle if hs else None,
                                   self.n_img, _np_ptr(w), _np_ptr(h), _np_ptr(p), _np_ptr(o),
                                   ctypes.byref(hd))
        ctx._check(st, "bd_batch_create")
        self.handle = hd
        ctx._adopt(self)

    def close(self):
        if getattr(self, "handle", None):
            lib().bd_batch_destroy(self.handle)
            self.handle = None

    def _ptrs(self, imgs):
        arr = (ctypes.c_void_p * self.n_img)(*[t.data_ptr() for t in imgs])
        return arr

    def describe(self, imgs, kps, bad_out=None, hs_out=None, graph: bool = False):
        self.ctx._stream()
        arr = self._ptrs(imgs)
        st = lib().bd_describe_batch(self.ctx.handle, self.handle, ctypes.cast(arr, ctypes.c_void_p),
                                     _ptr(kps), _ptr(bad_out), _ptr(hs_out), int(graph))
        self.ctx._check(st, "bd_describe_batch")

    def set_config(self, bad_kp_per_item: int, ctas_per_sm: int, hs_first: int,
                   hs_kp_per_item: int = 4, proj_fused: int = 0, bad_shared: int = 0,
                   proj_half: int = 0):
        c = BatchConfig(bad_kp_per_item, ctas_per_sm, hs_first, hs_kp_per_item, proj_fused,
                        bad_shared, proj_half)
        self.ctx._check(lib().bd_batch_set_config(self.handle, ctypes.byref(c)), "bd_batch_set_config")

    def config(self) -> dict:
        c = BatchConfig()
        self.ctx._check(lib().bd_batch_get_config(self.handle, ctypes.byref(c)), "bd_batch_get_config")
        return c.as_dict()

    def autotune(self, imgs, kps, bad_out=None, hs_out=None, reps: int = 3):
        self.ctx._stream()
        arr = self._ptrs(imgs)
        c = BatchConfig()
        ms = ctypes.c_float(0)
        st = lib().bd_batch_autotune(self.ctx.handle, self.handle, ctypes.cast(arr, ctypes.c_void_p),
                                     _ptr(kps), _ptr(bad_out), _ptr(hs_out), int(reps),
                                     ctypes.byref(c), ctypes.byref(ms))
        self.ctx._check(st, "bd_batch_autotune")
        return c.as_dict(), float(ms.value)

    def set_matches(self, jobs):
        """jobs: (desc, query_image, train_image, out, ratio_num, ratio_den)
        tuples; out is an int32 (n_kp(query_image), 3) device tensor (or None
        when that image has no keypoints).  [] clears them."""
        arr = (BatchMatch * max(1, len(jobs)))()
        self._match_outs = []
        for i, (desc, qi, ti, out, rn, rd) in enumerate(jobs):
            if out is not None:
                self._match_outs.append(out)  # kept alive with the plan
            arr[i] = BatchMatch(int(desc), int(qi), int(ti), int(rn), int(rd),
                                out.data_ptr() if out is not None else None)
        self.ctx._stream()
        self.ctx._check(lib().bd_batch_set_matches(self.handle, ctypes.cast(arr, ctypes.c_void_p),
                                                   len(jobs)), "bd_batch_set_matches")

    def set_wait_limit(self, ns: int = 0):
        """bd_batch_set_wait_limit: limit of each dependency wait of the
        persistent kernel in ns (0 = the default 2 s)."""
        self.ctx._check(lib().bd_batch_set_wait_limit(self.handle, ctypes.c_uint64(int(ns))),
                        "bd_batch_set_wait_limit")

    def set_timeline(self, enable: bool = True):
        self.ctx._stream()
        self.ctx._check(lib().bd_batch_set_timeline(self.handle, int(bool(enable))),
                        "bd_batch_set_timeline")

    def timeline(self):
        """Item records of the last launch as a numpy structured array
        (fields of bd_batch_event), in queue order."""
        import numpy as np
        n = ctypes.c_int(0)
        self.ctx._check(lib().bd_batch_get_timeline(self.handle, None, 0, ctypes.byref(n)),
                        "bd_batch_get_timeline")
        out = np.zeros(n.value, dtype=BATCH_EVENT_DTYPE)
        assert out.itemsize == ctypes.sizeof(BatchEvent)
        if n.value:
            self.ctx._check(lib().bd_batch_get_timeline(self.handle, _np_ptr(out), n.value,
                                                        ctypes.byref(n)), "bd_batch_get_timeline")
        return out

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class TrainStep:
    """A bd_train plan: relaxed BAD / HashSIFT responses of n triplets of
    32x32 patches, triplet ranking losses with hard-negative mining and anchor
    swap, and the hand-written backward."""

    def __init__(self, ctx: Context, bad, hs_bits: int, n: int, temperature: float = 0.1,
                 tau_bad=None, tau_hs=None):
        self.ctx, self.bad, self.n = ctx, bad, int(n)
        self.kb, self.kh = bad.nbits, int(hs_bits)
        self.tau_bad = self.kb / 2.0 if tau_bad is None else float(tau_bad)
        self.tau_hs = self.kh / 2.0 if tau_hs is None else float(tau_hs)
        h = ctypes.c_void_p()
        st = lib().bd_train_create(ctx.handle, bad.handle, self.kh, self.n, float(temperature),
                                   self.tau_bad, self.tau_hs, ctypes.byref(h))
        ctx._check(st, "bd_train_create")
        self.handle = h
        ctx._adopt(self)

    def close(self):
        if getattr(self, "handle", None):
            lib().bd_train_destroy(self.handle)
            self.handle = None

    def forward(self, patches, theta, W, b, fixed_mining=None):
        """(loss [2] float32 tensor: BAD, HashSIFT; mining [4, n] int32 tensor)."""
        torch = self.ctx._torch
        loss = torch.empty(2, dtype=torch.float32, device=patches.device)
        mining = torch.empty((4, self.n), dtype=torch.int32, device=patches.device)
        self.ctx._stream()
        st = lib().bd_train_forward(self.ctx.handle, self.handle, _ptr(patches), _ptr(theta), _ptr(W),
                                    _ptr(b), _ptr(fixed_mining), _ptr(loss), _ptr(mining))
        self.ctx._check(st, "bd_train_forward")
        return loss, mining

    def backward(self, patches, W, grad_loss):
        """(dpatches, dtheta, dW, db) of grad_loss[0]*L_bad + grad_loss[1]*L_hs."""
        torch = self.ctx._torch
        dev = patches.device
        dth = torch.empty(self.kb, dtype=torch.float32, device=dev)
        dW = torch.empty((128, self.kh), dtype=torch.float32, device=dev)
        db = torch.empty(self.kh, dtype=torch.float32, device=dev)
        dP = torch.empty_like(patches)
        g = grad_loss.to(device=dev, dtype=torch.float32).contiguous()
        self.ctx._stream()
        st = lib().bd_train_backward(self.ctx.handle, self.handle, _ptr(patches), _ptr(W), _ptr(g),
                                     _ptr(dth), _ptr(dW), _ptr(db), _ptr(dP))
        self.ctx._check(st, "bd_train_backward")
        return dP, dth, dW, db

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def triplet_loss(step: "TrainStep", patches, theta, W, b, fixed_mining=None):
    """Differentiable [L_bad, L_hs] of the training step (torch.autograd.Function).
    fixed_mining (device int32 [4, n], optional) replaces the hard-negative
    mining and anchor swap, as in TrainStep.forward; it gets no gradient."""
    return _TripletLoss.apply(step, patches, theta, W, b, fixed_mining)


def _make_autograd():
    import torch

    class TripletLoss(torch.autograd.Function):
        @staticmethod
        def forward(ctx_, step, patches, theta, W, b, fixed_mining=None):
            patches = patches.contiguous()
            W = W.contiguous()
            fm = None if fixed_mining is None else fixed_mining.contiguous()
            loss, mining = step.forward(patches, theta.contiguous(), W, b.contiguous(),
                                        fixed_mining=fm)
            ctx_.step = step
            ctx_.save_for_backward(patches, W)
            return loss

        @staticmethod
        def backward(ctx_, grad):
            patches, W = ctx_.saved_tensors
            dP, dth, dW, db = ctx_.step.backward(patches, W, grad)
            return None, dP, dth, dW, db, None

    return TripletLoss


class _Lazy:
    def __init__(self):
        self.fn = None

    def apply(self, *args):
        if self.fn is None:
            self.fn = _make_autograd()
        return self.fn.apply(*args)


_TripletLoss = _Lazy()


def unpack_matches(m):
    """(idx, d1, d2, accept) numpy arrays from the int32 [nq, 3] result of Context.match."""
    import numpy as np
    a = m.cpu().numpy() if hasattr(m, "cpu") else np.asarray(m)
    a = a.view(np.uint32)
    return (a[:, 0].view(np.int32).copy(), (a[:, 1] & 0xFFFF).astype(np.int32),
            (a[:, 1] >> 16).astype(np.int32), (a[:, 2] & 0xFF).astype(np.uint8))


class BadParamsHandle:
    def __init__(self, ctx: Context, p):
        import numpy as np
        self.ctx = ctx
        self.nbits = int(p.nbits)
        self.nbins = int(p.n_angle_bins)
        self.nlevels = int(len(p.level_scales))
        self._keep = [np.ascontiguousarray(p.centres, dtype=np.uint8),
                      np.ascontiguousarray(p.sides, dtype=np.uint8),
                      np.ascontiguousarray(p.thr_num, dtype=np.int32),
                      np.ascontiguousarray(p.level_scales, dtype=np.float32)]
        c, s, t, ls = self._keep
        h = ctypes.c_void_p()
        st = lib().bd_bad_params_create(ctx.handle, self.nbits, _np_ptr(c), _np_ptr(s), _np_ptr(t),
                                        int(p.thr_den), self.nbins, _np_ptr(ls), self.nlevels,
                                        ctypes.byref(h))
        ctx._check(st, "bd_bad_params_create")
        self.handle = h
        ctx._adopt(self)

    def close(self):
        if getattr(self, "handle", None):
            lib().bd_bad_params_destroy(self.handle)
            self.handle = None

    def table(self):
        import numpy as np
        off = np.empty((self.nlevels, self.nbins, self.nbits, 2, 2), dtype=np.int32)
        sides = np.empty((self.nlevels, self.nbits), dtype=np.int32)
        st = lib().bd_bad_params_table(self.handle, _np_ptr(off), _np_ptr(sides))
        if st != BD_OK:
            raise BindescError(st, "bd_bad_params_table")
        return off, sides

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class HsParamsHandle:
    def __init__(self, ctx: Context, p, precision: int, band: float):
        import numpy as np
        self.ctx = ctx
        self.nbits = int(p.nbits)
        W = np.ascontiguousarray(p.W, dtype=np.float32)
        b = np.ascontiguousarray(p.b, dtype=np.float32)
        h = ctypes.c_void_p()
        st = lib().bd_hs_params_create(ctx.handle, self.nbits, _np_ptr(W), _np_ptr(b), float(p.spacing),
                                       int(precision), float(band), ctypes.byref(h))
        ctx._check(st, "bd_hs_params_create")
        self.handle = h
        ctx._adopt(self)

    def set_variant(self, flags: int):
        """bd_hs_params_set_variant: OR of BD_HS_VARIANT_* (0 = the plain histogram)."""
        st = lib().bd_hs_params_set_variant(self.handle, int(flags))
        if st != BD_OK:
            raise BindescError(st, "bd_hs_params_set_variant")

    def close(self):
        if getattr(self, "handle", None):
            lib().bd_hs_params_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
