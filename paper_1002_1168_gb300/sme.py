"""Python binding of the C ABI in include/sme.h (argument marshalling only).

Every step of the motion-estimation pass runs in the CUDA library
``_build/libsme.so``; PyTorch only provides device memory and the stream.
There is no CPU fallback: if the library or a GPU is missing, calls raise.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libsme.so")

SME_TRANSPARENT, SME_OPAQUE, SME_BOUNDARY = 0, 1, 2
SME_OPT_SCHEDULE, SME_OPT_PAIR_WARPS, SME_OPT_MB_CTAS_PER_SM, SME_OPT_SPECULATE = 1, 2, 3, 4
SME_OPT_CLUSTER_SIZE = 5
SME_OPT_PAIR_DIRECT = 6
SME_OPT_FOUR_MV = 7
SME_OPT_BOUNDARY_T_TEXTURE = 8
SCHEDULES = {"auto": 0, "mb": 1, "pair": 2, "cluster": 3, "sparse": 4}
STATUS = {0: "SME_OK", 1: "SME_ERR_ARG", 2: "SME_ERR_SIZE", 3: "SME_ERR_CUDA", 4: "SME_ERR_TIMEOUT",
          5: "SME_ERR_STATE", 6: "SME_ERR_NOMEM", 7: "SME_ERR_RANGE", 8: "SME_ERR_SCRATCH"}

# Every entry point declared in include/sme.h.
EXPORTS = [
    "sme_default_params", "sme_strerror", "sme_create", "sme_destroy", "sme_set_stream",
    "sme_synchronize", "sme_classify", "sme_classify_table", "sme_packed_words", "sme_estimate_sequence",
    "sme_estimate_sequence_host", "sme_set_reference", "sme_set_current", "sme_estimate",
    "sme_advance", "sme_score", "sme_get_temporal_field", "sme_set_temporal_field", "sme_set_seed_field",
    "sme_compensate", "sme_psnr", "sme_eval_costs", "sme_gradient_step", "sme_profile_begin",
    "sme_profile_end", "sme_estimate_sequence_noalloc", "sme_set_option", "sme_get_option", "sme_autotune",
    "sme_full_search", "sme_packed_sad_rate_launch",
    "sme_batch_create", "sme_batch_tune", "sme_batch_run", "sme_batch_synchronize", "sme_batch_config",
    "sme_batch_set_config", "sme_batch_run_stage", "sme_batch_class_map", "sme_seednet_forward_active_table",
    "sme_batch_upload", "sme_batch_download", "sme_batch_set_pair_rounds", "sme_batch_run_pair",
    "sme_seednet_temporal_composite", "sme_batch_set_option",
    "sme_batch_destroy", "sme_seednet_param_count", "sme_seednet_create", "sme_seednet_destroy",
    "sme_seednet_set_params", "sme_seednet_get_params", "sme_seednet_features", "sme_seednet_features_table",
    "sme_seednet_forward",
    "sme_seednet_forward_active", "sme_seednet_set_stream", "sme_seednet_synchronize",
    "sme_seednet_gradients", "sme_seednet_train_step", "sme_debug_set_fault",
]


class SmeError(RuntimeError):
    def __init__(self, status, what=""):
        self.status = status
        name = STATUS.get(status, str(status))
        msg = _lib().sme_strerror(status).decode() if _LIB is not None else name
        super().__init__(f"{what}: {name} ({msg})")


class Params(C.Structure):
    _fields_ = [("width", C.c_int), ("height", C.c_int), ("search_range", C.c_int),
                ("subpel", C.c_int), ("theta", C.c_float), ("epsilon", C.c_float),
                ("max_iters", C.c_int), ("ref_distance", C.c_int)]


class Outputs(C.Structure):
    _fields_ = [("mv", C.c_void_p), ("cost", C.c_void_p), ("disp", C.c_void_p),
                ("iters", C.c_void_p), ("npos", C.c_void_p), ("mb_class", C.c_void_p),
                ("sse_mb", C.c_void_p), ("sse", C.c_void_p), ("pred", C.c_void_p)]


class HostIO(C.Structure):
    _fields_ = [("luma", C.c_void_p), ("alpha", C.c_void_p), ("out", Outputs)]


class Sequence(C.Structure):
    _fields_ = [("width", C.c_int), ("height", C.c_int), ("n_frames", C.c_int), ("luma", C.c_void_p),
                ("alpha", C.c_void_p), ("temporal_in", C.c_void_p), ("seed", C.c_void_p), ("out", Outputs)]


_LIB = None
_LOCK = threading.Lock()


def _lib():
    """Load libsme.so (built by build.py / __graft_entry__.build())."""
    global _LIB
    with _LOCK:
        if _LIB is not None:
            return _LIB
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"CUDA library not built: {LIB_PATH} is missing (run build())")
        lib = C.CDLL(LIB_PATH)
        vp, i, ip = C.c_void_p, C.c_int, C.POINTER(C.c_void_p)
        sig = {
            "sme_default_params": (None, [C.POINTER(Params), i, i]),
            "sme_strerror": (C.c_char_p, [i]),
            "sme_create": (i, [ip, C.POINTER(Params), vp]),
            "sme_destroy": (i, [vp]),
            "sme_set_stream": (i, [vp, vp]),
            "sme_synchronize": (i, [vp]),
            "sme_classify": (i, [vp, vp, i, vp, vp]),
            "sme_packed_words": (i, [i]),
            "sme_estimate_sequence": (i, [vp, vp, vp, i, vp, vp, C.POINTER(Outputs)]),
            "sme_estimate_sequence_host": (i, [vp, vp, vp, i, vp, vp, C.POINTER(Outputs)]),
            "sme_set_reference": (i, [vp, vp, vp]),
            "sme_set_current": (i, [vp, vp, vp]),
            "sme_estimate": (i, [vp, C.POINTER(Outputs)]),
            "sme_advance": (i, [vp]),
            "sme_score": (i, [vp, C.POINTER(C.c_double)]),
            "sme_get_temporal_field": (i, [vp, vp]),
            "sme_set_temporal_field": (i, [vp, vp]),
            "sme_set_seed_field": (i, [vp, vp]),
            "sme_compensate": (i, [vp, vp, vp, vp, vp, vp]),
            "sme_psnr": (C.c_double, [C.c_ulonglong, i, i]),
            "sme_eval_costs": (i, [vp, vp, vp, vp, vp, vp, i, vp, vp]),
            "sme_gradient_step": (i, [vp, vp, vp, vp, i, vp]),
            "sme_profile_begin": (i, [vp, i]),
            "sme_profile_end": (i, [vp, C.POINTER(C.c_int), C.POINTER(C.c_double), C.POINTER(C.c_double)]),
            "sme_estimate_sequence_noalloc": (i, [C.POINTER(Params), vp, vp, i, vp, vp, C.POINTER(Outputs), vp]),
            "sme_set_option": (i, [vp, i, i]),
            "sme_get_option": (i, [vp, i, C.POINTER(C.c_int)]),
            "sme_full_search": (i, [vp, vp, i, vp, vp]),
            "sme_packed_sad_rate_launch": (i, [i, i, vp, vp, C.POINTER(C.c_int)]),
            "sme_autotune": (i, [vp, vp, vp, i, C.POINTER(Outputs), i]),
            "sme_batch_create": (i, [ip, C.POINTER(Params), C.POINTER(Sequence), i, vp]),
            "sme_batch_tune": (i, [vp, i]),
            "sme_batch_run": (i, [vp]),
            "sme_batch_synchronize": (i, [vp]),
            "sme_batch_config": (i, [vp, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int),
                                     C.POINTER(C.c_float)]),
            "sme_batch_set_config": (i, [vp, i, i, i]),
            "sme_batch_run_stage": (i, [vp, i]),
            "sme_batch_set_pair_rounds": (i, [vp, i]),
            "sme_batch_set_option": (i, [vp, i, i]),
            "sme_batch_run_pair": (i, [vp, i]),
            "sme_batch_upload": (i, [vp, C.POINTER(HostIO), i]),
            "sme_batch_download": (i, [vp, C.POINTER(HostIO), i]),
            "sme_batch_class_map": (i, [vp, i, C.POINTER(C.c_void_p)]),
            "sme_seednet_forward_active_table": (i, [vp, vp, i, i, i, vp, i, vp, vp]),
            "sme_batch_destroy": (i, [vp]),
            "sme_seednet_param_count": (i, []),
            "sme_seednet_create": (i, [ip, i, vp]),
            "sme_seednet_destroy": (i, [vp]),
            "sme_seednet_set_params": (i, [vp, vp]),
            "sme_seednet_get_params": (i, [vp, vp]),
            "sme_seednet_features": (i, [vp, vp, i, i, i, i, i, vp, i, vp]),
            "sme_seednet_features_table": (i, [vp, vp, vp, i, i, i, i, vp]),
            "sme_seednet_temporal_composite": (i, [vp, vp, vp, i, i, i, i, vp]),
            "sme_seednet_forward": (i, [vp, vp, i, i, i, vp, vp]),
            "sme_seednet_forward_active": (i, [vp, vp, i, i, i, vp, i, C.c_longlong, vp]),
            "sme_seednet_set_stream": (i, [vp, vp]),
            "sme_seednet_synchronize": (i, [vp]),
            "sme_seednet_gradients": (i, [vp, vp, i, i, i, vp, vp, vp, C.POINTER(C.c_float)]),
            "sme_seednet_train_step": (i, [vp, vp, i, i, i, vp, vp, C.c_float, C.POINTER(C.c_float)]),
            "sme_debug_set_fault": (i, [vp, i, C.c_longlong]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _LIB = lib
        return lib


def psnr(sse, width, height) -> float:
    """PSNR (dB) of an 8-bit frame from its SSE (host computation in the library)."""
    return _lib().sme_psnr(int(sse), int(width), int(height))


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _check(rc, what):
    if rc != 0:
        raise SmeError(rc, what)


OUTPUT_FIELDS = ("mv", "cost", "disp", "iters", "npos", "mb_class", "sse_mb", "sse", "pred")


class Estimator:
    """One context of the library bound to the current CUDA device."""

    def __init__(self, width, height, search_range=16, subpel=1, theta=2.0, epsilon=1.0,
                 max_iters=8, ref_distance=1, four_mv=False, boundary_t_texture=False):
        import torch

        if not torch.cuda.is_available():
            raise RuntimeError("a CUDA GPU is required (no CPU fallback)")
        self.torch = torch
        lib = _lib()
        self.params = Params(width, height, search_range, subpel, theta, epsilon, max_iters, ref_distance)
        self.width, self.height = width, height
        self.M = (width // 16) * (height // 16)
        self.ref_distance = ref_distance
        h = C.c_void_p()
        _check(lib.sme_create(C.byref(h), C.byref(self.params), self._stream()), "sme_create")
        self._h = h
        # four vectors per MB (Sec. 3.2, 8x8 blocks): mv/cost/disp/iters/npos gain a block axis of 4
        self.four_mv = bool(four_mv)
        if self.four_mv:
            self.set_option(SME_OPT_FOUR_MV, 1)
        # Sec. 3.1 variant: boundary MBs judge T by texture against the shape winner of the others
        if boundary_t_texture:
            self.set_option(SME_OPT_BOUNDARY_T_TEXTURE, 1)

    # ------------------------------------------------------------ plumbing
    def _stream(self):
        return C.c_void_p(self.torch.cuda.current_stream().cuda_stream)

    def _bind(self):
        _check(_lib().sme_set_stream(self._h, self._stream()), "sme_set_stream")
        return self._h

    def close(self):
        if getattr(self, "_h", None):
            _lib().sme_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def synchronize(self):
        _check(_lib().sme_synchronize(self._bind()), "sme_synchronize")

    def _alloc_outputs(self, P, want, device):
        t = self.torch
        M, H, W = self.M, self.height, self.width
        B = (4,) if getattr(self, "four_mv", False) else ()
        shapes = {"mv": ((P, M) + B + (2,), t.int16), "cost": ((P, M) + B, t.int32),
                  "disp": ((P, M) + B + (2,), t.float32), "iters": ((P, M) + B, t.uint8),
                  "npos": ((P, M) + B, t.uint8), "mb_class": ((P, M), t.uint8),
                  "sse_mb": ((P, M), t.int32), "sse": ((P,), t.int64), "pred": ((P, H, W), t.uint8)}
        out = {}
        for k in OUTPUT_FIELDS:
            if k == "mv" or k in want:
                shp, dt = shapes[k]
                out[k] = t.empty(shp, dtype=dt, device=device)
        return out

    @staticmethod
    def _outputs_struct(out):
        return Outputs(*[_ptr(out.get(k)) for k in OUTPUT_FIELDS])

    # ---------------------------------------------------------- interface
    def estimate_sequence(self, luma, alpha, temporal_in=None, seed=None,
                          want=("cost", "disp", "iters", "npos", "mb_class", "sse"), out=None,
                          sync=True):
        """Fig. 1 over a sequence: luma/alpha uint8 CUDA tensors [F, H, W]."""
        F = luma.shape[0]
        P = F - self.ref_distance
        assert luma.is_cuda and alpha.is_cuda and luma.is_contiguous() and alpha.is_contiguous()
        if out is None:
            out = self._alloc_outputs(P, want, luma.device)
        st = self._outputs_struct(out)
        rc = _lib().sme_estimate_sequence(self._bind(), _ptr(luma), _ptr(alpha), F, _ptr(temporal_in),
                                          _ptr(seed), C.byref(st))
        _check(rc, "sme_estimate_sequence")
        if sync:
            self.synchronize()
        return out

    def estimate_sequence_host(self, luma, alpha, temporal_in=None, seed=None,
                               want=("cost", "disp", "iters", "npos", "mb_class", "sse"), out=None):
        """Same as estimate_sequence with host tensors (pinned for fast copies)."""
        F = luma.shape[0]
        P = F - self.ref_distance
        if out is None:
            out = self._alloc_outputs(P, want, "cpu")
        st = self._outputs_struct(out)
        rc = _lib().sme_estimate_sequence_host(self._bind(), _ptr(luma), _ptr(alpha), F,
                                               _ptr(temporal_in), _ptr(seed), C.byref(st))
        _check(rc, "sme_estimate_sequence_host")
        return out

    def classify_table(self, frames, out=None, sync=True):
        """MB classes [n, M] uint8 of the alpha planes whose device addresses
        are in frames (int64 CUDA tensor [n]; 0 = an empty plane), in one launch."""
        t = self.torch
        n = frames.numel()
        assert frames.is_cuda and frames.dtype == t.int64 and frames.is_contiguous()
        cls = out if out is not None else t.empty((n, self.M), dtype=t.uint8, device=frames.device)
        _check(_lib().sme_classify_table(self._bind(), _ptr(frames), n, _ptr(cls)), "sme_classify_table")
        if sync:
            self.synchronize()
        return cls

    def classify(self, alpha, want_packed=True, out=None, sync=True):
        """MB classes [F, M] uint8 (into out if given) and, optionally, the
        packed alpha rows."""
        t = self.torch
        F = alpha.shape[0]
        cls = out if out is not None else t.empty((F, self.M), dtype=t.uint8, device=alpha.device)
        wp = _lib().sme_packed_words(self.width)
        packed = t.empty((F, self.height, wp), dtype=t.int32, device=alpha.device) if want_packed else None
        _check(_lib().sme_classify(self._bind(), _ptr(alpha), F, _ptr(cls), _ptr(packed)), "sme_classify")
        if sync:
            self.synchronize()
        return cls, packed

    def compensate(self, ref, cur, mv, want_pred=True):
        t = self.torch
        sse = t.zeros(1, dtype=t.int64, device=ref.device)
        pred = t.empty_like(ref) if want_pred else None
        _check(_lib().sme_compensate(self._bind(), _ptr(ref), _ptr(cur), _ptr(mv), _ptr(pred), _ptr(sse)),
               "sme_compensate")
        self.synchronize()
        return int(sse.item()), pred

    def eval_costs(self, ref, cur, aref, acur, queries):
        t = self.torch
        q = t.as_tensor(np.asarray(queries, np.int32).reshape(-1, 3)).to(ref.device)
        n = q.shape[0]
        ts = t.empty(n, dtype=t.int32, device=ref.device)
        ss = t.empty(n, dtype=t.int32, device=ref.device) if aref is not None else None
        _check(_lib().sme_eval_costs(self._bind(), _ptr(ref), _ptr(cur), _ptr(aref), _ptr(acur), _ptr(q), n,
                                     _ptr(ts), _ptr(ss)), "sme_eval_costs")
        self.synchronize()
        return ts, ss

    def gradient_step(self, ref, cur, queries):
        t = self.torch
        q = t.as_tensor(np.asarray(queries, np.int32).reshape(-1, 3)).to(ref.device)
        n = q.shape[0]
        d = t.empty((n, 2), dtype=t.float32, device=ref.device)
        _check(_lib().sme_gradient_step(self._bind(), _ptr(ref), _ptr(cur), _ptr(q), n, _ptr(d)),
               "sme_gradient_step")
        self.synchronize()
        return d

    # ------------------------------------------------ stateful pair API
    def set_reference(self, luma, alpha):
        _check(_lib().sme_set_reference(self._bind(), _ptr(luma), _ptr(alpha)), "sme_set_reference")

    def set_current(self, luma, alpha):
        _check(_lib().sme_set_current(self._bind(), _ptr(luma), _ptr(alpha)), "sme_set_current")

    def estimate(self, want=("cost", "sse")):
        out = self._alloc_outputs(1, want, "cuda")
        st = self._outputs_struct(out)
        _check(_lib().sme_estimate(self._bind(), C.byref(st)), "sme_estimate")
        return out

    def advance(self):
        _check(_lib().sme_advance(self._bind()), "sme_advance")

    def score(self):
        v = C.c_double()
        _check(_lib().sme_score(self._bind(), C.byref(v)), "sme_score")
        return v.value

    def get_temporal_field(self):
        t = self.torch
        f = t.empty((self.M, 2), dtype=t.int16, device="cuda")
        _check(_lib().sme_get_temporal_field(self._bind(), _ptr(f)), "sme_get_temporal_field")
        return f

    def set_temporal_field(self, field):
        _check(_lib().sme_set_temporal_field(self._bind(), _ptr(field)), "sme_set_temporal_field")

    def set_seed_field(self, seed):
        """Seeds [M, 2] FP32 pixels (CUDA) for the following estimates; None clears."""
        _check(_lib().sme_set_seed_field(self._bind(), _ptr(seed)), "sme_set_seed_field")

    def set_option(self, option, value):
        _check(_lib().sme_set_option(self._h, int(option), int(value)), "sme_set_option")

    def set_schedule(self, name, pair_warps=0, cluster=0):
        """'auto', 'mb' (one warp per MB), 'pair' (one CTA per frame pair) or
        'cluster' (one thread-block cluster per sequence)."""
        self.set_option(SME_OPT_SCHEDULE, SCHEDULES[name])
        self.set_option(SME_OPT_PAIR_WARPS, pair_warps)
        self.set_option(SME_OPT_CLUSTER_SIZE, cluster)

    def full_search(self, luma, want_sad=True, sync=True):
        """Exhaustive search over V for every MB of every pair (the ES of
        Table 1); returns mv [P, M, 2] int16 and sad [P, M] int32 (device)."""
        t = self.torch
        P = luma.shape[0] - self.ref_distance
        mv = t.empty((P, self.M, 2), dtype=t.int16, device=luma.device)
        sad = t.empty((P, self.M), dtype=t.int32, device=luma.device) if want_sad else None
        _check(_lib().sme_full_search(self._bind(), _ptr(luma), luma.shape[0], _ptr(mv), _ptr(sad)), "sme_full_search")
        if sync:
            self.synchronize()
        return mv, sad

    def get_option(self, option):
        v = C.c_int()
        _check(_lib().sme_get_option(self._h, int(option), C.byref(v)), "sme_get_option")
        return v.value

    def config(self):
        """The execution configuration in use (after autotune: the chosen one)."""
        names = {v: k for k, v in SCHEDULES.items()}
        return {"schedule": names[self.get_option(SME_OPT_SCHEDULE)], "pair_warps": self.get_option(SME_OPT_PAIR_WARPS),
                "mb_ctas_per_sm": self.get_option(SME_OPT_MB_CTAS_PER_SM),
                "speculate": self.get_option(SME_OPT_SPECULATE), "cluster": self.get_option(SME_OPT_CLUSTER_SIZE),
                "pair_direct": self.get_option(SME_OPT_PAIR_DIRECT)}

    def autotune(self, luma, alpha, out=None, trials=3, want=("cost", "disp", "iters", "npos", "mb_class", "sse")):
        """Pick the fastest execution configuration for this sequence shape."""
        F = luma.shape[0]
        if out is None:
            out = self._alloc_outputs(F - self.ref_distance, want, luma.device)
        st = self._outputs_struct(out)
        _check(_lib().sme_autotune(self._bind(), _ptr(luma), _ptr(alpha), F, C.byref(st), int(trials)),
               "sme_autotune")
        return out

    def profile_begin(self, max_calls):
        _check(_lib().sme_profile_begin(self._h, int(max_calls)), "sme_profile_begin")

    def profile_end(self):
        """Returns (calls, classify_ms_total, me_ms_total) since profile_begin."""
        n, a, b = C.c_int(), C.c_double(), C.c_double()
        _check(_lib().sme_profile_end(self._h, C.byref(n), C.byref(a), C.byref(b)), "sme_profile_end")
        return n.value, a.value, b.value

    def debug_set_fault(self, skip_ticket=-1, timeout_ns=0):
        _check(_lib().sme_debug_set_fault(self._h, int(skip_ticket), int(timeout_ns)), "sme_debug_set_fault")


class Batch:
    """Many sequences (luma, alpha CUDA tensors [F, H, W], uneven sizes) in one
    persistent launch.  Outputs are allocated per sequence and reused by every
    run (the work is replayed from a CUDA graph once tuned)."""

    def __init__(self, luma_list, alpha_list, search_range=16, subpel=2, theta=2.0, epsilon=1.0,
                 max_iters=8, ref_distance=1, want=("cost", "disp", "iters", "npos", "mb_class", "sse"),
                 temporal_list=None, seed_list=None, four_mv=False):
        import torch

        self.torch = torch
        lib = _lib()
        W0, H0 = luma_list[0].shape[2], luma_list[0].shape[1]
        self.params = Params(W0, H0, search_range, subpel, theta, epsilon, max_iters, ref_distance)
        self.inputs = list(zip(luma_list, alpha_list))
        self.outputs = []
        n = len(luma_list)
        seqs = (Sequence * n)()
        self._keep = []
        for i, (l, a) in enumerate(self.inputs):
            F, H, W = l.shape
            est_like = Estimator.__new__(Estimator)
            est_like.torch, est_like.M, est_like.height, est_like.width = torch, (W // 16) * (H // 16), H, W
            est_like.four_mv = bool(four_mv)
            out = Estimator._alloc_outputs(est_like, F - ref_distance, want, l.device)
            self.outputs.append(out)
            tmp = None if temporal_list is None else temporal_list[i]
            sd = None if seed_list is None else seed_list[i]
            self._keep += [tmp, sd]
            seqs[i] = Sequence(W, H, F, l.data_ptr(), a.data_ptr(), None if tmp is None else tmp.data_ptr(),
                               None if sd is None else sd.data_ptr(), Estimator._outputs_struct(out))
        h = C.c_void_p()
        stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
        _check(lib.sme_batch_create(C.byref(h), C.byref(self.params), seqs, n, stream), "sme_batch_create")
        self._h = h
        if four_mv:  # Sec. 3.2: four vectors per MB, outputs [P, M, 4, ...]
            _check(lib.sme_batch_set_option(h, SME_OPT_FOUR_MV, 1), "sme_batch_set_option")

    def tune(self, trials=3):
        _check(_lib().sme_batch_tune(self._h, int(trials)), "sme_batch_tune")

    def run(self, sync=True):
        _check(_lib().sme_batch_run(self._h), "sme_batch_run")
        if sync:
            self.synchronize()
        return self.outputs

    def synchronize(self):
        _check(_lib().sme_batch_synchronize(self._h), "sme_batch_synchronize")

    def config(self):
        s_, p_, sp_, ms = C.c_int(), C.c_int(), C.c_int(), C.c_float()
        _check(_lib().sme_batch_config(self._h, C.byref(s_), C.byref(p_), C.byref(sp_), C.byref(ms)),
               "sme_batch_config")
        name = {v: k for k, v in SCHEDULES.items()}[s_.value]
        return {"schedule": name, "param": p_.value, "flag": sp_.value, "tuned_ms": ms.value}

    def host_io(self, host_inputs, host_outputs):
        """The sme_host_io array for host_inputs [(luma, alpha) CPU tensors]
        and host_outputs [{field: CPU tensor}] (pinned for link-speed copies)."""
        n = len(self.inputs)
        io = (HostIO * n)()
        for i in range(n):
            l, a = host_inputs[i]
            o = host_outputs[i] if host_outputs is not None else {}
            io[i] = HostIO(l.data_ptr(), a.data_ptr(), Outputs(*[_ptr(o.get(k)) for k in OUTPUT_FIELDS]))
        return io

    def upload(self, io):
        """Copy every sequence's inputs from host memory (sme_batch_upload)."""
        _check(_lib().sme_batch_upload(self._h, io, len(self.inputs)), "sme_batch_upload")

    def download(self, io):
        """Copy the requested outputs to host memory (sme_batch_download)."""
        _check(_lib().sme_batch_download(self._h, io, len(self.inputs)), "sme_batch_download")

    def run_host(self, io):
        """The whole host-to-host pass: upload, run, download, synchronise."""
        self.upload(io)
        self.run(sync=False)
        self.download(io)
        self.synchronize()
        return io

    def set_pair_rounds(self, on=True):
        """Pair rounds of the sparse schedule (sme_batch_set_pair_rounds)."""
        _check(_lib().sme_batch_set_pair_rounds(self._h, int(bool(on))), "sme_batch_set_pair_rounds")

    def run_pair(self, k):
        """Enqueue the search of pair k of every sequence (pair rounds)."""
        _check(_lib().sme_batch_run_pair(self._h, int(k)), "sme_batch_run_pair")

    def run_stage(self, stage):
        """Enqueue stage 1 (classification) or 2 (search) of one run."""
        _check(_lib().sme_batch_run_stage(self._h, int(stage)), "sme_batch_run_stage")

    def class_map_ptr(self, i):
        """Device address of sequence i's class map [F, M] (uint8)."""
        p = C.c_void_p()
        _check(_lib().sme_batch_class_map(self._h, int(i), C.byref(p)), "sme_batch_class_map")
        return p.value

    def set_config(self, schedule, param=0, flag=1):
        """Use one execution configuration instead of tuning ('mb', 'pair' or
        'sparse'; see sme_batch_set_config)."""
        _check(_lib().sme_batch_set_config(self._h, SCHEDULES[schedule], int(param), int(flag)),
               "sme_batch_set_config")

    def close(self):
        if getattr(self, "_h", None):
            _lib().sme_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class SeedNet:
    """The learned seed proposal network (device weights, FP32 master copy)."""

    def __init__(self, max_cells):
        import torch

        self.torch = torch
        lib = _lib()
        self.max_cells = int(max_cells)
        self.n_params = lib.sme_seednet_param_count()
        h = C.c_void_p()
        _check(lib.sme_seednet_create(C.byref(h), int(max_cells), C.c_void_p(torch.cuda.current_stream().cuda_stream)),
               "sme_seednet_create")
        self._h = h

    def _bind(self):
        """Launch on the current torch stream (as Estimator does)."""
        _check(_lib().sme_seednet_set_stream(self._h, C.c_void_p(self.torch.cuda.current_stream().cuda_stream)),
               "sme_seednet_set_stream")
        return self._h

    def set_params(self, flat):
        flat = np.ascontiguousarray(flat, np.float32)
        assert flat.size == self.n_params
        _check(_lib().sme_seednet_set_params(self._bind(), flat.ctypes.data_as(C.c_void_p)), "sme_seednet_set_params")

    def get_params(self):
        out = np.zeros(self.n_params, np.float32)
        _check(_lib().sme_seednet_get_params(self._bind(), out.ctypes.data_as(C.c_void_p)), "sme_seednet_get_params")
        return out

    def features(self, luma, ref_frame, cur_frame, temporal=None, subpel=2, out=None, n_pairs=1):
        """Input grid(s) of n_pairs frame pairs (ref_frame + q, cur_frame + q);
        [H/4, W/4, 16] for one pair, else [n_pairs, H/4, W/4, 16]."""
        t = self.torch
        F, H, W = luma.shape
        last = max(int(ref_frame), int(cur_frame)) + int(n_pairs) - 1
        if min(int(ref_frame), int(cur_frame)) < 0 or last >= F:
            raise ValueError(f"frames {ref_frame}/{cur_frame} + {n_pairs} pairs outside a {F}-frame sequence")
        if out is None:
            shape = (H // 4, W // 4, 16) if n_pairs == 1 else (n_pairs, H // 4, W // 4, 16)
            out = t.empty(shape, dtype=t.int16, device=luma.device)
        _check(_lib().sme_seednet_features(self._bind(), _ptr(luma), W, H, int(ref_frame), int(cur_frame), int(n_pairs),
                                           _ptr(temporal), int(subpel), _ptr(out)), "sme_seednet_features")
        return out

    def features_table(self, frames, width, height, subpel=2, out=None, temporal=None):
        """Input grids of the pairs whose (reference, current) luma frame
        addresses are in frames (int64 CUDA tensor [n, 2]), in one launch:
        [n, H/4, W/4, 16].  temporal: None or an int64 CUDA tensor [n] of
        temporal-field addresses (0: zeros)."""
        t = self.torch
        n = frames.shape[0]
        assert frames.is_cuda and frames.dtype == t.int64 and frames.is_contiguous() and frames.shape[1] == 2
        if out is None:
            out = t.empty((n, height // 4, width // 4, 16), dtype=t.int16, device=frames.device)
        _check(_lib().sme_seednet_features_table(self._bind(), _ptr(frames), _ptr(temporal), n, width, height,
                                                 int(subpel), _ptr(out)), "sme_seednet_features_table")
        return out

    def temporal_composite(self, fields, classes, n, n_vops, width, height, out):
        """One temporal field per scene for n scenes (sme_seednet_temporal_composite):
        fields, classes int64 CUDA tensors [n, n_vops] of addresses; out [n, M, 2]."""
        _check(_lib().sme_seednet_temporal_composite(self._bind(), _ptr(fields), _ptr(classes), int(n),
                                                     int(n_vops), int(width), int(height), _ptr(out)),
               "sme_seednet_temporal_composite")
        return out

    def forward(self, feat, want_cells=False):
        """feat [n, H/4, W/4, 16] (int16 view of bfloat16) -> seeds [n, M, 2] FP32 px."""
        t = self.torch
        n, Hc, Wc, _ = feat.shape
        seeds = t.empty((n, (Hc // 4) * (Wc // 4), 2), dtype=t.float32, device=feat.device)
        cells = t.empty((n, Hc, Wc, 16), dtype=t.float32, device=feat.device) if want_cells else None
        _check(_lib().sme_seednet_forward(self._bind(), _ptr(feat), n, 4 * Wc, 4 * Hc, _ptr(seeds), _ptr(cells)),
               "sme_seednet_forward")
        return (seeds, cells) if want_cells else seeds

    def forward_active_table(self, feat, rows, n_maps, out=None, seed_rows=None):
        """forward_active with the class maps as a device table [n_maps, n]
        (int64 CUDA tensor) of row addresses; 0 = an empty plane.  With
        seed_rows (int64 CUDA tensor [n] of [M, 2] row addresses) the seeds
        go there instead of `out`."""
        n, Hc, Wc, _ = feat.shape
        t = self.torch
        M = (Hc // 4) * (Wc // 4)
        if seed_rows is None and out is None:
            out = t.empty((n, M, 2), dtype=t.float32, device=feat.device)
        _check(_lib().sme_seednet_forward_active_table(self._bind(), _ptr(feat), n, 4 * Wc, 4 * Hc, _ptr(rows),
                                                        int(n_maps), _ptr(out), _ptr(seed_rows)),
               "sme_seednet_forward_active_table")
        return out

    def forward_active(self, feat, mb_class, out=None):
        """Seeds of the non-transparent MBs, (0, 0) on the others; the layers
        run only near those MBs.  mb_class: [n, M] uint8, or [V, n, M] for V
        VOPs over the same frames (an MB counts if it is visible in any)."""
        t = self.torch
        n, Hc, Wc, _ = feat.shape
        M = (Hc // 4) * (Wc // 4)
        maps = mb_class if mb_class.dim() == 3 else mb_class[None]
        if tuple(maps.shape[1:]) != (n, M) or maps.stride(2) != 1 or maps.stride(1) != M:
            raise ValueError("mb_class must be [n, M] or [V, n, M] with contiguous [n, M] slabs")
        if out is None:
            out = t.empty((n, M, 2), dtype=t.float32, device=feat.device)
        _check(_lib().sme_seednet_forward_active(self._bind(), _ptr(feat), n, 4 * Wc, 4 * Hc, _ptr(maps),
                                                 maps.shape[0], maps.stride(0), _ptr(out)),
               "sme_seednet_forward_active")
        return out

    def synchronize(self):
        """Wait for the network's work; raises if a device-side wait gave up."""
        _check(_lib().sme_seednet_synchronize(self._bind()), "sme_seednet_synchronize")

    def gradients(self, feat, labels, mask):
        n, Hc, Wc, _ = feat.shape
        g = np.zeros(self.n_params, np.float32)
        loss = C.c_float()
        _check(_lib().sme_seednet_gradients(self._bind(), _ptr(feat), n, 4 * Wc, 4 * Hc, _ptr(labels), _ptr(mask),
                                            g.ctypes.data_as(C.c_void_p), C.byref(loss)), "sme_seednet_gradients")
        return loss.value, g

    def train_step(self, feat, labels, mask, lr, want_loss=False):
        n, Hc, Wc, _ = feat.shape
        loss = C.c_float()
        _check(_lib().sme_seednet_train_step(self._bind(), _ptr(feat), n, 4 * Wc, 4 * Hc, _ptr(labels), _ptr(mask),
                                             float(lr), C.byref(loss) if want_loss else None),
               "sme_seednet_train_step")
        return loss.value if want_loss else None

    def close(self):
        if getattr(self, "_h", None):
            _lib().sme_seednet_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def packed_sad_rate(ctas_per_sm=8, iters=50000, reps=3):
    """Measured rate (operations per second, best of `reps` launches timed
    with events on the current stream) of the packed-SAD operation mix the
    integer rooflines count (sme_packed_sad_rate_launch)."""
    import torch

    st = torch.cuda.current_stream()
    n = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count * ctas_per_sm * 256
    out = torch.empty(n, dtype=torch.int32, device="cuda")
    grid = C.c_int()
    best = None
    for _ in range(reps + 1):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        _check(_lib().sme_packed_sad_rate_launch(int(ctas_per_sm), int(iters), _ptr(out), C.c_void_p(st.cuda_stream),
                                                 C.byref(grid)), "sme_packed_sad_rate_launch")
        e1.record(st)
        st.synchronize()
        ms = e0.elapsed_time(e1)
        best = ms if best is None or ms < best else best
    assert grid.value * 256 == n
    return grid.value * 256 * iters * 24 / (best / 1e3)


def pack_params(params):
    """Flatten [(w [cout,3,3,cin], b [cout]), ...] into the library's layout."""
    return np.concatenate([np.concatenate([np.asarray(w, np.float32).ravel(), np.asarray(b, np.float32)])
                           for w, b in params])


def unpack_params(flat, channels=(16, 32, 32, 32, 32, 16)):
    out, o = [], 0
    for li in range(5):
        cin, cout = channels[li], channels[li + 1]
        nw = cout * 9 * cin
        out.append((flat[o:o + nw].reshape(cout, 3, 3, cin), flat[o + nw:o + nw + cout]))
        o += nw + cout
    return out
