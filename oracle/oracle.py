"""ctypes front end of the C oracle (``sme_oracle.c``) -- TEST INFRASTRUCTURE ONLY.

Each wrapper names the passage of the paper its C function follows.  Arrays
are numpy; nothing here computes any part of the method itself.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sme_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "libsme_oracle.so")
_lock = threading.Lock()
_lib = None


def build_oracle(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, no FP contraction) into oracle/_build."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    fresh = os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)
    if fresh and not force:
        return _LIB_PATH
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-std=c99", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
           "-shared", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Params(C.Structure):
    _fields_ = [("width", C.c_int), ("height", C.c_int), ("search_range", C.c_int),
                ("subpel", C.c_int), ("theta", C.c_float), ("epsilon", C.c_float),
                ("max_iters", C.c_int), ("boundary_t_texture", C.c_int)]


@dataclass
class OracleParams:
    width: int
    height: int
    search_range: int = 16
    subpel: int = 1
    theta: float = 2.0
    epsilon: float = 1.0
    max_iters: int = 8
    boundary_t_texture: int = 0  # Sec. 3.1 variant: boundary T judged by texture (four-vector mode ignores it)

    def c(self) -> _Params:
        return _Params(self.width, self.height, self.search_range, self.subpel,
                       self.theta, self.epsilon, self.max_iters, self.boundary_t_texture)

    @property
    def mbs(self) -> int:
        return (self.width // 16) * (self.height // 16)


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        # SME_ORACLE_LIB: a deliberately broken build, for the pin-strength
        # tests (tests/test_oracle_mutations.py); unset in every other use.
        lib = C.CDLL(os.environ.get("SME_ORACLE_LIB") or build_oracle())
        P = C.POINTER
        u8p, i32p = P(C.c_uint8), P(C.c_int)
        lib.orc_valid_range.argtypes = [C.c_int] * 7 + [i32p] * 4
        lib.orc_interp.argtypes = [u8p, C.c_int, C.c_int, C.c_int, C.c_int]
        lib.orc_interp.restype = C.c_int
        lib.orc_texture_sad.argtypes = [u8p, u8p] + [C.c_int] * 6
        lib.orc_texture_sad.restype = C.c_uint32
        lib.orc_shape_sad.argtypes = [u8p, u8p] + [C.c_int] * 6
        lib.orc_shape_sad.restype = C.c_uint32
        lib.orc_classify_frame.argtypes = [u8p, C.c_int, C.c_int, u8p]
        lib.orc_gradient_step.argtypes = [P(_Params), u8p, u8p] + [C.c_int] * 4 + [P(C.c_float)]
        lib.orc_estimate_pair.argtypes = [P(_Params), u8p, u8p, u8p, u8p, C.c_void_p, C.c_void_p,
                                          C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                          C.c_void_p, C.c_void_p]
        lib.orc_estimate_pair.restype = C.c_int
        lib.orc_compensate.argtypes = [P(_Params), u8p, u8p, C.c_void_p, C.c_void_p]
        lib.orc_compensate.restype = C.c_uint64
        lib.orc_psnr.argtypes = [C.c_uint64, C.c_int, C.c_int]
        lib.orc_psnr.restype = C.c_double
        lib.orc_estimate_sequence.argtypes = [P(_Params), u8p, u8p, C.c_int, C.c_int, C.c_void_p,
                                              C.c_void_p] + [C.c_void_p] * 8
        lib.orc_estimate_sequence.restype = C.c_int
        lib.orc_full_search.argtypes = [C.c_void_p, C.c_void_p] + [C.c_int] * 5 + [C.c_void_p] * 2
        lib.orc_full_search.restype = C.c_uint64
        lib.orc_gradient_step_block.argtypes = [P(_Params), u8p, u8p] + [C.c_int] * 5 + [P(C.c_float)]
        lib.orc_estimate_pair4.argtypes = [P(_Params), u8p, u8p, u8p, u8p] + [C.c_void_p] * 7
        lib.orc_estimate_pair4.restype = C.c_int
        lib.orc_compensate4.argtypes = [P(_Params), u8p, u8p, C.c_void_p, C.c_void_p]
        lib.orc_compensate4.restype = C.c_uint64
        lib.orc_estimate_sequence4.argtypes = [P(_Params), u8p, u8p, C.c_int, C.c_int] + [C.c_void_p] * 9
        lib.orc_estimate_sequence4.restype = C.c_int
        _lib = lib
        return lib


def _u8(a):
    a = np.ascontiguousarray(a, dtype=np.uint8)
    return a, a.ctypes.data_as(C.POINTER(C.c_uint8))


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def valid_range(W, H, block, S, h, X0, Y0):
    """Valid set V of one block (Table 1's exhaustive-search convention)."""
    o = [C.c_int() for _ in range(4)]
    _load().orc_valid_range(W, H, block, S, h, X0, Y0, *[C.byref(x) for x in o])
    return tuple(x.value for x in o)


def interp(ref, h, x2, y2):
    """Reference sample at (x2, y2) in 1/h pixel units (MPEG-4 bilinear)."""
    ref, p = _u8(ref)
    return _load().orc_interp(p, ref.shape[1], h, x2, y2)


def texture_sad(ref, cur, h, X0, Y0, dx, dy):
    """Fig. 1 opaque branch: SAD of a 16x16 block displaced by (dx, dy)."""
    ref, pr = _u8(ref)
    cur, pc = _u8(cur)
    return _load().orc_texture_sad(pr, pc, ref.shape[1], h, X0, Y0, dx, dy)


def shape_sad(aref, acur, h, X0, Y0, dx, dy):
    """Fig. 1 boundary branch: alpha mismatches of a 16x16 BAB."""
    aref, pr = _u8(aref)
    acur, pc = _u8(acur)
    return _load().orc_shape_sad(pr, pc, aref.shape[1], h, X0, Y0, dx, dy)


def classify_frame(alpha):
    """Fig. 1 Block_Type: 0 transparent, 1 opaque, 2 boundary per 16x16 MB."""
    alpha, p = _u8(alpha)
    H, W = alpha.shape
    out = np.zeros((H // 16) * (W // 16), np.uint8)
    _load().orc_classify_frame(p, W, H, out.ctypes.data_as(C.POINTER(C.c_uint8)))
    return out


def gradient_step(params: OracleParams, ref, cur, X0, Y0, dx, dy):
    """Sec. 3.2, Eqs. 3-5: one FP32 gradient update (pixels) at displacement d."""
    ref, pr = _u8(ref)
    cur, pc = _u8(cur)
    out = (C.c_float * 2)()
    cp = params.c()
    _load().orc_gradient_step(C.byref(cp), pr, pc, X0, Y0, dx, dy, out)
    return np.array([out[0], out[1]], np.float32)


def _outputs(n):
    return dict(mv=np.zeros((n, 2), np.int16), cost=np.zeros(n, np.uint32),
                disp=np.zeros((n, 2), np.float32), iters=np.zeros(n, np.uint8),
                npos=np.zeros(n, np.uint8), mbclass=np.zeros(n, np.uint8))


def estimate_pair(params: OracleParams, ref, cur, aref, acur, temporal=None, seed=None):
    """Fig. 1 on one frame pair (raster order, Sec. 3.1)."""
    M = params.mbs
    ref, pr = _u8(ref)
    cur, pc = _u8(cur)
    aref, par = _u8(aref)
    acur, pac = _u8(acur)
    tmp = None if temporal is None else np.ascontiguousarray(temporal, np.int16).reshape(M, 2)
    sd = None if seed is None else np.ascontiguousarray(seed, np.float32).reshape(M, 2)
    o = _outputs(M)
    cp = params.c()
    rc = _load().orc_estimate_pair(C.byref(cp), pr, pc, par, pac, _ptr(tmp), _ptr(sd),
                                   _ptr(o["mv"]), _ptr(o["cost"]), _ptr(o["disp"]),
                                   _ptr(o["iters"]), _ptr(o["npos"]), _ptr(o["mbclass"]))
    if rc:
        raise ValueError("oracle rejected the arguments")
    return o


def compensate(params: OracleParams, ref, cur, mv, want_pred=False):
    """Motion compensation + SSE (Sec. 4); returns (sse, pred or None)."""
    ref, pr = _u8(ref)
    cur, pc = _u8(cur)
    mv = np.ascontiguousarray(mv, np.int16).reshape(params.mbs, 2)
    pred = np.zeros_like(ref) if want_pred else None
    cp = params.c()
    sse = _load().orc_compensate(C.byref(cp), pr, pc, _ptr(mv), _ptr(pred))
    if sse == 2 ** 64 - 1:
        raise ValueError("a motion vector lies outside the valid set")
    return sse, pred


def psnr(sse, W, H):
    """PSNR in dB of an 8-bit W x H frame from its SSE."""
    return _load().orc_psnr(int(sse), W, H)


def estimate_sequence(params: OracleParams, luma, alpha, ref_distance=1, temporal_in=None,
                      seed=None, want_pred=False):
    """Fig. 1 over a sequence of frames; pair k = (frame k, frame k + ref_distance)."""
    luma, pl = _u8(luma)
    alpha, pa = _u8(alpha)
    F = luma.shape[0]
    P, M = F - ref_distance, params.mbs
    tmp = None if temporal_in is None else np.ascontiguousarray(temporal_in, np.int16).reshape(M, 2)
    sd = None if seed is None else np.ascontiguousarray(seed, np.float32).reshape(P, M, 2)
    o = {k: v.reshape((P, M) + v.shape[1:]) for k, v in _outputs(P * M).items()}
    o["sse"] = np.zeros(P, np.uint64)
    pred = np.zeros((P,) + luma.shape[1:], np.uint8) if want_pred else None
    cp = params.c()
    rc = _load().orc_estimate_sequence(C.byref(cp), pl, pa, F, ref_distance, _ptr(tmp), _ptr(sd),
                                       _ptr(o["mv"]), _ptr(o["cost"]), _ptr(o["disp"]),
                                       _ptr(o["iters"]), _ptr(o["npos"]), _ptr(o["mbclass"]),
                                       _ptr(o["sse"]), _ptr(pred))
    if rc:
        raise ValueError("oracle rejected the arguments")
    o["pred"] = pred
    o["psnr"] = np.array([psnr(s, params.width, params.height) for s in o["sse"]])
    return o


def full_search(ref, cur, W, H, h, S, block=16):
    """Exhaustive search over V (Sec. 1, Table 1 ES row).

    With ref/cur None only the positions are counted.  Returns
    (best_mv [n,2], best_sad [n], total positions compared)."""
    n = (W // block) * (H // block)
    bm = np.zeros((n, 2), np.int16)
    bs = np.zeros(n, np.uint32)
    if ref is None:
        total = _load().orc_full_search(None, None, W, H, h, S, block, None, None)
        return None, None, total
    ref = np.ascontiguousarray(ref, np.uint8)
    cur = np.ascontiguousarray(cur, np.uint8)
    total = _load().orc_full_search(_ptr(ref), _ptr(cur), W, H, h, S, block, _ptr(bm), _ptr(bs))
    return bm, bs, total


# ---- four motion vectors per MB (Sec. 3.2: the recursive search on 8x8 blocks) ----

def gradient_step_block(params: OracleParams, ref, cur, X0, Y0, n, dx, dy):
    """Eqs. 3-5 over the n x n block at (X0, Y0): one FP32 update (pixels)."""
    ref, pr = _u8(ref)
    cur, pc = _u8(cur)
    out = (C.c_float * 2)()
    cp = params.c()
    _load().orc_gradient_step_block(C.byref(cp), pr, pc, X0, Y0, n, dx, dy, out)
    return np.array([out[0], out[1]], np.float32)


def _outputs4(n):
    return dict(mv=np.zeros((n, 4, 2), np.int16), cost=np.zeros((n, 4), np.uint32),
                disp=np.zeros((n, 4, 2), np.float32), iters=np.zeros((n, 4), np.uint8),
                npos=np.zeros((n, 4), np.uint8), mbclass=np.zeros(n, np.uint8))


def estimate_pair4(params: OracleParams, ref, cur, aref, acur, temporal4=None):
    """Fig. 1 at MB level, then the pixel recursive search of each 8x8 block
    (four vectors per MB); temporal4 [M, 4, 2] or None."""
    M = params.mbs
    ref, pr = _u8(ref)
    cur, pc = _u8(cur)
    aref, par = _u8(aref)
    acur, pac = _u8(acur)
    tmp = None if temporal4 is None else np.ascontiguousarray(temporal4, np.int16).reshape(M, 4, 2)
    o = _outputs4(M)
    cp = params.c()
    rc = _load().orc_estimate_pair4(C.byref(cp), pr, pc, par, pac, _ptr(tmp), _ptr(o["mv"]), _ptr(o["cost"]),
                                    _ptr(o["disp"]), _ptr(o["iters"]), _ptr(o["npos"]), _ptr(o["mbclass"]))
    if rc:
        raise ValueError("oracle rejected the arguments")
    return o


def compensate4(params: OracleParams, ref, cur, mv4, want_pred=False):
    """Motion compensation with one vector per 8x8 block; (sse, pred or None)."""
    ref, pr = _u8(ref)
    cur, pc = _u8(cur)
    mv4 = np.ascontiguousarray(mv4, np.int16).reshape(params.mbs, 4, 2)
    pred = np.zeros_like(ref) if want_pred else None
    cp = params.c()
    sse = _load().orc_compensate4(C.byref(cp), pr, pc, _ptr(mv4), _ptr(pred))
    if sse == 2 ** 64 - 1:
        raise ValueError("a motion vector lies outside the valid set")
    return sse, pred


def estimate_sequence4(params: OracleParams, luma, alpha, ref_distance=1, temporal_in4=None, want_pred=False):
    """Four vectors per MB over a sequence; outputs [P, M, 4, ...] (mbclass [P, M])."""
    luma, pl = _u8(luma)
    alpha, pa = _u8(alpha)
    F = luma.shape[0]
    P, M = F - ref_distance, params.mbs
    tmp = None if temporal_in4 is None else np.ascontiguousarray(temporal_in4, np.int16).reshape(M, 4, 2)
    o = {k: v.reshape((P, M) + v.shape[1:]) for k, v in _outputs4(P * M).items()}
    o["sse"] = np.zeros(P, np.uint64)
    pred = np.zeros((P,) + luma.shape[1:], np.uint8) if want_pred else None
    cp = params.c()
    rc = _load().orc_estimate_sequence4(C.byref(cp), pl, pa, F, ref_distance, _ptr(tmp), _ptr(o["mv"]),
                                        _ptr(o["cost"]), _ptr(o["disp"]), _ptr(o["iters"]), _ptr(o["npos"]),
                                        _ptr(o["mbclass"]), _ptr(o["sse"]), _ptr(pred))
    if rc:
        raise ValueError("oracle rejected the arguments")
    o["pred"] = pred
    o["psnr"] = np.array([psnr(s, params.width, params.height) for s in o["sse"]])
    return o
