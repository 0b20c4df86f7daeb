"""Python binding of the C ABI in include/orbg.h (ctypes).

Argument marshalling only: every step of the decode runs in the CUDA
library.  Names match the C functions.  Array arguments may be torch
tensors (CUDA or CPU) or NumPy arrays; they must be contiguous with the C
type's dtype.  There is no fallback: if liborbg.so is missing or a CUDA
call fails, these functions raise.
"""
import ctypes
import os

import numpy as np

from . import build as _build

ORBG_OK = 0
ORBG_EINVAL = -1
ORBG_ERANK = -2
ORBG_ELIMIT = -3
ORBG_ENAN = -4
ORBG_ENOMEM = -5
ORBG_ECUDA = -6
ORBG_ETIMEOUT = -7
ORBG_MAT_H = 0
ORBG_MAT_G = 1
ORBG_MAX_N = 256
ORBG_MAX_R = 128
ORBG_MAX_QUERY_CAP = 1 << 25
ORBG_DEFAULT_QUERY_CAP = 1 << 20
ORBG_BLOCK_DECODED = 0
ORBG_BLOCK_ABANDONED = 1
ORBG_BLOCK_NAN = 2
ORBG_BLOCK_RANGE = 3
ORBG_NOALLOC_MAX_BLOCKS = 1 << 19
ORBG_FIT_STRIDE = 24

LIB_PATH = _build.LIB
_lib = None


class OrbgTuning(ctypes.Structure):
    """struct orbg_tuning of include/orbg.h."""
    _fields_ = [("warps_per_cta", ctypes.c_int), ("ctas_per_sm", ctypes.c_int),
                ("blocks_per_grab", ctypes.c_int), ("warp_budget", ctypes.c_uint32),
                ("heavy_warps", ctypes.c_int)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class OrbgServerStats(ctypes.Structure):
    """struct orbg_server_stats of include/orbg.h."""
    _fields_ = [(f, ctypes.c_uint64) for f in (
        "submitted", "completed", "blocks_submitted", "blocks_done", "batches",
        "max_batch_blocks", "max_inflight_batches", "pending", "inflight_batches",
        "cancelled")]

    def as_dict(self):
        return {f: int(getattr(self, f)) for f, _ in self._fields_}


class OrbgError(RuntimeError):
    def __init__(self, status, what=""):
        self.status = status
        msg = "%s: %s (%d)" % (what, _status_string(status), status)
        if status == ORBG_ECUDA and _lib is not None:
            msg += " [cuda error %d]" % _lib.orbg_last_cuda_error()
        super().__init__(msg)


def _status_string(s):
    if _lib is None:
        return "status"
    return _lib.orbg_status_string(s).decode()


def load_library(path=None):
    """Load liborbg.so (built by paper_2202_13951_gb300.build)."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise RuntimeError("CUDA library %s is not built; run "
                           "paper_2202_13951_gb300.build.build()" % path)
    lib = ctypes.CDLL(path)
    vp = ctypes.c_void_p
    u32 = ctypes.c_uint32
    i32 = ctypes.c_int
    i64 = ctypes.c_int64
    lib.orbg_load_code.argtypes = [vp, i32, i32, i32, u32, ctypes.POINTER(vp)]
    lib.orbg_load_code_line.argtypes = [vp, i32, i32, i32, u32, i32, i32, ctypes.POINTER(vp)]
    lib.orbg_load_code_model.argtypes = [vp, i32, i32, i32, u32, i32, vp, vp, vp,
                                         ctypes.POINTER(vp)]
    lib.orbg_free_code.argtypes = [vp]
    lib.orbg_code_info.argtypes = [vp, ctypes.POINTER(i32), ctypes.POINTER(i32),
                                   ctypes.POINTER(u32), vp]
    lib.orbg_decode.argtypes = [vp, vp, i64, u32, vp, vp, vp, vp]
    lib.orbg_codeset_create.argtypes = [ctypes.POINTER(vp), i32, ctypes.POINTER(vp)]
    lib.orbg_codeset_free.argtypes = [vp]
    lib.orbg_decode_batched.argtypes = [vp, vp, vp, vp, i64, u32, vp, vp, vp, vp, vp]
    lib.orbg_decode_batched_noalloc.argtypes = [vp, vp, vp, vp, i64, u32, vp, vp, vp, vp, vp]
    lib.orbg_codeset_set_tuning.argtypes = [vp, ctypes.POINTER(OrbgTuning)]
    lib.orbg_codeset_autotune.argtypes = [vp, vp, vp, vp, i64, u32, vp, vp, vp, vp, i32, vp,
                                          ctypes.POINTER(OrbgTuning)]
    lib.orbg_codeset_get_tuning.argtypes = [vp, ctypes.POINTER(OrbgTuning)]
    lib.orbg_probe_int_lanes.argtypes = [ctypes.POINTER(ctypes.c_double)]
    lib.orbg_probe_smem_bytes.argtypes = [ctypes.POINTER(ctypes.c_double)]
    lib.orbg_status_string.argtypes = [i32]
    lib.orbg_status_string.restype = ctypes.c_char_p
    lib.orbg_last_cuda_error.argtypes = []
    lib.orbg_pool_trim.argtypes = []
    lib.orbg_version.argtypes = []
    lib.orbg_query_order.argtypes = [i32, u32, i32, vp]
    lib.orbg_query_order.restype = i64
    lib.orbg_query_order_line.argtypes = [i32, u32, i32, i32, i32, vp]
    lib.orbg_query_order_line.restype = i64
    lib.orbg_query_order_model.argtypes = [i32, u32, i32, i32, vp, vp, vp, vp]
    lib.orbg_fit_models.argtypes = [vp, i64, i32, i32, i32, vp, vp]
    lib.orbg_fitted_create.argtypes = [vp, i32, ctypes.POINTER(vp)]
    lib.orbg_fitted_decode.argtypes = [vp, vp, i64, u32, vp, vp, vp, vp, vp]
    lib.orbg_fitted_free.argtypes = [vp]
    lib.orbg_decode_fitted.argtypes = [vp, vp, i64, u32, i32, i32, vp, vp, vp, vp, vp]
    lib.orbg_query_order_model.restype = i64
    lib.orbg_server_create.argtypes = [vp, ctypes.c_size_t, u32, i32, i64, ctypes.POINTER(vp)]
    lib.orbg_server_submit.argtypes = [vp, ctypes.c_uint64, i32, vp, i64]
    lib.orbg_server_poll.argtypes = [vp, vp, i32, i32]
    lib.orbg_server_fetch.argtypes = [vp, ctypes.c_uint64, vp, vp, vp,
                                      ctypes.POINTER(ctypes.c_double)]
    lib.orbg_server_cancel.argtypes = [vp, ctypes.c_uint64]
    lib.orbg_server_stats_get.argtypes = [vp, ctypes.POINTER(OrbgServerStats)]
    lib.orbg_server_destroy.argtypes = [vp]
    lib.orbg_server_replay.argtypes = [vp, i64, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp,
                                       ctypes.POINTER(ctypes.c_double)]
    for f in ("orbg_load_code", "orbg_load_code_line", "orbg_load_code_model",
              "orbg_free_code", "orbg_code_info", "orbg_decode",
              "orbg_codeset_create", "orbg_codeset_free", "orbg_decode_batched",
              "orbg_decode_batched_noalloc", "orbg_server_create", "orbg_server_submit",
              "orbg_server_poll", "orbg_server_fetch", "orbg_server_cancel",
              "orbg_server_stats_get",
              "orbg_server_destroy", "orbg_server_replay",
              "orbg_codeset_set_tuning", "orbg_codeset_get_tuning", "orbg_probe_int_lanes",
              "orbg_probe_smem_bytes", "orbg_codeset_autotune", "orbg_fit_models",
              "orbg_fitted_create", "orbg_fitted_decode", "orbg_fitted_free",
              "orbg_decode_fitted", "orbg_last_cuda_error", "orbg_pool_trim", "orbg_version"):
        getattr(lib, f).restype = i32
    if path == LIB_PATH:
        _lib = lib
    return lib


def _check(rc, what):
    if rc != ORBG_OK:
        raise OrbgError(rc, what)


def _ok(dtype):
    # query counts are below 2^31, so an int32 buffer holds them bit-exactly
    return ("uint32", "int32") if dtype == "uint32" else (dtype,)


def _ptr(a, dtype=None):
    """Address of a torch tensor / NumPy array (None -> NULL)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):  # torch
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        if dtype is not None and str(a.dtype).replace("torch.", "") not in _ok(dtype):
            raise TypeError("expected dtype %s, got %s" % (dtype, a.dtype))
        return a.data_ptr() or None
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        if dtype is not None and str(a.dtype) not in _ok(dtype):
            raise TypeError("expected dtype %s, got %s" % (dtype, a.dtype))
        return a.ctypes.data or None
    if isinstance(a, int):
        return a
    raise TypeError("unsupported buffer type %r" % type(a))


def _stream(s):
    if s is None:
        return None
    if hasattr(s, "cuda_stream"):
        return s.cuda_stream or None
    return int(s) or None


# ------------------------------------------------------------- the C names

def orbg_load_code(mat, kind, n, k, max_query_cap=0):
    lib = load_library()
    m = np.ascontiguousarray(mat, dtype=np.uint8)
    h = ctypes.c_void_p()
    _check(lib.orbg_load_code(m.ctypes.data, int(kind), int(n), int(k),
                              int(max_query_cap), ctypes.byref(h)), "orbg_load_code")
    return h


def orbg_load_code_line(mat, kind, n, k, max_query_cap, J0, beta):
    lib = load_library()
    m = np.ascontiguousarray(mat, dtype=np.uint8)
    h = ctypes.c_void_p()
    _check(lib.orbg_load_code_line(m.ctypes.data, int(kind), int(n), int(k),
                                   int(max_query_cap), int(J0), int(beta), ctypes.byref(h)),
           "orbg_load_code_line")
    return h


def _model_arrays(model):
    """(anchors, J, beta) -> m and int32 arrays (kept alive by the caller)."""
    anchors, J, beta = model
    m = len(J)
    a = np.ascontiguousarray(list(anchors) or [0], dtype=np.int32)
    return (m, a, np.ascontiguousarray(J, dtype=np.int32),
            np.ascontiguousarray(beta, dtype=np.int32))


def orbg_load_code_model(mat, kind, n, k, max_query_cap, model):
    """model: (anchors I_1..I_{m-1}, J_0..J_{m-1}, beta_1..beta_m)."""
    lib = load_library()
    m = np.ascontiguousarray(mat, dtype=np.uint8)
    h = ctypes.c_void_p()
    segs, a, J, beta = _model_arrays(model)
    _check(lib.orbg_load_code_model(m.ctypes.data, int(kind), int(n), int(k),
                                    int(max_query_cap), segs, a.ctypes.data, J.ctypes.data,
                                    beta.ctypes.data, ctypes.byref(h)),
           "orbg_load_code_model")
    return h


def orbg_free_code(code):
    _check(load_library().orbg_free_code(code), "orbg_free_code")


def orbg_code_info(code):
    lib = load_library()
    n = ctypes.c_int()
    k = ctypes.c_int()
    cap = ctypes.c_uint32()
    _check(lib.orbg_code_info(code, ctypes.byref(n), ctypes.byref(k),
                              ctypes.byref(cap), None), "orbg_code_info")
    H = np.zeros((n.value - k.value, n.value), np.uint8)
    _check(lib.orbg_code_info(code, None, None, None, H.ctypes.data), "orbg_code_info")
    return n.value, k.value, cap.value, H


def orbg_decode(code, llr, B, query_cap, codeword, queries, abandoned, cuda_stream=None):
    rc = load_library().orbg_decode(code, _ptr(llr, "float32"), int(B), int(query_cap),
                                    _ptr(codeword, "uint8"), _ptr(queries, "uint32"),
                                    _ptr(abandoned, "uint8"), _stream(cuda_stream))
    _check(rc, "orbg_decode")


def orbg_decode_fitted(code, llr, B, query_cap, lines, divisible, codeword, queries, abandoned,
                       models=None, cuda_stream=None):
    rc = load_library().orbg_decode_fitted(code, _ptr(llr, "float32"), int(B), int(query_cap),
                                           int(lines), int(bool(divisible)),
                                           _ptr(codeword, "uint8"), _ptr(queries, "uint32"),
                                           _ptr(abandoned, "uint8"), _ptr(models, "int32"),
                                           _stream(cuda_stream))
    _check(rc, "orbg_decode_fitted")


def orbg_codeset_create(codes):
    lib = load_library()
    arr = (ctypes.c_void_p * len(codes))(*[c.value if hasattr(c, "value") else c
                                           for c in codes])
    h = ctypes.c_void_p()
    _check(lib.orbg_codeset_create(arr, len(codes), ctypes.byref(h)), "orbg_codeset_create")
    return h


def orbg_codeset_free(cs):
    _check(load_library().orbg_codeset_free(cs), "orbg_codeset_free")


def orbg_decode_batched(cs, code_id, llr_offset, llr, B, query_cap, codeword, cw_offset,
                        queries, abandoned, cuda_stream=None):
    rc = load_library().orbg_decode_batched(
        cs, _ptr(code_id, "int32"), _ptr(llr_offset, "int64"), _ptr(llr, "float32"), int(B),
        int(query_cap), _ptr(codeword, "uint8"), _ptr(cw_offset, "int64"),
        _ptr(queries, "uint32"), _ptr(abandoned, "uint8"), _stream(cuda_stream))
    _check(rc, "orbg_decode_batched")


def orbg_decode_batched_noalloc(cs, code_id, llr_offset, llr, B, query_cap, codeword,
                                cw_offset, queries, abandoned, cuda_stream=None):
    """orbg_decode_batched without any device allocation: its scratch lives
    in a fixed array inside the library.  Device buffers only; at most
    ORBG_NOALLOC_MAX_BLOCKS blocks per call; calls that overlap on the GPU
    race on the shared array."""
    rc = load_library().orbg_decode_batched_noalloc(
        cs, _ptr(code_id, "int32"), _ptr(llr_offset, "int64"), _ptr(llr, "float32"), int(B),
        int(query_cap), _ptr(codeword, "uint8"), _ptr(cw_offset, "int64"),
        _ptr(queries, "uint32"), _ptr(abandoned, "uint8"), _stream(cuda_stream))
    _check(rc, "orbg_decode_batched_noalloc")


def orbg_server_create(cs, mem_budget_bytes, query_cap, streams=0, max_batch_blocks=0):
    h = ctypes.c_void_p()
    _check(load_library().orbg_server_create(cs, int(mem_budget_bytes), int(query_cap),
                                             int(streams), int(max_batch_blocks),
                                             ctypes.byref(h)), "orbg_server_create")
    return h


def orbg_server_submit(srv, request_id, code_index, llr, B):
    _check(load_library().orbg_server_submit(srv, int(request_id), int(code_index),
                                             _ptr(llr, "float32"), int(B)),
           "orbg_server_submit")


def orbg_server_poll(srv, max_ids=1024, timeout_us=1000):
    ids = np.zeros(max_ids, np.uint64)
    k = load_library().orbg_server_poll(srv, ids.ctypes.data, int(max_ids), int(timeout_us))
    if k < 0:
        raise OrbgError(k, "orbg_server_poll")
    return [int(x) for x in ids[:k]]


def orbg_server_fetch(srv, request_id, codeword=None, queries=None, abandoned=None):
    lat = ctypes.c_double()
    _check(load_library().orbg_server_fetch(srv, int(request_id), _ptr(codeword, "uint8"),
                                            _ptr(queries, "uint32"), _ptr(abandoned, "uint8"),
                                            ctypes.byref(lat)), "orbg_server_fetch")
    return lat.value


def orbg_server_cancel(srv, request_id):
    _check(load_library().orbg_server_cancel(srv, int(request_id)), "orbg_server_cancel")


def orbg_server_stats_get(srv):
    st = OrbgServerStats()
    _check(load_library().orbg_server_stats_get(srv, ctypes.byref(st)), "orbg_server_stats_get")
    return st.as_dict()


def orbg_server_destroy(srv):
    _check(load_library().orbg_server_destroy(srv), "orbg_server_destroy")


def orbg_server_replay(srv, arrival_s, code, B, llr_off, blk_off, llr_all, cw_all, q_all,
                       ab_all, latency_s):
    wall = ctypes.c_double()
    _check(load_library().orbg_server_replay(
        srv, int(len(arrival_s)), _ptr(arrival_s, "float64"), _ptr(code, "int32"),
        _ptr(B, "int64"), _ptr(llr_off, "int64"), _ptr(blk_off, "int64"),
        _ptr(llr_all, "float32"), _ptr(cw_all, "uint8"), _ptr(q_all, "uint32"),
        _ptr(ab_all, "uint8"), _ptr(latency_s, "float64"), ctypes.byref(wall)),
        "orbg_server_replay")
    return wall.value


def orbg_codeset_set_tuning(cs, tuning=None):
    """tuning: OrbgTuning, a dict of its fields, or None for the defaults."""
    t = None
    if tuning is not None:
        if isinstance(tuning, dict):
            tuning = OrbgTuning(**tuning)
        t = ctypes.byref(tuning)
    _check(load_library().orbg_codeset_set_tuning(cs, t), "orbg_codeset_set_tuning")


def orbg_codeset_autotune(cs, code_id, llr_offset, llr, B, query_cap, codeword, cw_offset,
                          queries, abandoned, reps=3, cuda_stream=None):
    """Coordinate-descent autotuner of the batched form on a device sample;
    sets the fastest tuning on the code set and returns it."""
    t = OrbgTuning()
    rc = load_library().orbg_codeset_autotune(
        cs, _ptr(code_id, "int32"), _ptr(llr_offset, "int64"), _ptr(llr, "float32"), int(B),
        int(query_cap), _ptr(codeword, "uint8"), _ptr(cw_offset, "int64"),
        _ptr(queries, "uint32"), _ptr(abandoned, "uint8"), int(reps), _stream(cuda_stream),
        ctypes.byref(t))
    _check(rc, "orbg_codeset_autotune")
    return t


def orbg_codeset_get_tuning(cs):
    t = OrbgTuning()
    _check(load_library().orbg_codeset_get_tuning(cs, ctypes.byref(t)),
           "orbg_codeset_get_tuning")
    return t


def orbg_probe_int_lanes():
    """lop3.b32 lanes retired per SM per clock on the current device."""
    x = ctypes.c_double()
    _check(load_library().orbg_probe_int_lanes(ctypes.byref(x)), "orbg_probe_int_lanes")
    return x.value


def orbg_probe_smem_bytes():
    """Shared-memory bytes per SM per clock (64-bit loads, no conflicts)."""
    x = ctypes.c_double(0)
    _check(load_library().orbg_probe_smem_bytes(ctypes.byref(x)), "orbg_probe_smem_bytes")
    return x.value


def orbg_status_string(status):
    return load_library().orbg_status_string(int(status)).decode()


def orbg_last_cuda_error():
    return load_library().orbg_last_cuda_error()


def orbg_pool_trim():
    """Return the device memory the library's pool holds unused."""
    _check(load_library().orbg_pool_trim(), "orbg_pool_trim")


def orbg_version():
    return load_library().orbg_version()


def orbg_query_order(n, count, table=0):
    """First `count` patterns of the decoder's query order for length n, as
    tuples of 1-based sorted-order positions, from table 0 (warp) or 1
    (CTA)."""
    lib = load_library()
    out = np.zeros((count, n + 1), np.int32)
    got = lib.orbg_query_order(int(n), int(count), int(table), out.ctypes.data)
    if got < 0:
        raise OrbgError(int(got), "orbg_query_order")
    return [tuple(int(x) for x in row[1:1 + row[0]]) for row in out[:got]]


def orbg_query_order_line(n, count, table, J0, beta):
    """orbg_query_order for the one-line order of reliability weight
    J0 w_H + beta w_L."""
    lib = load_library()
    out = np.zeros((count, n + 1), np.int32)
    got = lib.orbg_query_order_line(int(n), int(count), int(table), int(J0), int(beta),
                                    out.ctypes.data)
    if got < 0:
        raise OrbgError(int(got), "orbg_query_order_line")
    return [tuple(int(x) for x in row[1:1 + row[0]]) for row in out[:got]]


def orbg_query_order_model(n, count, table, model):
    """orbg_query_order for the m-segment order of model (anchors, J, beta)."""
    lib = load_library()
    out = np.zeros((count, n + 1), np.int32)
    segs, a, J, beta = _model_arrays(model)
    got = lib.orbg_query_order_model(int(n), int(count), int(table), segs, a.ctypes.data,
                                     J.ctypes.data, beta.ctypes.data, out.ctypes.data)
    if got < 0:
        raise OrbgError(int(got), "orbg_query_order_model")
    return [tuple(int(x) for x in row[1:1 + row[0]]) for row in out[:got]]



def _out(shape, dtype, device):
    """An output tensor for a decode helper: torch.empty, or, when the
    environment sets ORBG_POISON_OUTPUTS=1 (the test suite does), filled
    with all-ones bits (codeword byte 255, q 2^32 - 1, flag 255), which no
    decode writes, so an output a call leaves unwritten cannot pass for a
    result left in recycled memory by an earlier call."""
    import torch
    t = torch.empty(shape, dtype=dtype, device=device)
    if os.environ.get("ORBG_POISON_OUTPUTS") == "1":
        t.fill_(-1 if dtype == torch.int32 else 0xFF)
    return t

def fit_models(llr, n, lines, divisible=False, stream=None):
    """orbg_fit_models on a device tensor of B x n FP32 LLRs: the int32
    [B, ORBG_FIT_STRIDE] model records (Sec. III-E), stream-ordered."""
    import torch
    lib = load_library()
    B = llr.numel() // n
    out = _out((B, ORBG_FIT_STRIDE), torch.int32, llr.device)
    st = _stream(stream if stream is not None else torch.cuda.current_stream(llr.device))
    _check(lib.orbg_fit_models(llr.data_ptr(), B, int(n), int(lines), int(bool(divisible)),
                               out.data_ptr(), st), "orbg_fit_models")
    return out


class Fitted:
    """Owning wrapper of an orbg_fitted object: one-line full ORBGRAND with
    each block's own fitted line (Sec. III-E)."""

    def __init__(self, code, divisible=False):
        lib = load_library()
        self.code = code  # the handle must outlive the object
        h = ctypes.c_void_p()
        _check(lib.orbg_fitted_create(code.handle, int(bool(divisible)), ctypes.byref(h)),
               "orbg_fitted_create")
        self.handle = h

    def decode(self, llr, query_cap, stream=None):
        """llr: CUDA tensor [B][n].  Returns (codeword u8, queries int32,
        abandoned u8, model records int32 [B][ORBG_FIT_STRIDE])."""
        import torch
        lib = load_library()
        n = self.code.n
        B = llr.numel() // n
        dev = llr.device
        cw = _out((B, n), torch.uint8, dev)
        q = _out((B,), torch.int32, dev)
        ab = _out((B,), torch.uint8, dev)
        rec = _out((B, ORBG_FIT_STRIDE), torch.int32, dev)
        st = _stream(stream if stream is not None else torch.cuda.current_stream(dev))
        _check(lib.orbg_fitted_decode(self.handle, llr.data_ptr(), B, int(query_cap),
                                      cw.data_ptr(), q.data_ptr(), ab.data_ptr(),
                                      rec.data_ptr(), st), "orbg_fitted_decode")
        return cw, q, ab, rec

    def close(self):
        if self.handle is not None and self.handle.value:
            load_library().orbg_fitted_free(self.handle)
        self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def model_of_record(rec):
    """(anchors, J, beta) of one model record; None for a NaN block (m = 0)."""
    rec = [int(x) for x in rec]
    m = rec[0]
    if m == 0:
        return None
    return tuple(rec[1:m]), tuple(rec[8:8 + m]), tuple(rec[16:16 + m])


# ------------------------------------------------------- convenience layer

class Code:
    """Owning wrapper of an orbg_code handle."""

    def __init__(self, mat, kind=ORBG_MAT_H, n=None, k=None, max_query_cap=0, line=None,
                 model=None):
        """line: (J0, beta) for one-line full ORBGRAND; model: (anchors, J,
        beta) for m-segment full ORBGRAND; neither for basic."""
        mat = np.asarray(mat, dtype=np.uint8)
        n = mat.shape[1] if n is None else n
        if k is None:
            k = n - mat.shape[0] if kind == ORBG_MAT_H else mat.shape[0]
        self.n, self.k = int(n), int(k)
        if line is not None and model is not None:
            raise ValueError("give a line or a model, not both")
        if model is not None:
            self.handle = orbg_load_code_model(mat, kind, n, k, max_query_cap, model)
        elif line is not None:
            self.handle = orbg_load_code_line(mat, kind, n, k, max_query_cap, *line)
        else:
            self.handle = orbg_load_code(mat, kind, n, k, max_query_cap)

    def close(self):
        if self.handle is not None and self.handle.value:
            orbg_free_code(self.handle)
        self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class CodeSet:
    def __init__(self, codes):
        self.codes = list(codes)
        self.handle = orbg_codeset_create([c.handle for c in self.codes])

    def close(self):
        if self.handle is not None and self.handle.value:
            orbg_codeset_free(self.handle)
        self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def decode(code, llr, query_cap, stream=None):
    """Plain form on a torch tensor llr[B][n] (CUDA): returns (codeword u8,
    queries int32, abandoned u8) tensors on the same device."""
    import torch
    B = llr.shape[0]
    cw = _out((B, code.n), torch.uint8, llr.device)
    q = _out((B,), torch.int32, llr.device)
    ab = _out((B,), torch.uint8, llr.device)
    orbg_decode(code.handle, llr, B, query_cap, cw, q, ab,
                stream if stream is not None else torch.cuda.current_stream(llr.device))
    return cw, q, ab


def decode_fitted(code, llr, query_cap, lines, divisible=False, stream=None):
    """Full ORBGRAND with a `lines`-line model fitted to each block (Sec.
    III-E), each block searched in its own order (Sec. III-D), on a torch
    tensor llr[B][n] (CUDA): returns (codeword u8, queries int32, abandoned
    u8, model records int32 [B][ORBG_FIT_STRIDE])."""
    import torch
    B = llr.shape[0]
    dev = llr.device
    cw = _out((B, code.n), torch.uint8, dev)
    q = _out((B,), torch.int32, dev)
    ab = _out((B,), torch.uint8, dev)
    rec = _out((B, ORBG_FIT_STRIDE), torch.int32, dev)
    orbg_decode_fitted(code.handle, llr, B, query_cap, lines, divisible, cw, q, ab, rec,
                       stream if stream is not None else torch.cuda.current_stream(dev))
    return cw, q, ab, rec


def decode_batched(codeset, llr, query_cap, code_id=None, llr_offset=None,
                   cw_offset=None, n_total=None, stream=None):
    """Batched persistent form.  Dense single-code layout when the offsets
    are None; otherwise n_total is the codeword buffer length."""
    import torch
    dev = llr.device
    if llr_offset is None:
        n = codeset.codes[0].n
        B = llr.numel() // n
        cw = _out((B, n), torch.uint8, dev)
    else:
        B = llr_offset.shape[0]
        cw = _out((n_total,), torch.uint8, dev)
    q = _out((B,), torch.int32, dev)
    ab = _out((B,), torch.uint8, dev)
    orbg_decode_batched(codeset.handle, code_id, llr_offset, llr, B, query_cap, cw,
                        cw_offset, q, ab,
                        stream if stream is not None else torch.cuda.current_stream(dev))
    return cw, q, ab
