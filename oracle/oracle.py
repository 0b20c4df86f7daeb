"""ctypes wrapper around oracle/orbg_oracle.c (test infrastructure only).

The C file is compiled on first use (plain gcc, no CUDA) into
oracle/liborbg_oracle.so; ``build_oracle()`` forces a rebuild.  ``Oracle``
can also wrap another build of the same source (the mutation tests compile
deliberately broken copies of it to check that the pins catch them).
"""
import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
ORACLE_SRC = os.path.join(_HERE, "orbg_oracle.c")
ORACLE_LIB = os.path.join(_HERE, "liborbg_oracle.so")
_lock = threading.Lock()


def compile_oracle(src, out):
    """gcc -O2, no fast-math (fabsf and the compares stay IEEE)."""
    tmp = out + ".%d.tmp" % os.getpid()
    subprocess.check_call(["gcc", "-O2", "-std=c99", "-fPIC", "-shared",
                           "-o", tmp, src, "-lm"])
    os.replace(tmp, out)
    return out


def build_oracle(force=False):
    with _lock:
        stale = (not os.path.exists(ORACLE_LIB)
                 or os.path.getmtime(ORACLE_LIB) < os.path.getmtime(ORACLE_SRC))
        if force or stale:
            compile_oracle(ORACLE_SRC, ORACLE_LIB)
    return ORACLE_LIB


class OracleError(RuntimeError):
    pass


def _ptr(a, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


class Oracle:
    def __init__(self, path):
        lib = ctypes.CDLL(path)
        u8p = ctypes.POINTER(ctypes.c_uint8)
        i32p = ctypes.POINTER(ctypes.c_int)
        i64p = ctypes.POINTER(ctypes.c_long)
        u64p = ctypes.POINTER(ctypes.c_uint64)
        f32p = ctypes.POINTER(ctypes.c_float)
        lib.orbg_oracle_decode.argtypes = [u8p, ctypes.c_int, ctypes.c_int,
                                           f32p, ctypes.c_uint64, u8p, u64p,
                                           i32p, u64p, i32p, i32p]
        lib.orbg_oracle_decode.restype = ctypes.c_int
        lib.orbg_oracle_decode_batch.argtypes = [u8p, ctypes.c_int,
                                                 ctypes.c_int, f32p,
                                                 ctypes.c_long,
                                                 ctypes.c_uint64, u8p, u64p,
                                                 u8p, u64p]
        lib.orbg_oracle_decode_batch.restype = ctypes.c_int
        lib.orbg_oracle_enumerate.argtypes = [ctypes.c_int, ctypes.c_long,
                                              i32p]
        lib.orbg_oracle_enumerate.restype = ctypes.c_long
        lib.orbg_oracle_landslide.argtypes = [ctypes.c_int, ctypes.c_int,
                                              ctypes.c_int, ctypes.c_long,
                                              i32p]
        lib.orbg_oracle_landslide.restype = ctypes.c_long
        lib.orbg_oracle_sort.argtypes = [f32p, ctypes.c_int, i32p]
        lib.orbg_oracle_sort.restype = ctypes.c_int
        lib.orbg_oracle_count_by_weight.argtypes = [ctypes.c_int,
                                                    ctypes.c_int, i64p]
        lib.orbg_oracle_count_by_weight.restype = ctypes.c_int
        lib.orbg_oracle_enumerate_1line.argtypes = [ctypes.c_int, ctypes.c_long,
                                                    ctypes.c_long, ctypes.c_long, i32p]
        lib.orbg_oracle_enumerate_1line.restype = ctypes.c_long
        lib.orbg_oracle_decode_1line.argtypes = [u8p, ctypes.c_int, ctypes.c_int, f32p,
                                                 ctypes.c_uint64, ctypes.c_long,
                                                 ctypes.c_long, u8p, u64p, i32p, u64p,
                                                 i32p, i32p]
        lib.orbg_oracle_decode_1line.restype = ctypes.c_int
        lib.orbg_oracle_decode_batch_1line.argtypes = [u8p, ctypes.c_int, ctypes.c_int,
                                                       f32p, ctypes.c_long, ctypes.c_uint64,
                                                       ctypes.c_long, ctypes.c_long, u8p,
                                                       u64p, u8p, u64p]
        lib.orbg_oracle_decode_batch_1line.restype = ctypes.c_int
        lib.orbg_oracle_enumerate_mline.argtypes = [ctypes.c_int, ctypes.c_int, i32p, i64p,
                                                    i64p, ctypes.c_long, i32p]
        lib.orbg_oracle_enumerate_mline.restype = ctypes.c_long
        lib.orbg_oracle_decode_batch_mline.argtypes = [u8p, ctypes.c_int, ctypes.c_int, f32p,
                                                       ctypes.c_long, ctypes.c_uint64,
                                                       ctypes.c_int, i32p, i64p, i64p, u8p,
                                                       u64p, u8p, u64p]
        lib.orbg_oracle_decode_batch_mline.restype = ctypes.c_int
        lib.orbg_oracle_fit.argtypes = [f32p, ctypes.c_int, ctypes.c_int, ctypes.c_int, i32p,
                                        i32p, i64p, i64p]
        lib.orbg_oracle_fit.restype = ctypes.c_int
        lib.orbg_oracle_decode_batch_fit.argtypes = [u8p, ctypes.c_int, ctypes.c_int, f32p,
                                                     ctypes.c_long, ctypes.c_uint64,
                                                     ctypes.c_int, ctypes.c_int, u8p, u64p,
                                                     u8p, u64p]
        lib.orbg_oracle_decode_batch_fit.restype = ctypes.c_int
        self.lib = lib
        self.path = path

    def decode(self, H, llr, cap):
        """Decode one block.  Returns (codeword uint8[n], queries, abandoned,
        sum_w, hit) where hit lists the 1-based sorted-order positions v of
        the winning pattern (None if abandoned)."""
        H = np.ascontiguousarray(H, dtype=np.uint8)
        r, n = H.shape
        llr = np.ascontiguousarray(llr, dtype=np.float32)
        assert llr.shape == (n,)
        c = np.zeros(n, np.uint8)
        q = ctypes.c_uint64(0)
        ab = ctypes.c_int(0)
        sw = ctypes.c_uint64(0)
        hw = ctypes.c_int(0)
        hv = np.zeros(n, np.int32)
        rc = self.lib.orbg_oracle_decode(
            _ptr(H, ctypes.c_uint8), n, r, _ptr(llr, ctypes.c_float),
            int(cap), _ptr(c, ctypes.c_uint8), ctypes.byref(q),
            ctypes.byref(ab), ctypes.byref(sw), ctypes.byref(hw),
            _ptr(hv, ctypes.c_int))
        if rc != 0:
            raise OracleError("oracle decode failed: %d" % rc)
        hit = None if hw.value < 0 else [int(x) for x in hv[:hw.value]]
        return c, int(q.value), int(ab.value), int(sw.value), hit

    def decode_batch(self, H, llr, cap):
        """Decode blocks llr[B][n].  Returns (codeword[B][n] uint8,
        queries[B] uint64, abandoned[B] uint8, sum_w[B] uint64)."""
        H = np.ascontiguousarray(H, dtype=np.uint8)
        r, n = H.shape
        llr = np.ascontiguousarray(llr, dtype=np.float32).reshape(-1, n)
        B = llr.shape[0]
        c = np.zeros((B, n), np.uint8)
        q = np.zeros(B, np.uint64)
        ab = np.zeros(B, np.uint8)
        sw = np.zeros(B, np.uint64)
        rc = self.lib.orbg_oracle_decode_batch(
            _ptr(H, ctypes.c_uint8), n, r, _ptr(llr, ctypes.c_float), B,
            int(cap), _ptr(c, ctypes.c_uint8), _ptr(q, ctypes.c_uint64),
            _ptr(ab, ctypes.c_uint8), _ptr(sw, ctypes.c_uint64))
        if rc != 0:
            raise OracleError("oracle batch decode failed: %d" % rc)
        return c, q, ab, sw

    def decode_1line(self, H, llr, cap, J0, beta):
        """decode() for one-line full ORBGRAND (Sec. III-D): queries in
        increasing J0 w_H + beta w_L."""
        H = np.ascontiguousarray(H, dtype=np.uint8)
        r, n = H.shape
        llr = np.ascontiguousarray(llr, dtype=np.float32)
        assert llr.shape == (n,)
        c = np.zeros(n, np.uint8)
        q = ctypes.c_uint64(0)
        ab = ctypes.c_int(0)
        sw = ctypes.c_uint64(0)
        hw = ctypes.c_int(0)
        hv = np.zeros(n, np.int32)
        rc = self.lib.orbg_oracle_decode_1line(
            _ptr(H, ctypes.c_uint8), n, r, _ptr(llr, ctypes.c_float), int(cap), int(J0),
            int(beta), _ptr(c, ctypes.c_uint8), ctypes.byref(q), ctypes.byref(ab),
            ctypes.byref(sw), ctypes.byref(hw), _ptr(hv, ctypes.c_int))
        if rc != 0:
            raise OracleError("oracle 1-line decode failed: %d" % rc)
        hit = None if hw.value < 0 else [int(x) for x in hv[:hw.value]]
        return c, int(q.value), int(ab.value), int(sw.value), hit

    def decode_batch_1line(self, H, llr, cap, J0, beta):
        """decode_batch() for one-line full ORBGRAND."""
        H = np.ascontiguousarray(H, dtype=np.uint8)
        r, n = H.shape
        llr = np.ascontiguousarray(llr, dtype=np.float32).reshape(-1, n)
        B = llr.shape[0]
        c = np.zeros((B, n), np.uint8)
        q = np.zeros(B, np.uint64)
        ab = np.zeros(B, np.uint8)
        sw = np.zeros(B, np.uint64)
        rc = self.lib.orbg_oracle_decode_batch_1line(
            _ptr(H, ctypes.c_uint8), n, r, _ptr(llr, ctypes.c_float), B, int(cap), int(J0),
            int(beta), _ptr(c, ctypes.c_uint8), _ptr(q, ctypes.c_uint64),
            _ptr(ab, ctypes.c_uint8), _ptr(sw, ctypes.c_uint64))
        if rc != 0:
            raise OracleError("oracle 1-line batch decode failed: %d" % rc)
        return c, q, ab, sw

    def enumerate_patterns_1line(self, n, count, J0, beta):
        """First `count` patterns of the one-line order (increasing
        J0 w_H + beta w_L), as tuples of 1-based sorted-order positions."""
        out = np.zeros((count, n + 1), np.int32)
        got = self.lib.orbg_oracle_enumerate_1line(n, int(J0), int(beta), count,
                                                   _ptr(out, ctypes.c_int))
        if got < 0:
            raise OracleError("enumerate failed: %d" % got)
        return [tuple(int(x) for x in row[1:1 + row[0]]) for row in out[:got]]

    @staticmethod
    def _model(model):
        """(anchors I_1..I_{m-1}, J_0..J_{m-1}, beta_1..beta_m) as C arrays."""
        anchors, J, beta = model
        m = len(J)
        assert len(beta) == m and len(anchors) == m - 1
        a = np.array(list(anchors) + [0], np.int32)
        return m, a, np.array(J, np.int64), np.array(beta, np.int64)

    def enumerate_patterns_mline(self, n, count, model):
        """First `count` patterns of the m-segment order (Sec. III-D), as
        tuples of 1-based sorted-order positions.  model = (anchors, J, beta)."""
        m, a, J, beta = self._model(model)
        out = np.zeros((count, n + 1), np.int32)
        got = self.lib.orbg_oracle_enumerate_mline(
            n, m, _ptr(a, ctypes.c_int), J.ctypes.data_as(ctypes.POINTER(ctypes.c_long)),
            beta.ctypes.data_as(ctypes.POINTER(ctypes.c_long)), count, _ptr(out, ctypes.c_int))
        if got < 0:
            raise OracleError("enumerate failed: %d" % got)
        return [tuple(int(x) for x in row[1:1 + row[0]]) for row in out[:got]]

    def decode_batch_mline(self, H, llr, cap, model):
        """decode_batch() for m-segment full ORBGRAND."""
        m, a, J, beta = self._model(model)
        H = np.ascontiguousarray(H, dtype=np.uint8)
        r, n = H.shape
        llr = np.ascontiguousarray(llr, dtype=np.float32).reshape(-1, n)
        B = llr.shape[0]
        c = np.zeros((B, n), np.uint8)
        q = np.zeros(B, np.uint64)
        ab = np.zeros(B, np.uint8)
        sw = np.zeros(B, np.uint64)
        rc = self.lib.orbg_oracle_decode_batch_mline(
            _ptr(H, ctypes.c_uint8), n, r, _ptr(llr, ctypes.c_float), B, int(cap), m,
            _ptr(a, ctypes.c_int), J.ctypes.data_as(ctypes.POINTER(ctypes.c_long)),
            beta.ctypes.data_as(ctypes.POINTER(ctypes.c_long)), _ptr(c, ctypes.c_uint8),
            _ptr(q, ctypes.c_uint64), _ptr(ab, ctypes.c_uint8), _ptr(sw, ctypes.c_uint64))
        if rc != 0:
            raise OracleError("oracle m-line batch decode failed: %d" % rc)
        return c, q, ab, sw

    def fit(self, llr, lines, divisible=False):
        """Piece-wise linear fit and quantisation of one block's ordered
        reliabilities (Sec. III-E): the model (anchors, J, beta)."""
        llr = np.ascontiguousarray(llr, dtype=np.float32)
        m = ctypes.c_int(0)
        a = np.zeros(8, np.int32)
        J = np.zeros(8, np.int64)
        beta = np.zeros(8, np.int64)
        rc = self.lib.orbg_oracle_fit(_ptr(llr, ctypes.c_float), llr.shape[0], int(lines),
                                      int(bool(divisible)), ctypes.byref(m),
                                      _ptr(a, ctypes.c_int),
                                      J.ctypes.data_as(ctypes.POINTER(ctypes.c_long)),
                                      beta.ctypes.data_as(ctypes.POINTER(ctypes.c_long)))
        if rc != 0:
            raise OracleError("fit failed: %d" % rc)
        k = m.value
        return (tuple(int(x) for x in a[:k - 1]), tuple(int(x) for x in J[:k]),
                tuple(int(x) for x in beta[:k]))

    def decode_batch_fit(self, H, llr, cap, lines, divisible=False):
        """decode_batch() for full ORBGRAND with each block's own fitted
        model (fit(), then the m-segment order)."""
        H = np.ascontiguousarray(H, dtype=np.uint8)
        r, n = H.shape
        llr = np.ascontiguousarray(llr, dtype=np.float32).reshape(-1, n)
        B = llr.shape[0]
        c = np.zeros((B, n), np.uint8)
        q = np.zeros(B, np.uint64)
        ab = np.zeros(B, np.uint8)
        sw = np.zeros(B, np.uint64)
        rc = self.lib.orbg_oracle_decode_batch_fit(
            _ptr(H, ctypes.c_uint8), n, r, _ptr(llr, ctypes.c_float), B, int(cap), int(lines),
            int(bool(divisible)), _ptr(c, ctypes.c_uint8), _ptr(q, ctypes.c_uint64),
            _ptr(ab, ctypes.c_uint8), _ptr(sw, ctypes.c_uint64))
        if rc != 0:
            raise OracleError("oracle fitted batch decode failed: %d" % rc)
        return c, q, ab, sw

    def enumerate_patterns(self, n, count):
        """First `count` patterns of the query order for length n, as tuples
        of 1-based sorted-order positions (the zero pattern is ())."""
        out = np.zeros((count, n + 1), np.int32)
        got = self.lib.orbg_oracle_enumerate(n, count, _ptr(out, ctypes.c_int))
        if got < 0:
            raise OracleError("enumerate failed: %d" % got)
        return [tuple(int(x) for x in row[1:1 + row[0]]) for row in out[:got]]

    def landslide(self, Wp, w, np_, cap=1 << 16):
        """Algorithm 2 output for (W', w, n') as tuples u_1..u_w."""
        out = np.zeros((cap, w), np.int32)
        got = self.lib.orbg_oracle_landslide(Wp, w, np_, cap,
                                             _ptr(out, ctypes.c_int))
        if got < 0:
            raise OracleError("landslide failed: %d" % got)
        return [tuple(int(x) for x in row) for row in out[:got]]

    def sort_reliability(self, llr):
        llr = np.ascontiguousarray(llr, dtype=np.float32)
        pi = np.zeros(llr.shape[0], np.int32)
        rc = self.lib.orbg_oracle_sort(_ptr(llr, ctypes.c_float),
                                       llr.shape[0], _ptr(pi, ctypes.c_int))
        if rc != 0:
            raise OracleError("sort failed: %d" % rc)
        return pi

    def count_by_weight(self, n, Wmax):
        """counts[W][w]: patterns of logistic weight W and Hamming weight w
        met by the query order, W <= Wmax."""
        out = np.zeros((Wmax + 1, n + 1), np.int64)
        rc = self.lib.orbg_oracle_count_by_weight(
            n, Wmax, out.ctypes.data_as(ctypes.POINTER(ctypes.c_long)))
        if rc != 0:
            raise OracleError("count failed: %d" % rc)
        return out


_default = None


def default():
    global _default
    if _default is None:
        _default = Oracle(build_oracle())
    return _default


def decode(H, llr, cap):
    return default().decode(H, llr, cap)


def decode_batch(H, llr, cap):
    return default().decode_batch(H, llr, cap)


def enumerate_patterns(n, count):
    return default().enumerate_patterns(n, count)


def landslide(Wp, w, np_, cap=1 << 16):
    return default().landslide(Wp, w, np_, cap)


def sort_reliability(llr):
    return default().sort_reliability(llr)


def count_by_weight(n, Wmax):
    return default().count_by_weight(n, Wmax)


def decode_1line(H, llr, cap, J0, beta):
    return default().decode_1line(H, llr, cap, J0, beta)


def decode_batch_1line(H, llr, cap, J0, beta):
    return default().decode_batch_1line(H, llr, cap, J0, beta)


def enumerate_patterns_1line(n, count, J0, beta):
    return default().enumerate_patterns_1line(n, count, J0, beta)


def enumerate_patterns_mline(n, count, model):
    return default().enumerate_patterns_mline(n, count, model)


def decode_batch_mline(H, llr, cap, model):
    return default().decode_batch_mline(H, llr, cap, model)


def fit(llr, lines, divisible=False):
    return default().fit(llr, lines, divisible)


def decode_batch_fit(H, llr, cap, lines, divisible=False):
    return default().decode_batch_fit(H, llr, cap, lines, divisible)
