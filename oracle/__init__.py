"""CPU oracle for the ABFT-protected GEMM (FT-BLAS, Zhai et al., ICS '21, Sections II.A and V).

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's CPU-baseline
leg and reference arm may import this package; the library itself never does. Parity
unpinned: the ACC32 model's values against the hardware beyond the stated bound (named
in the C source's header). The C source next to this
file (``ftgemm_oracle.c``) is plain binary64 code compiled with ``-ffp-contract=off``; it
shares no code with the CUDA path. Buffers are flat numpy float64 arrays in BLAS storage
with explicit leading dimensions, exactly as the C ABI takes them.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

ROW_MAJOR, COL_MAJOR = 101, 102
NO_TRANS, TRANS = 111, 112
SITE_ACCUM, SITE_OUTPUT, SITE_CHECKSUM = 1, 2, 3
MODE_BITFLIP, MODE_ADD_REL = 0, 1
KIND_CORRECTED, KIND_CHECKSUM_ONLY, KIND_UNCORRECTABLE, KIND_INPUT_NONFINITE = 1, 2, 3, 4
PREC_FP64, PREC_ACC32, PREC_ACC32_E4M3 = 0, 1, 2
U_ACC32 = 2.0 ** -23
MAX_RECORDS = 256

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ftgemm_oracle.c")
_SRCS = (_SRC, os.path.join(_HERE, "emu_oracle.c"))
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


class Problem(C.Structure):
    _fields_ = [
        ("layout", C.c_int32), ("transa", C.c_int32), ("transb", C.c_int32), ("pad_", C.c_int32),
        ("M", C.c_int64), ("N", C.c_int64), ("K", C.c_int64),
        ("alpha", C.c_double),
        ("A", C.c_void_p), ("lda", C.c_int64),
        ("B", C.c_void_p), ("ldb", C.c_int64),
        ("beta", C.c_double),
        ("Cin", C.c_void_p), ("ldc", C.c_int64),
        ("tile_m", C.c_int64), ("tile_n", C.c_int64),
        ("bk", C.c_int64),
        ("precision", C.c_int32), ("pad2_", C.c_int32),
        ("u_acc", C.c_double),
        ("kc", C.c_int64),
    ]


class EmuProblem(C.Structure):
    _fields_ = [
        ("layout", C.c_int32), ("transa", C.c_int32), ("transb", C.c_int32), ("slices", C.c_int32),
        ("M", C.c_int64), ("N", C.c_int64), ("K", C.c_int64),
        ("alpha", C.c_double),
        ("A", C.c_void_p), ("lda", C.c_int64),
        ("B", C.c_void_p), ("ldb", C.c_int64),
        ("beta", C.c_double),
        ("Cin", C.c_void_p), ("ldc", C.c_int64),
        ("tile_m", C.c_int64), ("tile_n", C.c_int64),
    ]


class Injection(C.Structure):
    _fields_ = [
        ("i", C.c_int64), ("j", C.c_int64),
        ("site", C.c_int32), ("mode", C.c_int32), ("bit", C.c_int32),
        ("rel_log2", C.c_int32), ("sign", C.c_int32), ("kt", C.c_int32),
    ]


class Record(C.Structure):
    _fields_ = [
        ("tile_row", C.c_int64), ("tile_col", C.c_int64), ("i", C.c_int64), ("j", C.c_int64),
        ("delta_row", C.c_double), ("delta_col", C.c_double),
        ("tau_row", C.c_double), ("tau_col", C.c_double),
        ("value_before", C.c_double), ("value_after", C.c_double), ("value_subtracted", C.c_double),
        ("kind", C.c_int32), ("rows_flagged", C.c_int32), ("cols_flagged", C.c_int32), ("pad_", C.c_int32),
    ]


class Report(C.Structure):
    _fields_ = [
        ("tiles_checked", C.c_uint64), ("detected", C.c_uint64), ("corrected", C.c_uint64),
        ("uncorrectable", C.c_uint64), ("checksum_only", C.c_uint64), ("input_nonfinite", C.c_uint64),
        ("n_records", C.c_uint32), ("pad_", C.c_uint32),
        ("rec", Record * MAX_RECORDS),
    ]

    def records(self):
        return [self.rec[q] for q in range(min(self.n_records, MAX_RECORDS))]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C, -ffp-contract=off). Returns the library path."""
    with _lock:
        if not force and os.path.exists(_LIB_PATH) and all(os.path.getmtime(_LIB_PATH) >= os.path.getmtime(x)
                                                           for x in _SRCS):
            return _LIB_PATH
        os.makedirs(_BUILD, exist_ok=True)
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math",
               "-fopenmp", "-Wall", "-o", tmp, *_SRCS, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
        return _LIB_PATH


def lib():
    global _lib
    if _lib is None:
        # ORACLE_LIB points the tests at a deliberately broken build (mutation tests).
        path = os.environ.get("ORACLE_LIB") or build()
        L = C.CDLL(path)
        L.oracle_gemm.argtypes = [C.POINTER(Problem), C.c_void_p]
        L.oracle_gemm.restype = C.c_int
        L.oracle_gemm_rows.argtypes = [C.POINTER(Problem), C.c_int64, C.c_void_p, C.c_void_p]
        L.oracle_gemm_rows.restype = C.c_int
        L.oracle_ft_gemm.argtypes = [C.POINTER(Problem), C.c_int64, C.c_void_p, C.c_int64, C.c_void_p,
                                     C.c_void_p, C.POINTER(Report)]
        L.oracle_ft_gemm.restype = C.c_int
        L.oracle_draw_injections.argtypes = [C.c_uint64, C.c_uint64, C.c_int32, C.c_int32, C.c_int32, C.c_int32,
                                             C.c_int32, C.c_int32, C.c_int32, C.c_int32,
                                             C.c_int64, C.c_int64, C.c_int64, C.c_int64, C.c_int64, C.c_void_p]
        L.oracle_draw_injections.restype = C.c_int64
        L.oracle_trsm_left.argtypes = [C.c_int64, C.c_int64, C.c_void_p, C.c_int64, C.c_int, C.c_void_p, C.c_int64]
        L.oracle_trsm_left.restype = None
        L.oracle_emu_gemm.argtypes = [C.POINTER(EmuProblem), C.c_int64, C.c_void_p, C.c_int64, C.c_void_p,
                                      C.c_void_p, C.POINTER(Report)]
        L.oracle_emu_gemm.restype = C.c_int
        L.oracle_emu_split.argtypes = [C.c_double, C.c_int, C.c_void_p]
        L.oracle_emu_split.restype = None
        L.oracle_emu_digits.argtypes = [C.c_int64, C.c_void_p]
        L.oracle_emu_digits.restype = None
        L.oracle_emu_i128_to_double.argtypes = [C.c_int64, C.c_uint64]
        L.oracle_emu_i128_to_double.restype = C.c_double
        L.oracle_emu_max_k.argtypes = [C.c_int]
        L.oracle_emu_max_k.restype = C.c_int64
        L.oracle_num_threads.argtypes = []
        L.oracle_num_threads.restype = C.c_int
        _lib = L
    return _lib


def num_threads() -> int:
    return int(lib().oracle_num_threads())


def _f64(x):
    a = np.ascontiguousarray(x, dtype=np.float64)
    return a


def make_problem(layout, transa, transb, M, N, K, alpha, A, lda, B, ldb, beta, Cin, ldc,
                 tile_m=128, tile_n=128, bk=16, keep=None, precision=PREC_FP64, u_acc=U_ACC32, kc=0):
    """Fill a Problem; ``keep`` (a list) receives the arrays that must outlive the call."""
    A = _f64(A); B = _f64(B)
    Cin = _f64(Cin) if Cin is not None else np.zeros(1)
    if keep is not None:
        keep.extend([A, B, Cin])
    p = Problem(layout=layout, transa=transa, transb=transb, pad_=0, M=M, N=N, K=K, alpha=alpha,
                A=A.ctypes.data, lda=lda, B=B.ctypes.data, ldb=ldb, beta=beta,
                Cin=Cin.ctypes.data, ldc=ldc, tile_m=tile_m, tile_n=tile_n, bk=bk,
                precision=precision, pad2_=0, u_acc=u_acc, kc=kc)
    return p


def gemm(layout, transa, transb, M, N, K, alpha, A, lda, B, ldb, beta, Cin, ldc, precision=PREC_FP64):
    """Plain C = alpha*op(A)*op(B) + beta*C_in (the GEMM definition; with PREC_ACC32 the
    result is rounded to binary32). Returns a new buffer."""
    keep = []
    p = make_problem(layout, transa, transb, M, N, K, alpha, A, lda, B, ldb, beta, Cin, ldc, keep=keep,
                     precision=precision)
    out = np.array(keep[2], copy=True) if Cin is not None else np.zeros(max(1, ldc * (N if layout == COL_MAJOR else M)))
    rc = lib().oracle_gemm(C.byref(p), out.ctypes.data)
    if rc != 0:
        raise ValueError("oracle_gemm: bad arguments")
    return out


def trsm_left(T, W, lower):
    """Solve T X = W (T n x n, W n x nrhs, logical matrices) by plain substitution, reading
    only T's lower or upper triangle. Returns X (n x nrhs)."""
    n = T.shape[0]
    nrhs = W.shape[1]
    t = np.asfortranarray(np.asarray(T, dtype=np.float64))
    w = np.array(W, dtype=np.float64, order="F", copy=True)
    lib().oracle_trsm_left(n, nrhs, t.ctypes.data, max(1, n), 1 if lower else 0, w.ctypes.data, max(1, n))
    return w


def gemm_rows(layout, transa, transb, M, N, K, alpha, A, lda, B, ldb, beta, Cin, ldc, rows):
    """Rows ``rows`` of the plain product, as an array of shape (len(rows), N)."""
    keep = []
    p = make_problem(layout, transa, transb, M, N, K, alpha, A, lda, B, ldb, beta, Cin, ldc, keep=keep)
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    out = np.zeros((len(rows), N), dtype=np.float64)
    lib().oracle_gemm_rows(C.byref(p), len(rows), rows.ctypes.data, out.ctypes.data)
    return out


def injections_array(points):
    """``points``: iterable of dicts/tuples (i, j, site, mode, bit, rel_log2, sign[, kt]);
    kt: the accumulator flip lands after kt * bk products (0: after bk * floor(nk / 2))."""
    pts = list(points)
    arr = (Injection * max(1, len(pts)))()
    for q, pt in enumerate(pts):
        if isinstance(pt, dict):
            pt = (pt["i"], pt["j"], pt.get("site", SITE_ACCUM), pt.get("mode", MODE_BITFLIP),
                  pt.get("bit", 0), pt.get("rel_log2", 0), pt.get("sign", 1), pt.get("kt", 0))
        if len(pt) == 7:
            pt = tuple(pt) + (0,)
        i, j, site, mode, bit, rel, sign, kt = pt
        arr[q] = Injection(i=i, j=j, site=site, mode=mode, bit=bit, rel_log2=rel, sign=sign, kt=kt)
    return arr, len(pts)


def ft_gemm(layout, transa, transb, M, N, K, alpha, A, lda, B, ldb, beta, Cin, ldc,
            tile_m, tile_n, bk, injections=(), tiles=None, out=None, precision=PREC_FP64, u_acc=U_ACC32, kc=0):
    """ABFT-protected GEMM. Returns ``(Cout_buffer, Report)``.

    ``tiles``: None for all tiles, else tile numbers t = tile_row + tile_col * n_tile_rows
    (only those tiles of the output are written; ``out`` may carry the rest).
    """
    keep = []
    p = make_problem(layout, transa, transb, M, N, K, alpha, A, lda, B, ldb, beta, Cin, ldc,
                     tile_m, tile_n, bk, keep=keep, precision=precision, u_acc=u_acc, kc=kc)
    if out is None:
        n_store = max(1, ldc * (N if layout == COL_MAJOR else M))
        out = np.array(keep[2], copy=True) if Cin is not None and beta != 0.0 else np.zeros(n_store)
    inj, n_inj = injections_array(injections)
    rep = Report()
    if tiles is None:
        rc = lib().oracle_ft_gemm(C.byref(p), n_inj, C.addressof(inj), 0, None, out.ctypes.data, C.byref(rep))
    else:
        t = np.ascontiguousarray(tiles, dtype=np.int64)
        rc = lib().oracle_ft_gemm(C.byref(p), n_inj, C.addressof(inj), len(t), t.ctypes.data, out.ctypes.data,
                                  C.byref(rep))
    if rc != 0:
        raise ValueError("oracle_ft_gemm: bad arguments")
    return out, rep


def draw_injections(seed, launch, every_n, per_launch, site, mode, bit_lo, bit_hi, log2_lo, log2_hi,
                    M, N, tile_m, tile_n, cap=256):
    """The seeded injection draw of one launch (the oracle's own SplitMix64)."""
    arr = (Injection * cap)()
    n = lib().oracle_draw_injections(seed, launch, every_n, per_launch, site, mode, bit_lo, bit_hi,
                                     log2_lo, log2_hi, M, N, tile_m, tile_n, cap, C.addressof(arr))
    return [dict(i=arr[q].i, j=arr[q].j, site=arr[q].site, mode=arr[q].mode, bit=arr[q].bit,
                 rel_log2=arr[q].rel_log2, sign=arr[q].sign) for q in range(n)]


# ------------------------------------------------------------------------------------
# The emulated FP64 product (emu_oracle.c): binary64 operands as integer slices with
# exact group products and exact integer checksums.
# ------------------------------------------------------------------------------------
EMU_SLICES = 14
EMU_TILE_M, EMU_TILE_N = 128, 248


def emu_gemm(layout, transa, transb, M, N, K, alpha, A, lda, B, ldb, beta, Cin, ldc, slices=EMU_SLICES,
             injections=(), tiles=None, out=None, tile_m=EMU_TILE_M, tile_n=EMU_TILE_N):
    """The emulated protected GEMM. Returns ``(Cout_buffer, Report)``; ``tiles`` as in
    ``ft_gemm`` (caller tile numbering; tiles are tile_n x tile_m for row-major calls)."""
    A = _f64(A); B = _f64(B)
    Cin_ = _f64(Cin) if Cin is not None else np.zeros(1)
    p = EmuProblem(layout=layout, transa=transa, transb=transb, slices=slices, M=M, N=N, K=K, alpha=alpha,
                   A=A.ctypes.data, lda=lda, B=B.ctypes.data, ldb=ldb, beta=beta, Cin=Cin_.ctypes.data, ldc=ldc,
                   tile_m=tile_m, tile_n=tile_n)
    if out is None:
        n_store = max(1, ldc * (N if layout == COL_MAJOR else M))
        out = np.array(Cin_, copy=True) if Cin is not None and beta != 0.0 else np.zeros(n_store)
    inj, n_inj = injections_array(injections)
    rep = Report()
    if tiles is None:
        rc = lib().oracle_emu_gemm(C.byref(p), n_inj, C.addressof(inj), 0, None, out.ctypes.data, C.byref(rep))
    else:
        t = np.ascontiguousarray(tiles, dtype=np.int64)
        rc = lib().oracle_emu_gemm(C.byref(p), n_inj, C.addressof(inj), len(t), t.ctypes.data, out.ctypes.data,
                                   C.byref(rep))
    if rc != 0:
        raise ValueError(f"oracle_emu_gemm: rc {rc}")
    return out, rep


def emu_split(x, slices=EMU_SLICES):
    """The integer slices of x in (-1, 1)."""
    out = (C.c_int32 * slices)()
    lib().oracle_emu_split(float(x), slices, out)
    return [int(v) for v in out]


def emu_digits(v):
    """The four base-16 digits (each in [-8, 8]) of the integer v."""
    out = (C.c_int32 * 4)()
    lib().oracle_emu_digits(int(v), out)
    return [int(d) for d in out]


def emu_i128_to_double(x):
    """The oracle's rounded-to-nearest conversion of a 128-bit integer x."""
    x = int(x) & ((1 << 128) - 1)
    hi = x >> 64
    if hi >= 1 << 63:
        hi -= 1 << 64
    return lib().oracle_emu_i128_to_double(hi, x & ((1 << 64) - 1))


def emu_max_k(slices=EMU_SLICES):
    return int(lib().oracle_emu_max_k(slices))
