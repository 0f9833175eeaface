"""Python binding of libftblas (the ABFT-protected GEMM of FT-BLAS on GB300).

Argument marshalling only: every function here forwards to the C ABI of
``include/ftblas.h`` under the same name, and the torch helpers just turn tensors into
pointers, leading dimensions and the current CUDA stream. No step of the product,
checksum encode, verification or correction runs in Python, and there is no CPU
fallback: if the CUDA library is missing or cannot be loaded, importing the binding's
functions raises.
"""
from __future__ import annotations

import ctypes as C
import os

from . import build as _build

ROW_MAJOR, COL_MAJOR = 101, 102
NO_TRANS, TRANS = 111, 112
UPPER, LOWER = 121, 122
NON_UNIT, UNIT = 131, 132
LEFT, RIGHT = 141, 142
R_64F, R_32F, R_16BF, R_8F_E4M3 = 0, 1, 2, 3
SITE_ACCUM, SITE_OUTPUT, SITE_CHECKSUM, SITE_STALL = 1, 2, 3, 4
MODE_BITFLIP, MODE_ADD_REL = 0, 1
KIND_CORRECTED, KIND_CHECKSUM_ONLY, KIND_UNCORRECTABLE, KIND_INPUT_NONFINITE = 1, 2, 3, 4
STATUS_TIMEOUT, STATUS_RECORDS_TRUNCATED = 1, 2
STATUS_NOT_SUPPORTED, STATUS_CUDA_ERROR, STATUS_ALLOC_FAILED, STATUS_WORKSPACE_LIMIT = 2, 3, 4, 5
ENGINE_DFMA, ENGINE_DMMA = 0, 1
MAX_RECORDS = 64
MAX_FIXED_INJECTIONS = 16
MAX_INJECTIONS_PER_LAUNCH = 64


class FtErrorRecord(C.Structure):
    _fields_ = [
        ("tile_row", C.c_int64), ("tile_col", C.c_int64), ("i", C.c_int64), ("j", C.c_int64),
        ("delta_row", C.c_double), ("delta_col", C.c_double),
        ("tau_row", C.c_double), ("tau_col", C.c_double),
        ("value_before", C.c_double), ("value_after", C.c_double),
        ("kind", C.c_int32), ("rows_flagged", C.c_int32), ("cols_flagged", C.c_int32), ("reserved", C.c_int32),
    ]


class FtReport(C.Structure):
    _fields_ = [
        ("tiles_checked", C.c_uint64), ("detected", C.c_uint64), ("corrected", C.c_uint64),
        ("uncorrectable", C.c_uint64), ("checksum_only", C.c_uint64), ("input_nonfinite", C.c_uint64),
        ("status", C.c_uint32), ("n_records", C.c_uint32),
        ("rec", FtErrorRecord * MAX_RECORDS),
    ]

    def records(self):
        return [self.rec[q] for q in range(min(self.n_records, MAX_RECORDS))]

    def as_dict(self):
        return dict(tiles_checked=self.tiles_checked, detected=self.detected, corrected=self.corrected,
                    uncorrectable=self.uncorrectable, checksum_only=self.checksum_only,
                    input_nonfinite=self.input_nonfinite, status=self.status, n_records=self.n_records,
                    records=[{f: getattr(r, f) for f, _ in FtErrorRecord._fields_} for r in self.records()])


class FtInjectPoint(C.Structure):
    _fields_ = [("i", C.c_int64), ("j", C.c_int64), ("site", C.c_int32), ("mode", C.c_int32),
                ("bit", C.c_int32), ("rel_log2", C.c_int32), ("sign", C.c_int32), ("k_tile", C.c_int32)]


class FtInject(C.Structure):
    _fields_ = [("seed", C.c_uint64), ("site", C.c_int32), ("mode", C.c_int32),
                ("bit_lo", C.c_int32), ("bit_hi", C.c_int32), ("log2_lo", C.c_int32), ("log2_hi", C.c_int32),
                ("every_n_launches", C.c_int32), ("errors_per_launch", C.c_int32),
                ("n_fixed", C.c_int32), ("reserved", C.c_int32),
                ("fixed", FtInjectPoint * MAX_FIXED_INJECTIONS)]


REPORT_BYTES = C.sizeof(FtReport)

# (name, restype, argtypes) of every entry point declared in include/ftblas.h
_GEMM_ARGS = [C.c_int, C.c_int, C.c_int, C.c_int64, C.c_int64, C.c_int64, C.c_double, C.c_void_p, C.c_int64,
              C.c_void_p, C.c_int64, C.c_double, C.c_void_p, C.c_int64]
_GEMM_EX_ARGS = [C.c_int, C.c_int, C.c_int, C.c_int64, C.c_int64, C.c_int64, C.c_void_p, C.c_void_p, C.c_int,
                 C.c_int64, C.c_void_p, C.c_int, C.c_int64, C.c_void_p, C.c_void_p, C.c_int, C.c_int64, C.c_int,
                 C.c_void_p, C.c_void_p, C.c_void_p]
SIGNATURES = {
    "ftblas_gemm_ex": (C.c_int, _GEMM_EX_ARGS + [C.c_void_p]),
    "ftblas_gemm_ex_noabft": (C.c_int, _GEMM_EX_ARGS),
    "ftblas_gemm_ex_noalloc": (C.c_int, _GEMM_EX_ARGS + [C.c_void_p]),
    "ftblas_set_injection": (C.c_int, [C.c_void_p]),
    "ftblas_injection_launch_count": (C.c_uint64, []),
    "ftblas_dgemm": (C.c_int, _GEMM_ARGS + [C.c_void_p, C.c_void_p]),
    "ftblas_dgemm_noabft": (C.c_int, _GEMM_ARGS + [C.c_void_p]),
    "ftblas_dgemm_host": (C.c_int, _GEMM_ARGS + [C.c_void_p, C.c_void_p]),
    "ftblas_dgemm_unfused": (C.c_int, _GEMM_ARGS + [C.c_void_p, C.c_void_p]),
    "ftblas_dgemm_emulated": (C.c_int, _GEMM_ARGS + [C.c_void_p, C.c_void_p]),
    "ftblas_dgemm_emulated_noabft": (C.c_int, _GEMM_ARGS + [C.c_void_p]),
    "ftblas_set_emulation_slices": (C.c_int, [C.c_int]),
    "ftblas_emulation_max_k": (C.c_int64, [C.c_int]),
    "ftblas_emu_convert_i128": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p]),
    "ftblas_dsymm": (C.c_int, [C.c_int, C.c_int, C.c_int, C.c_int64, C.c_int64, C.c_double, C.c_void_p, C.c_int64,
                               C.c_void_p, C.c_int64, C.c_double, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p]),
    "ftblas_dtrmm": (C.c_int, [C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int64, C.c_int64, C.c_double,
                               C.c_void_p, C.c_int64, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p]),
    "ftblas_dtrsm": (C.c_int, [C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int64, C.c_int64, C.c_double,
                               C.c_void_p, C.c_int64, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p]),
    "ftblas_verification_tile": (C.c_int, [C.c_int, C.c_int, C.c_int64, C.c_int64, C.c_int64,
                                           C.c_void_p, C.c_void_p, C.c_void_p]),
    "ftblas_set_fp64_engine": (C.c_int, [C.c_int]),
    "ftblas_set_tc_cta_group": (C.c_int, [C.c_int]),
    "ftblas_set_fp64_tile": (C.c_int, [C.c_int]),
    "ftblas_set_verification_interval": (C.c_int64, [C.c_int64]),
    "ftblas_status_string": (C.c_char_p, [C.c_int]),
    "ftblas_last_cuda_error": (C.c_int, []),
    "ftblas_last_launch_used_tma": (C.c_int, []),
    "ftblas_version": (C.c_char_p, []),
    "ftblas_decode_e4m3": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p]),
    "ftblas_kernel_timing_begin": (C.c_int, []),
    "ftblas_kernel_timing_end": (C.c_int, [C.c_void_p, C.c_void_p]),
}

_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_needed: bool = True):
    """Load libftblas.so (building it first if asked). Raises if it cannot be loaded."""
    global _lib
    if _lib is None:
        path = _build.build() if build_if_needed else _build.LIB
        if not os.path.exists(path):
            raise RuntimeError(f"libftblas.so not found at {path}; run paper_2104_00897_gb300.build.build()")
        lib = C.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def _call(name, *args):
    return getattr(load(), name)(*args)


# ------------------------------------------------------------------ C ABI, same names
def ftblas_dgemm(layout, transa, transb, M, N, K, alpha, A, lda, B, ldb, beta, C_, ldc, stream, report):
    return _call("ftblas_dgemm", layout, transa, transb, M, N, K, alpha, A, lda, B, ldb, beta, C_, ldc, stream, report)


def ftblas_dgemm_noabft(layout, transa, transb, M, N, K, alpha, A, lda, B, ldb, beta, C_, ldc, stream):
    return _call("ftblas_dgemm_noabft", layout, transa, transb, M, N, K, alpha, A, lda, B, ldb, beta, C_, ldc, stream)


def ftblas_dgemm_unfused(layout, transa, transb, M, N, K, alpha, A, lda, B, ldb, beta, C_, ldc, stream, report):
    return _call("ftblas_dgemm_unfused", layout, transa, transb, M, N, K, alpha, A, lda, B, ldb, beta, C_, ldc, stream,
                 report)


def ftblas_dgemm_emulated(layout, transa, transb, M, N, K, alpha, A, lda, B, ldb, beta, C_, ldc, stream, report):
    return _call("ftblas_dgemm_emulated", layout, transa, transb, M, N, K, alpha, A, lda, B, ldb, beta, C_, ldc,
                 stream, report)


def ftblas_dgemm_emulated_noabft(layout, transa, transb, M, N, K, alpha, A, lda, B, ldb, beta, C_, ldc, stream):
    return _call("ftblas_dgemm_emulated_noabft", layout, transa, transb, M, N, K, alpha, A, lda, B, ldb, beta, C_,
                 ldc, stream)


def ftblas_set_emulation_slices(slices):
    return _call("ftblas_set_emulation_slices", slices)


def ftblas_emulation_max_k(slices):
    return _call("ftblas_emulation_max_k", slices)


def ftblas_emu_convert_i128(words, out, n, stream=None):
    return _call("ftblas_emu_convert_i128", words, out, n, stream)


def ftblas_dsymm(layout, side, uplo, M, N, alpha, A, lda, B, ldb, beta, C_, ldc, stream, report):
    return _call("ftblas_dsymm", layout, side, uplo, M, N, alpha, A, lda, B, ldb, beta, C_, ldc, stream, report)


def ftblas_dtrmm(layout, side, uplo, transa, diag, M, N, alpha, A, lda, B, ldb, stream, report):
    return _call("ftblas_dtrmm", layout, side, uplo, transa, diag, M, N, alpha, A, lda, B, ldb, stream, report)


def ftblas_dtrsm(layout, side, uplo, transa, diag, M, N, alpha, A, lda, B, ldb, stream, report):
    return _call("ftblas_dtrsm", layout, side, uplo, transa, diag, M, N, alpha, A, lda, B, ldb, stream, report)


def ftblas_dgemm_host(layout, transa, transb, M, N, K, alpha, A, lda, B, ldb, beta, C_, ldc, stream, report):
    return _call("ftblas_dgemm_host", layout, transa, transb, M, N, K, alpha, A, lda, B, ldb, beta, C_, ldc, stream,
                 report)


def ftblas_gemm_ex(layout, transa, transb, M, N, K, alpha, A, Atype, lda, B, Btype, ldb, beta, C_, Ctype, ldc,
                   compute_type, a_scale, b_scale, stream, report):
    """alpha / beta: host scalars, passed by pointer as the compute type requires."""
    al, be = _scalar(alpha, compute_type), _scalar(beta, compute_type)
    return _call("ftblas_gemm_ex", layout, transa, transb, M, N, K, C.addressof(al), A, Atype, lda, B, Btype, ldb,
                 C.addressof(be), C_, Ctype, ldc, compute_type, a_scale, b_scale, stream, report)


def ftblas_gemm_ex_noabft(layout, transa, transb, M, N, K, alpha, A, Atype, lda, B, Btype, ldb, beta, C_, Ctype,
                          ldc, compute_type, a_scale, b_scale, stream):
    al, be = _scalar(alpha, compute_type), _scalar(beta, compute_type)
    return _call("ftblas_gemm_ex_noabft", layout, transa, transb, M, N, K, C.addressof(al), A, Atype, lda, B, Btype,
                 ldb, C.addressof(be), C_, Ctype, ldc, compute_type, a_scale, b_scale, stream)


def ftblas_gemm_ex_noalloc(layout, transa, transb, M, N, K, alpha, A, Atype, lda, B, Btype, ldb, beta, C_, Ctype,
                           ldc, compute_type, a_scale, b_scale, stream, report):
    """ftblas_gemm_ex on the library's static 16 MiB device scratch: allocates nothing."""
    al, be = _scalar(alpha, compute_type), _scalar(beta, compute_type)
    return _call("ftblas_gemm_ex_noalloc", layout, transa, transb, M, N, K, C.addressof(al), A, Atype, lda, B, Btype,
                 ldb, C.addressof(be), C_, Ctype, ldc, compute_type, a_scale, b_scale, stream, report)


def _scalar(x, compute_type):
    return C.c_double(float(x)) if compute_type == R_64F else C.c_float(float(x))


def ftblas_set_injection(cfg):
    """cfg: FtInject, or None to switch injection off (also resets the launch counter)."""
    return _call("ftblas_set_injection", None if cfg is None else C.addressof(cfg))


def ftblas_injection_launch_count():
    return int(_call("ftblas_injection_launch_count"))


def ftblas_verification_tile(layout, compute_type, M, N, K):
    r, c, k = C.c_int64(), C.c_int64(), C.c_int64()
    rc = _call("ftblas_verification_tile", layout, compute_type, M, N, K, C.addressof(r), C.addressof(c),
               C.addressof(k))
    if rc != 0:
        raise ValueError(f"ftblas_verification_tile: argument {-rc} invalid")
    return r.value, c.value, k.value


def ftblas_set_verification_interval(k_interval):
    return _call("ftblas_set_verification_interval", int(k_interval))


def ftblas_set_fp64_engine(engine):
    return _call("ftblas_set_fp64_engine", engine)


def ftblas_set_tc_cta_group(cta_group):
    return _call("ftblas_set_tc_cta_group", cta_group)


def tc_cta_group(protected=True):
    """The tensor-core kernel form a call takes (1: one CTA per tile, 2: CTA pairs)."""
    cur = ftblas_set_tc_cta_group(0)
    ftblas_set_tc_cta_group(cur)
    return cur if cur != 0 else 2


def ftblas_set_fp64_tile(edge):
    return _call("ftblas_set_fp64_tile", int(edge))


def ftblas_status_string(code):
    return _call("ftblas_status_string", code).decode()


def ftblas_last_cuda_error():
    return _call("ftblas_last_cuda_error")


def ftblas_last_launch_used_tma():
    return _call("ftblas_last_launch_used_tma")


def ftblas_version():
    return _call("ftblas_version").decode()


def ftblas_decode_e4m3(codes, out, n, stream=None):
    return _call("ftblas_decode_e4m3", codes, out, int(n), stream)


# ------------------------------------------------------------------ helpers
def ftblas_kernel_timing_begin():
    return _call("ftblas_kernel_timing_begin")


def ftblas_kernel_timing_end():
    """Returns (rc, total_ms, launches) of the product kernels timed since begin."""
    t = C.c_double(0.0)
    n = C.c_int64(0)
    rc = _call("ftblas_kernel_timing_end", C.byref(t), C.byref(n))
    return rc, t.value, n.value


def make_injection(seed=0, site=SITE_ACCUM, mode=MODE_BITFLIP, bit_lo=40, bit_hi=62, log2_lo=0, log2_hi=0,
                   every_n_launches=0, errors_per_launch=0, fixed=()):
    """Build an FtInject. ``fixed``: iterable of dicts with i, j and optional site, mode,
    bit, rel_log2, sign and kt (FP64 accumulator flips: after kt k-tiles, 0 = floor(nk/2));
    when given, those points are injected on every launch."""
    cfg = FtInject(seed=seed, site=site, mode=mode, bit_lo=bit_lo, bit_hi=bit_hi, log2_lo=log2_lo, log2_hi=log2_hi,
                   every_n_launches=every_n_launches, errors_per_launch=errors_per_launch, n_fixed=0, reserved=0)
    pts = list(fixed)
    if len(pts) > MAX_FIXED_INJECTIONS:
        raise ValueError("too many fixed injection points")
    for q, p in enumerate(pts):
        cfg.fixed[q] = FtInjectPoint(i=p["i"], j=p["j"], site=p.get("site", SITE_ACCUM),
                                     mode=p.get("mode", MODE_BITFLIP), bit=p.get("bit", 0),
                                     rel_log2=p.get("rel_log2", 0), sign=p.get("sign", 1), k_tile=p.get("kt", 0))
    cfg.n_fixed = len(pts)
    return cfg


def check(rc, what="ftblas call"):
    if rc != 0:
        raise RuntimeError(f"{what} failed: {rc} ({ftblas_status_string(rc)}; cuda error {ftblas_last_cuda_error()})")
    return rc


def report_from_device(buf) -> FtReport:
    """Copy a device report (a torch uint8 tensor of REPORT_BYTES) into an FtReport."""
    host = buf.detach().to("cpu").numpy().tobytes()
    return FtReport.from_buffer_copy(host)


def new_report(device=None):
    """A device buffer for one ft_report_t (torch uint8 tensor)."""
    import torch
    return torch.zeros(REPORT_BYTES, dtype=torch.uint8, device=device or "cuda")


def _layout_of(t):
    """(layout, ld) of a 2-D tensor whose storage is row- or column-major with a unit stride."""
    r, c = t.shape
    s0, s1 = t.stride()
    if s1 == 1 and (s0 >= max(1, c) or r <= 1):
        return ROW_MAJOR, max(s0, max(1, c))
    if s0 == 1 and (s1 >= max(1, r) or c <= 1):
        return COL_MAJOR, max(s1, max(1, r))
    return None, None


def _require_cuda(name, t, dtype=None, device=None, numel=None):
    """Raise unless t is a CUDA tensor (of the given dtype, on the given device, with the
    given number of elements): the C ABI takes raw device pointers, so a host tensor or a
    wrong element type must be refused before any launch."""
    if not getattr(t, "is_cuda", False):
        raise ValueError(f"{name} must be a CUDA tensor (got {getattr(t, 'device', type(t))})")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if device is not None and t.device != device:
        raise ValueError(f"{name} is on {t.device}, the operands on {device}")
    if numel is not None and t.numel() != numel:
        raise ValueError(f"{name} must have {numel} element(s), has {t.numel()}")


def dgemm(a, b, c=None, alpha=1.0, beta=0.0, trans_a=False, trans_b=False, report=None, protect=True,
          stream=None):
    """c = alpha * op(a) @ op(b) + beta * c on float64 CUDA tensors, protected by ABFT.

    Tensors may be row-major or column-major (a unit stride in either dimension); the
    layout of ``c`` decides the call's layout and the operands are brought to it by
    copies when they differ. ``report``: a buffer from new_report() (or None). Returns c.
    """
    import torch
    _require_cuda("a", a, torch.float64)
    _require_cuda("b", b, torch.float64, a.device)
    if c is not None:
        _require_cuda("c", c, torch.float64, a.device)
    if report is not None:
        _require_cuda("report", report, device=a.device)
    Ma, Ka = (a.shape[1], a.shape[0]) if trans_a else (a.shape[0], a.shape[1])
    Kb, Nb = (b.shape[1], b.shape[0]) if trans_b else (b.shape[0], b.shape[1])
    if Ka != Kb:
        raise ValueError(f"inner dimensions differ: {Ka} vs {Kb}")
    M, N, K = Ma, Nb, Ka
    if c is None:
        c = torch.empty((M, N), dtype=torch.float64, device=a.device)
        if beta != 0.0:
            raise ValueError("beta != 0 needs c")
    layout, ldc = _layout_of(c)
    if layout is None:
        raise ValueError("c must have a unit stride in one dimension")

    def as_layout(x):
        lay, ld = _layout_of(x)
        if lay == layout:
            return x, ld
        y = x.contiguous() if layout == ROW_MAJOR else x.t().contiguous().t()
        return y, _layout_of(y)[1]

    a2, lda = as_layout(a)
    b2, ldb = as_layout(b)
    st = stream if stream is not None else torch.cuda.current_stream(a.device).cuda_stream
    ta = TRANS if trans_a else NO_TRANS
    tb = TRANS if trans_b else NO_TRANS
    if protect:
        rc = ftblas_dgemm(layout, ta, tb, M, N, K, float(alpha), a2.data_ptr(), lda, b2.data_ptr(), ldb, float(beta),
                          c.data_ptr(), ldc, st, report.data_ptr() if report is not None else None)
    else:
        rc = ftblas_dgemm_noabft(layout, ta, tb, M, N, K, float(alpha), a2.data_ptr(), lda, b2.data_ptr(), ldb,
                                 float(beta), c.data_ptr(), ldc, st)
    check(rc, "ftblas_dgemm")
    return c


# ---------------------------------------------------------------------------------------
# Torch-level API: gemm on tensors of any supported dtype, and a protected linear layer.
# ---------------------------------------------------------------------------------------

def _kmajor_rows(x):
    """x (rows x K) as a row-major tensor whose rows are K-contiguous, 16-byte aligned and
    with a 16-byte multiple pitch (what the tensor maps need); copies when x is not."""
    import torch
    es = x.element_size()
    if (x.stride(1) == 1 and x.stride(0) >= max(1, x.shape[1]) and (x.stride(0) * es) % 16 == 0
            and x.data_ptr() % 16 == 0):
        return x, x.stride(0)
    pitch = -(-max(1, x.shape[1]) * es // 16) * 16 // es
    y = torch.zeros((x.shape[0], pitch), dtype=x.dtype, device=x.device)[:, :x.shape[1]]
    y.copy_(x)
    return y, pitch


def _row_major_operand(x):
    """How a (rows x K) tensor x enters a row-major call: (NO_TRANS, x, ld) when its rows
    of K are contiguous (copied first when the base or pitch is not 16-byte aligned), or
    (TRANS, x, ld) when its columns are, x then being read as the transpose of a row-major
    K x rows array (the library copies it K-major itself)."""
    if x.stride(1) == 1 and (x.shape[0] <= 1 or x.stride(0) >= max(1, x.shape[1])):
        y, ld = _kmajor_rows(x)
        return NO_TRANS, y, ld
    if x.stride(0) == 1 and (x.shape[1] <= 1 or x.stride(1) >= max(1, x.shape[0])):
        return TRANS, x, max(1, x.stride(1) if x.shape[1] > 1 else x.shape[0])
    y, ld = _kmajor_rows(x)
    return NO_TRANS, y, ld


def gemm(a, b, c=None, alpha=1.0, beta=0.0, trans_a=False, trans_b=False, report=None, protect=True,
         a_scale=None, b_scale=None, stream=None, out_dtype=None):
    """c = alpha * op(a) @ op(b) + beta * c on CUDA tensors, protected by ABFT.

    float64 operands run the FP64 kernel (c float64, see dgemm). bfloat16 or
    float8_e4m3fn operands run the tensor-core kernel with FP32 accumulation and a float32
    or bfloat16 c (``out_dtype`` when c is None, float32 by default; a bfloat16 c is
    verified and corrected in FP32 and rounded once); a_scale / b_scale are 1-element
    float32 CUDA tensors (FP8 per-tensor scales) or None. Operands are passed through in
    either storage order (the library copies an MN-major operand K-major for the
    tensor-core kernel). ``report``: a buffer from new_report() (or None). Returns c.
    """
    import torch
    if a.dtype == torch.float64:
        return dgemm(a, b, c, alpha, beta, trans_a, trans_b, report, protect, stream)
    fp8 = a.dtype == getattr(torch, "float8_e4m3fn", None)
    if a.dtype != b.dtype or not (a.dtype == torch.bfloat16 or fp8):
        raise TypeError(f"unsupported operand dtypes {a.dtype}, {b.dtype}")
    _require_cuda("a", a)
    _require_cuda("b", b, device=a.device)
    if c is not None:
        _require_cuda("c", c, device=a.device)
    if report is not None:
        _require_cuda("report", report, device=a.device)
    for name, sc in (("a_scale", a_scale), ("b_scale", b_scale)):
        if sc is not None:
            _require_cuda(name, sc, torch.float32, a.device, numel=1)
    opa = a.t() if trans_a else a          # M x K
    opb_t = b if trans_b else b.t()        # N x K
    M, K = opa.shape
    N, Kb = opb_t.shape
    if K != Kb:
        raise ValueError(f"inner dimensions differ: {K} vs {Kb}")
    if c is None:
        if beta != 0.0:
            raise ValueError("beta != 0 needs c")
        c = torch.empty((M, N), dtype=out_dtype if out_dtype is not None else torch.float32, device=a.device)
    if c.dtype not in (torch.float32, torch.bfloat16):
        raise TypeError("c must be float32 or bfloat16 for bfloat16 / float8 operands")
    if c.shape != (M, N):
        raise ValueError(f"c has shape {tuple(c.shape)}, expected {(M, N)}")
    if c.stride(1) != 1:
        if c.stride(0) == 1:  # column-major c: compute c^T = op(b)^T op(a)^T into its row-major view
            return gemm(b, a, c.t(), alpha, beta, not trans_b, not trans_a, report, protect, b_scale, a_scale, stream,
                        out_dtype)
        raise ValueError("c must have a unit stride in one dimension")
    # Row-major call. An operand whose rows of K are contiguous is passed as it is (the
    # tensor maps want a 16-byte aligned base and pitch; otherwise it is copied into that
    # form); one stored the other way is passed transposed, and the library makes its own
    # K-major copy.
    ta_, a2, lda = _row_major_operand(opa)
    tb_k, b2, ldb = _row_major_operand(opb_t)
    tb_ = TRANS if tb_k == NO_TRANS else NO_TRANS   # op(B) = opb_t^T
    st = stream if stream is not None else torch.cuda.current_stream(a.device).cuda_stream
    dt = R_8F_E4M3 if fp8 else R_16BF
    sa = a_scale.data_ptr() if a_scale is not None else None
    sb = b_scale.data_ptr() if b_scale is not None else None
    ct = R_16BF if c.dtype == torch.bfloat16 else R_32F
    args = (ROW_MAJOR, ta_, tb_, M, N, K, float(alpha), a2.data_ptr(), dt, lda, b2.data_ptr(), dt, ldb,
            float(beta), c.data_ptr(), ct, max(1, c.stride(0)), R_32F, sa, sb, st)
    if protect:
        rc = ftblas_gemm_ex(*args, report.data_ptr() if report is not None else None)
    else:
        rc = ftblas_gemm_ex_noabft(*args)
    check(rc, "ftblas_gemm_ex")
    return c


class FTMonitor:
    """Collects the report of every protected GEMM issued through it (one device buffer per
    call); summary() synchronises and sums them."""

    def __init__(self, device=None):
        self.device = device
        self.reports = []

    def next_report(self):
        # every protected call zeroes its report on the stream before anything else, so the
        # monitor's buffers need no fill of their own
        import torch
        r = torch.empty(REPORT_BYTES, dtype=torch.uint8, device=self.device or "cuda")
        self.reports.append(r)
        return r

    def summary(self):
        tot = dict(calls=len(self.reports), tiles_checked=0, detected=0, corrected=0, uncorrectable=0,
                   checksum_only=0, status=0)
        for buf in self.reports:
            r = report_from_device(buf)
            for k in ("tiles_checked", "detected", "corrected", "uncorrectable", "checksum_only"):
                tot[k] += int(getattr(r, k))
            tot["status"] |= int(r.status)
        return tot


def _ft_linear_class():
    import torch

    class FTLinearFn(torch.autograd.Function):
        """Y = X W^T with every GEMM ABFT-protected: the forward product and, in the
        backward pass, dX = dY W and dW = dY^T X. float64 X, W run the FP64 kernel (Y and
        the gradients float64). bfloat16 X, W run the tensor-core kernel with FP32
        accumulation: Y and the gradients are bfloat16, each verified and corrected in FP32
        and rounded once by the library (a dY of another dtype is rounded to bfloat16 first).
        ``monitor`` (an FTMonitor or None) receives the three calls' reports."""

        @staticmethod
        def forward(ctx, x, w, monitor=None):
            ctx.save_for_backward(x, w)
            ctx.monitor = monitor
            rep = monitor.next_report() if monitor is not None else None
            return gemm(x, w, trans_b=True, report=rep, out_dtype=x.dtype)

        @staticmethod
        def backward(ctx, dy):
            x, w = ctx.saved_tensors
            mon = ctx.monitor
            dyq = dy.to(x.dtype) if x.dtype != dy.dtype else dy
            dx = dw = None
            if ctx.needs_input_grad[0]:
                dx = gemm(dyq, w, report=mon.next_report() if mon is not None else None, out_dtype=x.dtype)
            if ctx.needs_input_grad[1]:
                dw = gemm(dyq, x, trans_a=True, report=mon.next_report() if mon is not None else None,
                          out_dtype=w.dtype)
            return dx, dw, None

    return FTLinearFn


def __getattr__(name):
    if name == "FTLinearFn":
        cls = _ft_linear_class()
        globals()["FTLinearFn"] = cls
        return cls
    raise AttributeError(name)
