"""ctypes binding of ``libgbgreen.so`` (argument marshalling only).

Every step of the shifted Green's-function path runs in the library's CUDA
kernels; this module only converts PyTorch tensors / NumPy arrays into the
plain pointers and sizes of the C ABI (``include/gbgreen.h``).  There is no
CPU fallback: if the library is missing or no CUDA device is present, calls
raise.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.environ.get("GBGREEN_LIB") or os.path.join(_HERE, "libgbgreen.so")

GB_OK, GB_EINVAL, GB_ENOMEM, GB_ECUDA, GB_ENOTSPD, GB_EBREAKDOWN, GB_ENOCONV, GB_ETIMEOUT = 0, -1, -2, -3, -4, -5, -6, -7
FLAG_STALL = 64  # gb_solve_params.flags bit 6: stop stalled columns early
GB_FP64, GB_MIXED = 0, 1
_STATUS = {0: "GB_OK", -1: "GB_EINVAL", -2: "GB_ENOMEM", -3: "GB_ECUDA", -4: "GB_ENOTSPD", -5: "GB_EBREAKDOWN",
           -6: "GB_ENOCONV", -7: "GB_ETIMEOUT"}

EXPORTED = (
    "gb_abi_version",
    "gb_last_error",
    "gb_bsr_to_host",
    "gb_block_factor_to_host",
    "gb_build_bsr",
    "gb_matrix_get_info",
    "gb_free",
    "gb_spmm",
    "gb_apply_sinv",
    "gb_solve_workspace_size",
    "gb_solve_plan",
    "gb_shifted_solve",
    "gb_shifted_solve_static",
    "gb_static_scratch_bytes",
    "gb_shifted_solve_batched",
    "gb_true_residual",
    "gb_fermi_density",
    "gb_correct_batched",
    "gb_forces",
    "gb_wavepacket",
    "gb_wavepacket_workspace_size",
    "gb_add_sinv_terms",
    "gb_add_sinv_terms_workspace_size",
    "gb_forces_workspace_size",
    "gb_correct_batched_workspace_size",
    "gb_fermi_workspace_size",
    "gb_true_residual_workspace_size",
    "gb_correct_unconverged",
    "gb_correct_workspace_size",
    "gb_batched_workspace_size",
    "gb_tune_panel_batched",
)


class GBError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


class MatrixInfo(C.Structure):
    _fields_ = [("n", C.c_int64), ("nnz", C.c_int64), ("nb", C.c_int64), ("nnzb", C.c_int64),
                ("max_row", C.c_int32), ("block", C.c_int32), ("device", C.c_int32), ("factor_bw", C.c_int32),
                ("s_lam_min", C.c_double), ("s_lam_max", C.c_double), ("factor_nblk", C.c_int64)]


class SolveParams(C.Structure):
    _fields_ = [
        ("nshift", C.c_int32),
        ("z_re", C.POINTER(C.c_double)),
        ("z_im", C.POINTER(C.c_double)),
        ("w_rho", C.POINTER(C.c_double)),
        ("w_edm", C.POINTER(C.c_double)),
        ("nrhs", C.c_int32),
        ("rhs_cols", C.POINTER(C.c_int32)),
        ("tol", C.c_double),
        ("maxit", C.c_int32),
        ("prec", C.c_int32),
        ("inner_tol", C.c_double),
        ("panel", C.c_int32),
        ("flags", C.c_int32),
        ("seed_shift", C.c_int32),
        ("reserved", C.c_int32),
    ]


class Outputs(C.Structure):
    _fields_ = [(f, C.c_void_p) for f in ("ldos", "rho", "edm", "q", "e_loc", "iters", "converged", "resid", "g_proj",
                                            "inner_iters", "col_status")]


_lib = None


def load() -> C.CDLL:
    """Load the in-tree library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: run `python -c 'import __graft_entry__ as g; g.build()'`")
    lib = C.CDLL(LIB_PATH)
    lib.gb_abi_version.restype = C.c_int32
    lib.gb_last_error.restype = C.c_char_p
    lib.gb_bsr_to_host.restype = C.c_int
    lib.gb_bsr_to_host.argtypes = [C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                   C.POINTER(C.c_int64), C.POINTER(C.c_int64),
                                   C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
    lib.gb_block_factor_to_host.restype = C.c_int
    lib.gb_block_factor_to_host.argtypes = [C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                            C.POINTER(C.c_int32), C.POINTER(C.c_int64), C.c_void_p]
    lib.gb_build_bsr.restype = C.c_int
    lib.gb_build_bsr.argtypes = [C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                 C.POINTER(C.c_void_p)]
    lib.gb_matrix_get_info.restype = C.c_int
    lib.gb_matrix_get_info.argtypes = [C.c_void_p, C.POINTER(MatrixInfo)]
    lib.gb_free.restype = None
    lib.gb_free.argtypes = [C.c_void_p]
    lib.gb_spmm.restype = C.c_int
    lib.gb_spmm.argtypes = [C.c_void_p, C.c_int32, C.c_int, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p]
    lib.gb_apply_sinv.restype = C.c_int
    lib.gb_apply_sinv.argtypes = [C.c_void_p, C.c_int, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p]
    lib.gb_solve_workspace_size.restype = C.c_size_t
    lib.gb_solve_workspace_size.argtypes = [C.c_void_p, C.POINTER(SolveParams)]
    lib.gb_solve_plan.restype = C.c_int
    lib.gb_solve_plan.argtypes = [C.c_void_p, C.POINTER(SolveParams), C.c_void_p]
    lib.gb_shifted_solve.restype = C.c_int
    lib.gb_shifted_solve.argtypes = [C.c_void_p, C.POINTER(SolveParams), C.POINTER(Outputs), C.c_void_p,
                                     C.c_size_t, C.c_void_p]
    lib.gb_correct_unconverged.restype = C.c_int
    lib.gb_correct_unconverged.argtypes = [C.c_void_p, C.POINTER(SolveParams), C.POINTER(Outputs), C.c_void_p,
                                           C.c_size_t, C.c_void_p, C.POINTER(C.c_int32)]
    lib.gb_correct_workspace_size.restype = C.c_size_t
    lib.gb_correct_workspace_size.argtypes = [C.c_void_p, C.POINTER(SolveParams), C.c_int32]
    lib.gb_true_residual.restype = C.c_int
    lib.gb_true_residual.argtypes = [C.c_void_p, C.POINTER(SolveParams), C.c_int32, C.c_void_p, C.c_void_p,
                                     C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p, C.POINTER(C.c_int32)]
    lib.gb_true_residual_workspace_size.restype = C.c_size_t
    lib.gb_true_residual_workspace_size.argtypes = [C.c_void_p, C.POINTER(SolveParams), C.c_int32]
    lib.gb_correct_batched.restype = C.c_int
    lib.gb_correct_batched.argtypes = [C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_size_t,
                                       C.c_void_p, C.POINTER(C.c_int32)]
    lib.gb_correct_batched_workspace_size.restype = C.c_size_t
    lib.gb_correct_batched_workspace_size.argtypes = [C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
    lib.gb_add_sinv_terms.restype = C.c_int
    lib.gb_add_sinv_terms.argtypes = [C.c_void_p, C.POINTER(SolveParams), C.c_double, C.c_double, C.c_double,
                                      C.POINTER(Outputs), C.c_void_p, C.c_size_t, C.c_void_p]
    lib.gb_add_sinv_terms_workspace_size.restype = C.c_size_t
    lib.gb_add_sinv_terms_workspace_size.argtypes = [C.c_void_p, C.POINTER(SolveParams)]
    lib.gb_wavepacket.restype = C.c_int
    lib.gb_wavepacket.argtypes = [C.c_void_p, C.c_int32, C.c_void_p, C.c_int32, C.c_double, C.c_double, C.c_double,
                                  C.POINTER(C.c_int32), C.c_void_p, C.c_size_t, C.c_void_p]
    lib.gb_wavepacket_workspace_size.restype = C.c_size_t
    lib.gb_wavepacket_workspace_size.argtypes = [C.c_void_p, C.c_int32]
    lib.gb_forces.restype = C.c_int
    lib.gb_forces.argtypes = [C.c_void_p, C.POINTER(SolveParams), C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                              C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p]
    lib.gb_forces_workspace_size.restype = C.c_size_t
    lib.gb_forces_workspace_size.argtypes = [C.c_void_p, C.POINTER(SolveParams), C.c_int32]
    lib.gb_fermi_density.restype = C.c_int
    lib.gb_fermi_density.argtypes = [C.c_void_p, C.POINTER(SolveParams), C.c_void_p, C.c_void_p, C.c_double,
                                     C.c_double, C.c_double, C.POINTER(C.c_double), C.POINTER(Outputs), C.c_void_p,
                                     C.c_size_t, C.c_void_p]
    lib.gb_fermi_workspace_size.restype = C.c_size_t
    lib.gb_fermi_workspace_size.argtypes = [C.c_void_p, C.POINTER(SolveParams)]
    lib.gb_shifted_solve_static.restype = C.c_int
    lib.gb_shifted_solve_static.argtypes = [C.c_void_p, C.POINTER(SolveParams), C.POINTER(Outputs), C.c_void_p]
    lib.gb_static_scratch_bytes.restype = C.c_size_t
    lib.gb_shifted_solve_batched.restype = C.c_int
    lib.gb_shifted_solve_batched.argtypes = [C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32,
                                             C.c_void_p, C.c_size_t, C.c_void_p]
    lib.gb_batched_workspace_size.restype = C.c_size_t
    lib.gb_batched_workspace_size.argtypes = [C.c_int32, C.c_void_p, C.c_void_p, C.c_int32, C.c_int32]
    lib.gb_tune_panel_batched.restype = C.c_int
    lib.gb_tune_panel_batched.argtypes = [C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p,
                                          C.c_size_t, C.c_void_p, C.POINTER(C.c_int32), C.c_void_p]
    _lib = lib
    return lib


def _check(st: int):
    if st != GB_OK:
        raise GBError(st, load().gb_last_error().decode())


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def _csr(system):
    rp = np.ascontiguousarray(system.row_ptr, dtype=np.int64)
    ci = np.ascontiguousarray(system.col_idx, dtype=np.int32)
    hv = np.ascontiguousarray(system.h_val, dtype=np.float64)
    sv = np.ascontiguousarray(system.s_val, dtype=np.float64)
    return int(system.n), rp, ci, hv, sv


def bsr_to_host(system) -> dict:
    """The builder's 4x4 block form of (H, S), computed on the host (no GPU)."""
    lib = load()
    n, rp, ci, hv, sv = _csr(system)
    nb, nnzb = C.c_int64(), C.c_int64()
    _check(lib.gb_bsr_to_host(n, _ptr(rp), _ptr(ci), _ptr(hv), _ptr(sv), C.byref(nb), C.byref(nnzb),
                              None, None, None, None))
    bp = np.zeros(nb.value + 1, np.int32)
    bc = np.zeros(nnzb.value, np.int32)
    bh = np.zeros(nnzb.value * 16, np.float64)
    bs = np.zeros(nnzb.value * 16, np.float64)
    _check(lib.gb_bsr_to_host(n, _ptr(rp), _ptr(ci), _ptr(hv), _ptr(sv), C.byref(nb), C.byref(nnzb),
                              _ptr(bp), _ptr(bc), _ptr(bh), _ptr(bs)))
    return dict(nb=nb.value, nnzb=nnzb.value, blk_ptr=bp, blk_col=bc, blk_h=bh.reshape(-1, 4, 4),
                blk_s=bs.reshape(-1, 4, 4))


def block_factor_to_host(system) -> dict:
    """The block-bidiagonal Cholesky factor of S used by the exact inner solve,
    computed on the host (no GPU): bw and nblk (both 0 if unavailable), and the
    four [nblk, 64, 64] arrays Dinv, DinvT, E, F with entry (r, k) of each
    block at [blk, k, r] (k-major, as stored on the device)."""
    lib = load()
    n, rp, ci, hv, sv = _csr(system)
    bw, nblk = C.c_int32(), C.c_int64()
    _check(lib.gb_block_factor_to_host(n, _ptr(rp), _ptr(ci), _ptr(hv), _ptr(sv), C.byref(bw), C.byref(nblk), None))
    nb_ = int(nblk.value)
    f = np.zeros((4, nb_, 64, 64), np.float64)
    if nb_:
        _check(lib.gb_block_factor_to_host(n, _ptr(rp), _ptr(ci), _ptr(hv), _ptr(sv), C.byref(bw), C.byref(nblk),
                                           _ptr(f)))
    return dict(bw=int(bw.value), nblk=nb_, dinv=f[0], dinvt=f[1], e=f[2], f=f[3])


def _stream_handle(stream):
    import torch

    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


class Matrix:
    """(H, S) resident on the current CUDA device (owns a gb_matrix)."""

    def __init__(self, system, stream=None):
        import torch

        if not torch.cuda.is_available():
            raise RuntimeError("no CUDA device: the library has no CPU path")
        lib = load()
        n, rp, ci, hv, sv = _csr(system)
        h = C.c_void_p()
        _check(lib.gb_build_bsr(n, _ptr(rp), _ptr(ci), _ptr(hv), _ptr(sv), _stream_handle(stream), C.byref(h)))
        self._h = h
        self.system = system
        info = MatrixInfo()
        _check(lib.gb_matrix_get_info(h, C.byref(info)))
        self.info = {f: getattr(info, f) for f, _ in MatrixInfo._fields_}
        self.n = self.info["n"]

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load().gb_free(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def spmm(self, which: int, x, prec: str = "fp64", out=None, stream=None):
        """Y = A X with A = H (which=0) or S (which=1); X complex [n, w] on the GPU."""
        import torch

        dt = torch.complex128 if prec == "fp64" else torch.complex64
        x = x.to(dt).contiguous()
        assert x.is_cuda and x.dim() == 2 and x.shape[0] == self.n
        y = out if out is not None else torch.empty_like(x)
        _check(load().gb_spmm(self._h, int(which), GB_FP64 if prec == "fp64" else GB_MIXED, int(x.shape[1]),
                              C.c_void_p(x.data_ptr()), C.c_void_p(y.data_ptr()), _stream_handle(stream)))
        return y


    def apply_sinv(self, x, prec: str = "fp64", out=None, stream=None):
        """Y = S^-1 X by the exact factor solve; X complex [n, w] on the GPU,
        w in {1, 2, 4, 8, 16, 32} (FP32: one unrefined solve)."""
        import torch

        dt = torch.complex128 if prec == "fp64" else torch.complex64
        x = x.to(dt).contiguous()
        assert x.is_cuda and x.dim() == 2 and x.shape[0] == self.n
        y = out if out is not None else torch.empty_like(x)
        _check(load().gb_apply_sinv(self._h, GB_FP64 if prec == "fp64" else GB_MIXED, int(x.shape[1]),
                                    C.c_void_p(x.data_ptr()), C.c_void_p(y.data_ptr()), _stream_handle(stream)))
        return y


def pattern_offsets(system, cols) -> np.ndarray:
    cols = np.asarray(cols, dtype=np.int64)
    m = system.row_ptr[cols + 1] - system.row_ptr[cols]
    off = np.zeros(len(cols) + 1, dtype=np.int64)
    np.cumsum(m, out=off[1:])
    return off


def _params(z, cols, tol, maxit, prec, w_rho, w_edm, inner_tol, panel, seed_shift, keep, flags=0):
    z = np.asarray(z, dtype=np.complex128)
    zr = np.ascontiguousarray(z.real)
    zi = np.ascontiguousarray(z.imag)
    cols = np.ascontiguousarray(cols, dtype=np.int32)
    keep += [zr, zi, cols]
    p = SolveParams()
    p.nshift = len(z)
    p.z_re = zr.ctypes.data_as(C.POINTER(C.c_double))
    p.z_im = zi.ctypes.data_as(C.POINTER(C.c_double))
    for name, w in (("w_rho", w_rho), ("w_edm", w_edm)):
        if w is None:
            setattr(p, name, C.POINTER(C.c_double)())
        else:
            wv = np.ascontiguousarray(np.asarray(w, dtype=np.complex128).view(np.float64))
            keep.append(wv)
            setattr(p, name, wv.ctypes.data_as(C.POINTER(C.c_double)))
    p.nrhs = len(cols)
    p.rhs_cols = cols.ctypes.data_as(C.POINTER(C.c_int32))
    p.tol = float(tol)
    p.maxit = int(maxit)
    p.prec = GB_FP64 if prec == "fp64" else GB_MIXED
    p.inner_tol = float(inner_tol)
    p.panel = int(panel)
    p.flags = int(flags)
    p.seed_shift = int(seed_shift)
    p.reserved = 0
    return p


def workspace_bytes(mat: Matrix, z, cols, tol=1e-10, maxit=1000, prec="fp64", panel=0) -> int:
    keep = []
    p = _params(z, cols, tol, maxit, prec, None, None, 0.0, panel, -1, keep)
    nb = load().gb_solve_workspace_size(mat.handle, C.byref(p))
    if nb == 0:
        raise GBError(GB_EINVAL, load().gb_last_error().decode())
    return int(nb)


def solve_plan(mat: Matrix, z, cols, tol=1e-10, maxit=1000, prec="fp64", panel=0, flags=0) -> dict:
    """Launch plan of gb_shifted_solve: panel width, teams, shared-memory use."""
    keep = []
    p = _params(z, cols, tol, maxit, prec, None, None, 0.0, panel, -1, keep, flags)
    plan = np.zeros(6, np.int32)
    _check(load().gb_solve_plan(mat.handle, C.byref(p), _ptr(plan)))
    return dict(panel=int(plan[0]), teams=int(plan[1]), cg_smem=bool(plan[2]), dyn_smem=int(plan[3]),
                inner=("cg", "chebyshev", "factor")[int(plan[4])], teams_per_sm=int(plan[5]))


def shifted_solve(mat: Matrix, z, cols, tol=1e-10, maxit=1000, prec="fp64", w_rho=None, w_edm=None,
                  inner_tol=0.0, panel=0, seed_shift=-1, want_g=False, workspace=None, stream=None, flags=0,
                  raise_on=(GB_EINVAL, GB_ENOMEM, GB_ECUDA, GB_ENOTSPD), correct=False, verify=None):
    """Solve (z_k S - H) x = e_j for all shifts and columns; returns device tensors.

    Keys: ldos [K, nrhs], rho / edm [P], q / e_loc [nrhs], iters [nrhs],
    converged [K, nrhs] (uint8), resid [K, nrhs], g_proj [K, P] complex (if
    want_g), off [nrhs+1] (host, packed offsets), status (int).

    ``verify``: indices into ``cols`` (or True for all) whose FP64 true
    residual is checked after the solve (gb_true_residual); ``resid_true``
    [K, len(verify)] then holds it, and columns that miss tol become
    unconverged in the outputs.  With ``correct=True`` a GB_ENOCONV result
    (from the solve or the check) is passed to gb_correct_batched (one FP64
    re-solve of all failing columns, then seed switching for the rest);
    ``corrected`` then holds the number of columns it fixed, and the first
    solve stops stalled columns early (flags bit 6).
    """
    import torch

    if correct:
        flags |= FLAG_STALL
    dev = torch.device("cuda", torch.cuda.current_device())
    keep = []
    p = _params(z, cols, tol, maxit, prec, w_rho, w_edm, inner_tol, panel, seed_shift, keep, flags)
    K, nrhs = p.nshift, p.nrhs
    lib = load()
    need = lib.gb_solve_workspace_size(mat.handle, C.byref(p))  # validates every parameter
    if need == 0:
        raise GBError(GB_EINVAL, lib.gb_last_error().decode())
    off = pattern_offsets(mat.system, cols)
    P = int(off[-1])
    f64 = dict(dtype=torch.float64, device=dev)
    res = dict(
        ldos=torch.empty((K, nrhs), **f64),
        rho=torch.empty(P, **f64) if w_rho is not None else None,
        edm=torch.empty(P, **f64) if w_edm is not None else None,
        q=torch.empty(nrhs, **f64) if w_rho is not None else None,
        e_loc=torch.empty(nrhs, **f64) if w_rho is not None else None,
        iters=torch.empty(nrhs, dtype=torch.int32, device=dev),
        converged=torch.empty((K, nrhs), dtype=torch.uint8, device=dev),
        resid=torch.empty((K, nrhs), **f64),
        g_proj=torch.empty((K, P), dtype=torch.complex128, device=dev) if want_g else None,
        inner_iters=torch.empty(nrhs, dtype=torch.int32, device=dev),
        col_status=torch.empty(nrhs, dtype=torch.int32, device=dev),
    )
    o = Outputs()
    for f, _ in Outputs._fields_:
        t = res[f]
        setattr(o, f, C.c_void_p(t.data_ptr()) if t is not None else None)
    if workspace is None or workspace.numel() < need:
        workspace = torch.empty(int(need), dtype=torch.uint8, device=dev)
    st = lib.gb_shifted_solve(mat.handle, C.byref(p), C.byref(o), C.c_void_p(workspace.data_ptr()),
                              C.c_size_t(workspace.numel()), _stream_handle(stream))
    if st in raise_on:
        _check(st)
    res["status"] = st
    res["message"] = lib.gb_last_error().decode()
    res["off"] = off
    res["workspace"] = workspace
    if verify is not None and st in (GB_OK, GB_ENOCONV):
        ver = np.arange(nrhs, dtype=np.int32) if verify is True else np.ascontiguousarray(verify, dtype=np.int32)
        nver = len(ver)
        vneed = lib.gb_true_residual_workspace_size(mat.handle, C.byref(p), nver)
        if vneed == 0:
            raise GBError(GB_EINVAL, lib.gb_last_error().decode())
        vws = torch.empty(int(vneed), dtype=torch.uint8, device=dev)
        rtrue = torch.empty((K, nver), dtype=torch.float64, device=dev)
        nflag = C.c_int32(0)
        vst = lib.gb_true_residual(mat.handle, C.byref(p), nver, _ptr(ver), C.c_void_p(rtrue.data_ptr()),
                                   C.byref(o), C.c_void_p(vws.data_ptr()), C.c_size_t(vws.numel()),
                                   _stream_handle(stream), C.byref(nflag))
        _check(vst)
        del vws
        res["resid_true"] = rtrue
        res["verified"] = ver
        res["flagged"] = int(nflag.value)
        if nflag.value > 0:
            st = GB_ENOCONV
            res["status"] = st
            res["message"] = f"{nflag.value} checked column(s) miss tol by their true residual"
    if correct and st == GB_ENOCONV:
        h1 = (C.c_void_p * 1)(mat.handle.value)
        p1 = (SolveParams * 1)(p)
        o1 = (Outputs * 1)(o)
        sh = _stream_handle(stream)
        cneed = lib.gb_correct_batched_workspace_size(1, h1, p1, o1, sh)
        if cneed == 0:
            raise GBError(GB_EINVAL, lib.gb_last_error().decode())
        cws = workspace if workspace.numel() >= cneed else torch.empty(int(cneed), dtype=torch.uint8, device=dev)
        fixed = C.c_int32(0)
        st = lib.gb_correct_batched(1, h1, p1, o1, C.c_void_p(cws.data_ptr()), C.c_size_t(cws.numel()), sh,
                                    C.byref(fixed))
        if st in raise_on:
            _check(st)
        res["status"] = st
        res["message"] = lib.gb_last_error().decode()
        res["corrected"] = int(fixed.value)
    return res


def fermi_density(mat: Matrix, z, cols, solved: dict, n_electrons: float, kT: float, spin: float = 2.0,
                  stream=None) -> dict:
    """Chemical potential and Fermi-weighted rho / edm / q / e_loc from a
    finished solve of every orbital (``solved`` = the result of
    :func:`shifted_solve` with ``want_g=True``): gb_fermi_density."""
    import torch

    if solved.get("g_proj") is None:
        raise ValueError("the solve must keep g_proj (want_g=True)")
    dev = torch.device("cuda", torch.cuda.current_device())
    keep = []
    p = _params(z, cols, 1e-10, 1, "fp64", None, None, 0.0, 0, -1, keep)
    lib = load()
    need = lib.gb_fermi_workspace_size(mat.handle, C.byref(p))
    if need == 0:
        raise GBError(GB_EINVAL, lib.gb_last_error().decode())
    ws = torch.empty(int(need), dtype=torch.uint8, device=dev)
    P = int(solved["off"][-1])
    nrhs = p.nrhs
    f64 = dict(dtype=torch.float64, device=dev)
    res = dict(rho=torch.empty(P, **f64), edm=torch.empty(P, **f64), q=torch.empty(nrhs, **f64),
               e_loc=torch.empty(nrhs, **f64))
    o = Outputs()
    for f, _ in Outputs._fields_:
        t = res.get(f)
        setattr(o, f, C.c_void_p(t.data_ptr()) if t is not None else None)
    mu = C.c_double(0.0)
    _check(lib.gb_fermi_density(mat.handle, C.byref(p), C.c_void_p(solved["g_proj"].data_ptr()),
                                C.c_void_p(solved["ldos"].data_ptr()), float(n_electrons), float(kT), float(spin),
                                C.byref(mu), C.byref(o), C.c_void_p(ws.data_ptr()), C.c_size_t(ws.numel()),
                                _stream_handle(stream)))
    res["mu"] = float(mu.value)
    res["off"] = solved["off"]
    return res


def add_sinv_terms(mat: Matrix, cols, solved: dict, a_rho: float, b_edm: float, c_shs: float, stream=None) -> dict:
    """Add a_rho S^-1 to rho and b_edm S^-1 + c_shs S^-1 H S^-1 to P^E on the
    pattern of ``cols`` (the outputs of :func:`shifted_solve`, updated in place;
    q and e_loc recomputed): gb_add_sinv_terms."""
    import torch

    dev = torch.device("cuda", torch.cuda.current_device())
    keep = []
    z = np.zeros(1, dtype=np.complex128) + 1j
    p = _params(z, cols, 1e-10, 1, "fp64", None, None, 0.0, 0, -1, keep)
    lib = load()
    need = lib.gb_add_sinv_terms_workspace_size(mat.handle, C.byref(p))
    if need == 0:
        raise GBError(GB_EINVAL, lib.gb_last_error().decode())
    ws = torch.empty(int(need), dtype=torch.uint8, device=dev)
    o = Outputs()
    for f, _ in Outputs._fields_:
        t = solved.get(f) if f in ("rho", "edm", "q", "e_loc") else None
        setattr(o, f, C.c_void_p(t.data_ptr()) if t is not None else None)
    _check(lib.gb_add_sinv_terms(mat.handle, C.byref(p), float(a_rho), float(b_edm), float(c_shs), C.byref(o),
                                 C.c_void_p(ws.data_ptr()), C.c_size_t(ws.numel()), _stream_handle(stream)))
    return solved


def wavepacket(mat: Matrix, psi, nsteps: int, tau: float, e_min: float, e_max: float, stream=None):
    """Propagate the columns of ``psi`` (complex128 device tensor [n, w], in
    place) by ``nsteps`` steps exp(-i tau S^-1 H) (gb_wavepacket); returns
    (psi, terms per step)."""
    import torch

    dev = torch.device("cuda", torch.cuda.current_device())
    if psi.dtype != torch.complex128 or not psi.is_contiguous() or psi.dim() != 2:
        raise ValueError("psi must be a contiguous complex128 [n, w] tensor")
    lib = load()
    nwp = int(psi.shape[1])
    need = lib.gb_wavepacket_workspace_size(mat.handle, nwp)
    if need == 0:
        raise GBError(GB_EINVAL, lib.gb_last_error().decode())
    ws = torch.empty(int(need), dtype=torch.uint8, device=dev)
    nt = C.c_int32(0)
    _check(lib.gb_wavepacket(mat.handle, nwp, C.c_void_p(psi.data_ptr()), int(nsteps), float(tau), float(e_min),
                             float(e_max), C.byref(nt), C.c_void_p(ws.data_ptr()), C.c_size_t(ws.numel()),
                             _stream_handle(stream)))
    return psi, int(nt.value)


def forces(mat: Matrix, cols, rho, edm, grad_h, grad_s, atom_off, stream=None):
    """Atomic forces [n_atoms, 3] (gb_forces) from packed rho / P^E (device
    tensors of a solve of every orbital in ``cols``), per-element gradients
    grad_h, grad_s [3, nnz] (CSR order, numpy or device tensors) and the
    orbital ranges of the atoms ``atom_off`` [n_atoms + 1]."""
    import torch

    dev = torch.device("cuda", torch.cuda.current_device())
    keep = []
    z = np.zeros(1, dtype=np.complex128) + 1j
    p = _params(z, cols, 1e-10, 1, "fp64", None, None, 0.0, 0, -1, keep)
    ao = np.ascontiguousarray(atom_off, dtype=np.int64)
    n_atoms = len(ao) - 1
    lib = load()
    need = lib.gb_forces_workspace_size(mat.handle, C.byref(p), n_atoms)
    if need == 0:
        raise GBError(GB_EINVAL, lib.gb_last_error().decode())
    ws = torch.empty(int(need), dtype=torch.uint8, device=dev)
    f64 = dict(dtype=torch.float64, device=dev)
    gh = torch.as_tensor(np.ascontiguousarray(grad_h) if isinstance(grad_h, np.ndarray) else grad_h, **f64).contiguous()
    gs = torch.as_tensor(np.ascontiguousarray(grad_s) if isinstance(grad_s, np.ndarray) else grad_s, **f64).contiguous()
    out = torch.empty((n_atoms, 3), **f64)
    _check(lib.gb_forces(mat.handle, C.byref(p), C.c_void_p(rho.data_ptr()), C.c_void_p(edm.data_ptr()),
                         C.c_void_p(gh.data_ptr()), C.c_void_p(gs.data_ptr()), _ptr(ao), n_atoms,
                         C.c_void_p(out.data_ptr()), C.c_void_p(ws.data_ptr()), C.c_size_t(ws.numel()),
                         _stream_handle(stream)))
    return out


def true_residual(mat: Matrix, z, cols, verify, tol=1e-10, maxit=1000, prec="fp64", inner_tol=0.0, panel=0,
                  seed_shift=-1, flags=0, stream=None):
    """FP64 true residuals ||e_j - (z_k S - H) x^k|| [K, len(verify)] of the
    columns cols[verify] as the solve with these parameters produces them
    (gb_true_residual: the columns are re-run with their full history)."""
    import torch

    dev = torch.device("cuda", torch.cuda.current_device())
    keep = []
    p = _params(z, cols, tol, maxit, prec, None, None, inner_tol, panel, seed_shift, keep, flags)
    lib = load()
    ver = np.ascontiguousarray(verify, dtype=np.int32)
    need = lib.gb_true_residual_workspace_size(mat.handle, C.byref(p), len(ver))
    if need == 0:
        raise GBError(GB_EINVAL, lib.gb_last_error().decode())
    ws = torch.empty(int(need), dtype=torch.uint8, device=dev)
    out = torch.empty((p.nshift, len(ver)), dtype=torch.float64, device=dev)
    _check(lib.gb_true_residual(mat.handle, C.byref(p), len(ver), _ptr(ver), C.c_void_p(out.data_ptr()), None,
                                C.c_void_p(ws.data_ptr()), C.c_size_t(ws.numel()), _stream_handle(stream), None))
    return out


def shifted_solve_static(mat: Matrix, z, cols, tol=1e-10, maxit=1000, prec="fp64", w_rho=None, w_edm=None,
                         inner_tol=0.0, panel=0, seed_shift=-1, want_g=False, stream=None, flags=0):
    """Like :func:`shifted_solve`, through gb_shifted_solve_static (no scratch
    allocation: the library's fixed per-device scratch is used)."""
    import torch

    dev = torch.device("cuda", torch.cuda.current_device())
    keep = []
    p = _params(z, cols, tol, maxit, prec, w_rho, w_edm, inner_tol, panel, seed_shift, keep, flags)
    K, nrhs = p.nshift, p.nrhs
    lib = load()
    if lib.gb_solve_workspace_size(mat.handle, C.byref(p)) == 0:  # validates the parameters
        raise GBError(GB_EINVAL, lib.gb_last_error().decode())
    off = pattern_offsets(mat.system, cols)
    P = int(off[-1])
    f64 = dict(dtype=torch.float64, device=dev)
    res = dict(
        ldos=torch.empty((K, nrhs), **f64),
        rho=torch.empty(P, **f64) if w_rho is not None else None,
        edm=torch.empty(P, **f64) if w_edm is not None else None,
        q=torch.empty(nrhs, **f64) if w_rho is not None else None,
        e_loc=torch.empty(nrhs, **f64) if w_rho is not None else None,
        iters=torch.empty(nrhs, dtype=torch.int32, device=dev),
        converged=torch.empty((K, nrhs), dtype=torch.uint8, device=dev),
        resid=torch.empty((K, nrhs), **f64),
        g_proj=torch.empty((K, P), dtype=torch.complex128, device=dev) if want_g else None,
        inner_iters=torch.empty(nrhs, dtype=torch.int32, device=dev),
        col_status=torch.empty(nrhs, dtype=torch.int32, device=dev),
    )
    o = Outputs()
    for f, _ in Outputs._fields_:
        t = res[f]
        setattr(o, f, C.c_void_p(t.data_ptr()) if t is not None else None)
    st = lib.gb_shifted_solve_static(mat.handle, C.byref(p), C.byref(o), _stream_handle(stream))
    res["status"] = st
    res["message"] = lib.gb_last_error().decode()
    res["off"] = off
    return res


def _alloc_outputs(mat, K, cols, w_rho, w_edm, want_g, dev):
    import torch

    nrhs = len(cols)
    off = pattern_offsets(mat.system, cols)
    P = int(off[-1])
    f64 = dict(dtype=torch.float64, device=dev)
    res = dict(
        ldos=torch.empty((K, nrhs), **f64),
        rho=torch.empty(P, **f64) if w_rho is not None else None,
        edm=torch.empty(P, **f64) if w_edm is not None else None,
        q=torch.empty(nrhs, **f64) if w_rho is not None else None,
        e_loc=torch.empty(nrhs, **f64) if w_rho is not None else None,
        iters=torch.empty(nrhs, dtype=torch.int32, device=dev),
        converged=torch.empty((K, nrhs), dtype=torch.uint8, device=dev),
        resid=torch.empty((K, nrhs), **f64),
        g_proj=torch.empty((K, P), dtype=torch.complex128, device=dev) if want_g else None,
        inner_iters=torch.empty(nrhs, dtype=torch.int32, device=dev),
        col_status=torch.empty(nrhs, dtype=torch.int32, device=dev),
    )
    o = Outputs()
    for f, _ in Outputs._fields_:
        t = res[f]
        setattr(o, f, C.c_void_p(t.data_ptr()) if t is not None else None)
    res["off"] = off
    return res, o


def shifted_solve_batched(mats, problems, prec="mixed", panel=0, want_g=False, workspace=None, stream=None,
                          tune_probe_maxit=0, correct=False, flags=0):
    """Solve many independent systems in one persistent launch.

    ``problems`` is a list of dicts with keys z, cols, tol, maxit and optional
    w_rho, w_edm (one per matrix in ``mats``).  With ``tune_probe_maxit > 0``
    the panel width is first picked by the library's autotuner
    (gb_tune_panel_batched) on probe runs of that many iterations.  With
    ``correct=True`` a GB_ENOCONV batch goes to gb_correct_batched (one FP64
    launch over every failing column, then seed switching where needed).  Returns a list of per-system result dicts plus the
    batch status/message/panel (and ``corrected`` columns).
    """
    import torch

    if correct:
        flags |= FLAG_STALL
    dev = torch.device("cuda", torch.cuda.current_device())
    lib = load()
    nsys = len(mats)
    keep = []
    params = (SolveParams * nsys)()
    outs = (Outputs * nsys)()
    results = []
    for s_, (mat, pr) in enumerate(zip(mats, problems)):
        p = _params(pr["z"], pr["cols"], pr["tol"], pr["maxit"], prec, pr.get("w_rho"), pr.get("w_edm"), 0.0,
                    panel, -1, keep, flags)
        params[s_] = p
        res, o = _alloc_outputs(mat, len(pr["z"]), pr["cols"], pr.get("w_rho"), pr.get("w_edm"), want_g, dev)
        outs[s_] = o
        results.append(res)
    handles = (C.c_void_p * nsys)(*[m.handle.value for m in mats])
    info = {}
    if tune_probe_maxit > 0:
        probe = (SolveParams * nsys)(*params)
        for q in range(nsys):
            probe[q].maxit = min(probe[q].maxit, tune_probe_maxit)
        need = max(lib.gb_batched_workspace_size(nsys, handles, probe, w, int(want_g)) for w in (8, 16, 32))
        tws = torch.empty(int(need), dtype=torch.uint8, device=dev)
        best = C.c_int32()
        times = np.zeros(3, np.float32)
        _check(lib.gb_tune_panel_batched(nsys, handles, probe, outs, int(tune_probe_maxit),
                                         C.c_void_p(tws.data_ptr()), C.c_size_t(tws.numel()),
                                         _stream_handle(stream), C.byref(best), _ptr(times)))
        panel = int(best.value)
        info["tuned_panel"] = panel
        info["tune_times_ms"] = times.tolist()
        del tws
    need = lib.gb_batched_workspace_size(nsys, handles, params, int(panel), int(want_g))
    if need == 0:
        raise GBError(GB_EINVAL, lib.gb_last_error().decode())
    if workspace is None or workspace.numel() < need:
        workspace = torch.empty(int(need), dtype=torch.uint8, device=dev)
    st = lib.gb_shifted_solve_batched(nsys, handles, params, outs, int(panel), C.c_void_p(workspace.data_ptr()),
                                      C.c_size_t(workspace.numel()), _stream_handle(stream))
    if st in (GB_EINVAL, GB_ENOMEM, GB_ECUDA):
        _check(st)
    msg = lib.gb_last_error().decode()
    if correct and st == GB_ENOCONV:
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        sh = _stream_handle(stream)
        cneed = lib.gb_correct_batched_workspace_size(nsys, handles, params, outs, sh)
        if cneed == 0:
            raise GBError(GB_EINVAL, lib.gb_last_error().decode())
        if workspace.numel() < cneed:
            workspace = torch.empty(int(cneed), dtype=torch.uint8, device=dev)
        fixed = C.c_int32(0)
        st = lib.gb_correct_batched(nsys, handles, params, outs, C.c_void_p(workspace.data_ptr()),
                                    C.c_size_t(workspace.numel()), sh, C.byref(fixed))
        if st not in (GB_OK, GB_ENOCONV):
            _check(st)
        e1.record()
        torch.cuda.synchronize()
        msg = "" if st == GB_OK else lib.gb_last_error().decode()
        info["corrected"] = int(fixed.value)
        info["correct_ms"] = e0.elapsed_time(e1)
    info.update(status=st, message=msg, panel=panel, workspace=workspace)
    return results, info
