"""Learned surrogate for the local charge and local energy, with the solver as judge.

A 64-float environment descriptor per orbital (``gb_descriptors``) feeds an MLP
64 -> 128 -> 128 -> 128 -> 2 (GELU, BF16 weights, FP32 accumulation) whose
forward, backward and Adam steps are the library's CUDA kernels
(``include/gbgreen_surrogate.h``).  The labels (q_j, E_j) are produced by the
shifted solver itself; at inference the solver re-solves a random sample of
the orbitals (the judge) plus every orbital whose descriptor lies outside the
training range (the fallback), and replaces the sampled predictions that miss
by more than the error threshold.  Python only marshals arguments and drives
the loop; the arithmetic runs in the kernels.
"""
from __future__ import annotations

import ctypes as C
import time

import numpy as np

from ._binding import GBError, Matrix, _check, _stream_handle, load, shifted_solve, shifted_solve_batched

DESC = 64
LAYERS = 4


class _MLPStruct(C.Structure):
    _fields_ = [("dims", C.c_int32 * (LAYERS + 1))] + [
        (f, C.c_void_p * LAYERS) for f in ("w", "w_bf16", "b", "gw", "gb", "mw", "vw", "mb", "vb")
    ]


def _lib():
    lib = load()
    if not getattr(lib, "_surrogate_ready", False):
        lib.gb_descriptors.restype = C.c_int
        lib.gb_descriptors.argtypes = [C.c_void_p, C.c_int32] + [C.c_void_p] * 5 + [C.c_void_p]
        lib.gb_mlp_workspace_size.restype = C.c_size_t
        lib.gb_mlp_workspace_size.argtypes = [C.c_void_p, C.c_int32]
        lib.gb_mlp_forward.restype = C.c_int
        lib.gb_mlp_forward.argtypes = [C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p, C.c_size_t,
                                       C.c_void_p]
        lib.gb_mlp_backward.restype = C.c_int
        lib.gb_mlp_backward.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p, C.c_size_t,
                                        C.c_void_p]
        lib.gb_mse_grad.restype = C.c_int
        lib.gb_mse_grad.argtypes = [C.c_void_p, C.c_void_p, C.c_int32, C.c_int32, C.c_void_p, C.c_void_p,
                                    C.POINTER(C.c_int32), C.c_void_p]
        lib.gb_mlp_adam.restype = C.c_int
        lib.gb_mlp_adam.argtypes = [C.c_void_p, C.c_float, C.c_float, C.c_float, C.c_float, C.c_int32, C.c_void_p]
        lib.gb_mlp_sync_bf16.restype = C.c_int
        lib.gb_mlp_sync_bf16.argtypes = [C.c_void_p, C.c_void_p]
        lib.gb_affine_cols.restype = C.c_int
        lib.gb_affine_cols.argtypes = [C.c_void_p, C.c_int32, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p]
        lib._surrogate_ready = True
    return lib


def _p(t):
    return C.c_void_p(t.data_ptr())


def descriptors(mat: Matrix, system, stream=None):
    """[n, 64] float32 device tensor of per-orbital environment descriptors."""
    import torch

    dev = torch.device("cuda", torch.cuda.current_device())
    lib = _lib()
    first = np.zeros(len(system.atom_norb) + 1, dtype=np.int32)
    np.cumsum(system.atom_norb, out=first[1:])
    species = (system.atom_norb == 1).astype(np.int32)  # 1-orbital atoms are hydrogens
    pos = torch.as_tensor(np.ascontiguousarray(system.positions, dtype=np.float32), device=dev)
    oa = torch.as_tensor(np.ascontiguousarray(system.orb_atom, dtype=np.int32), device=dev)
    fa = torch.as_tensor(first, device=dev)
    sp = torch.as_tensor(species, device=dev)
    out = torch.empty((system.n, DESC), dtype=torch.float32, device=dev)
    _check(lib.gb_descriptors(mat.handle, len(system.atom_norb), _p(pos), _p(oa), _p(fa), _p(sp), _p(out),
                              _stream_handle(stream)))
    return out


def affine_cols(X, scale, shift, stream=None):
    """In place X[:, c] = X[:, c] * scale[c] + shift[c] (device tensors)."""
    _check(_lib().gb_affine_cols(_p(X), X.shape[0], X.shape[1], _p(scale), _p(shift), _stream_handle(stream)))
    return X


class MLP:
    """The surrogate network; parameters, gradients and Adam moments on the GPU."""

    def __init__(self, dims=(DESC, 128, 128, 128, 2), seed=0):
        import torch

        self.dims = tuple(int(d) for d in dims)
        dev = torch.device("cuda", torch.cuda.current_device())
        rng = np.random.default_rng(seed)
        f32 = dict(dtype=torch.float32, device=dev)
        self.w, self.wb, self.b = [], [], []
        self.gw, self.gb, self.mw, self.vw, self.mb, self.vb = [], [], [], [], [], []
        for l in range(LAYERS):
            nin, nout = self.dims[l], self.dims[l + 1]
            std = np.sqrt((2.0 if l < LAYERS - 1 else 1.0) / nin)
            self.w.append(torch.as_tensor(rng.normal(0.0, std, (nout, nin)).astype(np.float32), device=dev))
            self.wb.append(torch.empty((nout, nin), dtype=torch.int16, device=dev))
            self.b.append(torch.zeros(nout, **f32))
            self.gw.append(torch.zeros((nout, nin), **f32))
            self.gb.append(torch.zeros(nout, **f32))
            self.mw.append(torch.zeros((nout, nin), **f32))
            self.vw.append(torch.zeros((nout, nin), **f32))
            self.mb.append(torch.zeros(nout, **f32))
            self.vb.append(torch.zeros(nout, **f32))
        s = _MLPStruct()
        for l in range(LAYERS + 1):
            s.dims[l] = self.dims[l]
        for name in ("w", "b", "gw", "gb", "mw", "vw", "mb", "vb"):
            arr = getattr(s, name)
            for l, t in enumerate(getattr(self, name)):
                arr[l] = t.data_ptr()
        for l, t in enumerate(self.wb):
            s.w_bf16[l] = t.data_ptr()
        self._s = s
        self.step = 0
        self._ws = None
        self._partial = torch.empty(4096, **f32)
        self.sync_bf16()

    def sync_bf16(self):
        _check(_lib().gb_mlp_sync_bf16(C.byref(self._s), _stream_handle(None)))

    def _workspace(self, batch):
        import torch

        need = _lib().gb_mlp_workspace_size(C.byref(self._s), batch)
        if self._ws is None or self._ws.numel() * 4 < need:
            self._ws = torch.empty((need + 3) // 4, dtype=torch.float32, device=self.w[0].device)
        return self._ws

    def forward(self, X):
        import torch

        B = X.shape[0]
        Y = torch.empty((B, self.dims[-1]), dtype=torch.float32, device=X.device)
        ws = self._workspace(B)
        _check(_lib().gb_mlp_forward(C.byref(self._s), _p(X), B, _p(Y), _p(ws), C.c_size_t(ws.numel() * 4),
                                     _stream_handle(None)))
        return Y

    def backward(self, X, dY):
        ws = self._workspace(X.shape[0])
        _check(_lib().gb_mlp_backward(C.byref(self._s), _p(X), _p(dY), X.shape[0], _p(ws),
                                      C.c_size_t(ws.numel() * 4), _stream_handle(None)))

    def train_step(self, X, T, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
        """One Adam step on the mean-squared error; returns the loss (host float)."""
        import torch

        lib = _lib()
        Y = self.forward(X)
        dY = torch.empty_like(Y)
        npart = C.c_int32()
        _check(lib.gb_mse_grad(_p(Y), _p(T), X.shape[0], Y.shape[1], _p(dY), _p(self._partial), C.byref(npart),
                               _stream_handle(None)))
        self.backward(X, dY)
        self.step += 1
        _check(lib.gb_mlp_adam(C.byref(self._s), lr, beta1, beta2, eps, self.step, _stream_handle(None)))
        return self._partial[: npart.value]

    def numpy_params(self):
        return [w.cpu().numpy() for w in self.w], [b.cpu().numpy() for b in self.b]


class Surrogate:
    """Standardisation + MLP; predicts (q_j, E_j) from descriptors."""

    def __init__(self, seed=0):
        self.net = MLP(seed=seed)
        self.x_scale = self.x_shift = self.y_scale = self.y_shift = None

    def fit(self, X, Y, epochs=40, batch=2048, lr=2e-3, seed=0, log=None):
        """X [n, 64] and Y [n, 2] device float32 tensors (not modified)."""
        import torch

        dev = X.device
        xm = X.mean(0)
        xs = X.std(0)
        xs = torch.where(xs > 1e-8, xs, torch.ones_like(xs))
        ym = Y.mean(0)
        ys = Y.std(0)
        ys = torch.where(ys > 1e-12, ys, torch.ones_like(ys))
        self.x_scale, self.x_shift = (1.0 / xs).contiguous(), (-xm / xs).contiguous()
        self.y_scale, self.y_shift = ys.contiguous(), ym.contiguous()
        Xs = affine_cols(X.clone(), self.x_scale, self.x_shift)
        Ys = affine_cols(Y.clone(), (1.0 / ys).contiguous(), (-ym / ys).contiguous())
        self.x_abs_max = Xs.abs().max(0).values
        g = torch.Generator(device=dev)
        g.manual_seed(seed)
        n = X.shape[0]
        history = []
        for ep in range(epochs):
            perm = torch.randperm(n, device=dev, generator=g)
            rate = lr * 0.5 * (1.0 + np.cos(np.pi * ep / epochs))  # cosine schedule
            tot = torch.zeros((), device=dev)
            nb = 0
            for s in range(0, n - batch + 1, batch):
                idx = perm[s : s + batch]
                part = self.net.train_step(Xs[idx].contiguous(), Ys[idx].contiguous(), lr=rate)
                tot += part.sum()
                nb += 1
            history.append(float(tot) / max(nb, 1))
            if log:
                log(f"epoch {ep}: loss {history[-1]:.4e}")
        return history

    def predict(self, X):
        """Physical-unit predictions [n, 2] for descriptors X [n, 64]."""
        Xs = affine_cols(X.clone(), self.x_scale, self.x_shift)
        Y = self.net.forward(Xs)
        return affine_cols(Y, self.y_scale, self.y_shift)

    def out_of_range(self, X, factor=1.5):
        """Boolean mask of rows whose standardised features exceed the training range."""
        Xs = affine_cols(X.clone(), self.x_scale, self.x_shift)
        return (Xs.abs() > factor * self.x_abs_max + 1e-6).any(1)


def solve_local_outputs(mats, systems, z, w_rho, w_edm, tol, maxit, cols_list=None, prec="mixed"):
    """(q, E) for the requested columns of each system through one batched launch."""
    problems = []
    for k, sysm in enumerate(systems):
        cols = np.arange(sysm.n, dtype=np.int32) if cols_list is None else np.asarray(cols_list[k], np.int32)
        problems.append(dict(z=z, cols=cols, w_rho=w_rho, w_edm=w_edm, tol=tol, maxit=maxit))
    res, info = shifted_solve_batched(mats, problems, prec=prec)
    if info["status"] not in (0,):
        raise GBError(info["status"], info["message"])
    return [(r["q"], r["e_loc"]) for r in res]


def infer_with_judge(sur: Surrogate, mat: Matrix, system, z, w_rho, w_edm, tol, maxit, sample_frac=0.05,
                     threshold=1e-3, seed=0):
    """Surrogate predictions for every orbital, judged and repaired by the solver.

    A random ``sample_frac`` of the orbitals plus every out-of-range orbital is
    re-solved; re-solved values replace predictions, and if more than a tenth
    of the sample misses by more than ``threshold`` (absolute, in the output
    units) every orbital is solved instead.  Returns (q, E, report).
    """
    import torch

    t0 = time.perf_counter()
    X = descriptors(mat, system)
    pred = sur.predict(X)
    oor = sur.out_of_range(X).cpu().numpy()
    torch.cuda.synchronize()
    t_pred = time.perf_counter() - t0
    rng = np.random.default_rng(seed)
    n = system.n
    sample = rng.choice(n, size=max(1, int(round(sample_frac * n))), replace=False)
    resolve = np.unique(np.concatenate([sample, np.nonzero(oor)[0]])).astype(np.int32)
    out = shifted_solve(mat, z, resolve, tol=tol, maxit=maxit, prec="mixed", w_rho=w_rho, w_edm=w_edm,
                        raise_on=(-1, -2, -3, -4))
    torch.cuda.synchronize()
    t_judge = time.perf_counter() - t0 - t_pred
    q = pred[:, 0].clone()
    e = pred[:, 1].clone()
    rq = out["q"].float()
    re = out["e_loc"].float()
    pos = {int(j): k for k, j in enumerate(resolve)}
    sidx = torch.as_tensor([pos[int(j)] for j in sample], device=q.device)
    samp = torch.as_tensor(sample, device=q.device)
    err_q = (q[samp] - rq[sidx]).abs()
    err_e = (e[samp] - re[sidx]).abs()
    miss = ((err_q > threshold) | (err_e > threshold)).float().mean().item()
    fell_back = miss > 0.1
    if fell_back:
        full = shifted_solve(mat, z, np.arange(n, dtype=np.int32), tol=tol, maxit=maxit, prec="mixed", w_rho=w_rho,
                             w_edm=w_edm, raise_on=(-1, -2, -3, -4))
        q, e = full["q"].float(), full["e_loc"].float()
    else:
        ridx = torch.as_tensor(resolve, device=q.device)
        q[ridx] = rq
        e[ridx] = re
    torch.cuda.synchronize()
    report = dict(n=n, resolved=int(len(resolve)), out_of_range=int(oor.sum()), sample=int(len(sample)),
                  sample_mae_q=float(err_q.mean()), sample_mae_e=float(err_e.mean()),
                  sample_max_q=float(err_q.max()), sample_max_e=float(err_e.max()), sample_miss_frac=miss,
                  fell_back=bool(fell_back), t_predict_s=t_pred, t_judge_s=t_judge,
                  t_total_s=time.perf_counter() - t0)
    return q, e, report
